// Autotuner for batched forests (an addition to the paper's method, which
// fixes N_down = N_up = 2 and one box size per run): times afg_forest_solve
// for each candidate forest (the same problems built with different box
// sizes) and each pair of smoothing steps, and reports the configuration
// with the most unknowns per second.
#include <algorithm>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <string>
#include <vector>

#include "../../include/afgpu.h"
#include "handles.h"

namespace {

// the integers of a JSON array value following "key": nested brackets are
// flattened ([[1,1],[2,2]] -> 1 1 2 2); an absent key leaves `out` empty
bool json_ints(const char *js, const char *key, std::vector<int> &out, std::string &err) {
    out.clear();
    if (!js) return true;
    const std::string k = std::string("\"") + key + "\"";
    const char *p = std::strstr(js, k.c_str());
    if (!p) return true;
    p += k.size();
    while (*p == ' ' || *p == '\t' || *p == '\n' || *p == '\r') ++p;
    if (*p != ':') { err = std::string("expected ':' after ") + k; return false; }
    ++p;
    while (*p == ' ' || *p == '\t' || *p == '\n' || *p == '\r') ++p;
    int depth = 0;
    do {
        if (*p == '[') ++depth;
        else if (*p == ']') --depth;
        else if ((*p >= '0' && *p <= '9') || *p == '-') {
            char *end = nullptr;
            const long v = std::strtol(p, &end, 10);
            out.push_back((int)v);
            p = end;
            if (depth == 0) return true;  // a plain number
            continue;
        } else if (*p == '\0') { err = "unterminated array for " + k; return false; }
        else if (!(*p == ',' || *p == ' ' || *p == '\t' || *p == '\n' || *p == '\r')) {
            err = "unexpected character in the value of " + k;
            return false;
        }
        ++p;
    } while (depth > 0);
    return true;
}

struct Row {
    int cand, box_n, nd, nu, tpb, max_cycles;
    double ms, unknowns, worst;
    bool converged;
};

}  // namespace

extern "C" int afg_autotune(afg_forest *const *cands, int n, const afg_mg_opts *base, const char *json_in,
                            char *json_out, size_t cap) {
    if (!cands || n < 1 || !json_out || cap < 2) return afg::api_fail(AFG_ERR_ARG, "bad arguments");
    for (int i = 0; i < n; ++i)
        if (!cands[i] || !cands[i]->grid) return afg::api_fail(AFG_ERR_ARG, "null candidate forest");
    std::vector<int> sw, reps_v, vpts;
    std::string err;
    if (!json_ints(json_in, "sweeps", sw, err) || !json_ints(json_in, "reps", reps_v, err) ||
        !json_ints(json_in, "vectors_per_thread", vpts, err))
        return afg::api_fail(AFG_ERR_ARG, "json_in: " + err);
    if (vpts.empty()) vpts = {1};
    for (int v : vpts)
        if (v != 1 && v != 2) return afg::api_fail(AFG_ERR_ARG, "json_in: vectors_per_thread must be 1 or 2");
    if (sw.empty()) sw = {1, 1, 2, 2, 3, 3};
    if (sw.size() % 2) return afg::api_fail(AFG_ERR_ARG, "json_in: sweeps must be pairs [n_down, n_up]");
    const int reps = reps_v.empty() ? 3 : reps_v[0];
    if (reps < 1 || reps > 100) return afg::api_fail(AFG_ERR_ARG, "json_in: reps must be in [1, 100]");
    afg_mg_opts o0;
    if (base) o0 = *base;
    else {
        afg_default_opts(&o0);
        o0.precision = AFG_MIXED;
        o0.rel_tol = 1e-8;
    }
    std::vector<Row> rows;
    try {
        for (int c = 0; c < n; ++c) {
            afg_forest *f = cands[c];
            afg::DeviceGuard dg(f->device);
            afg::Grid &g = *f->grid;
            std::vector<afg_stats> st(g.T);
            double unknowns = 0;
            for (long long x : g.tree_cells) unknowns += (double)x;
            cudaEvent_t e0, e1;
            afg::check(cudaEventCreate(&e0), "event");
            afg::check(cudaEventCreate(&e1), "event");
            const int half = (g.D == 2 ? g.N * g.N : g.N * g.N * g.N) / 2;
            const int nv = std::min(half / 4, 256);
            for (size_t k = 0; k + 1 < sw.size(); k += 2)
            for (int vp : vpts) {
                if (nv / vp < 1) continue;
                afg_mg_opts o = o0;
                o.n_down = sw[k];
                o.n_up = sw[k + 1];
                o.threads_per_box = nv / vp;
                int rc = afg_forest_solve(f, &o, st.data());  // warm-up: captures the graphs
                if (rc != AFG_OK && rc != AFG_ERR_NOT_CONVERGED) return rc;
                float best = 1e30f;
                for (int r = 0; r < reps; ++r) {
                    afg::check(cudaEventRecord(e0, f->stream), "event");
                    rc = afg_forest_solve(f, &o, st.data());
                    if (rc != AFG_OK && rc != AFG_ERR_NOT_CONVERGED) return rc;
                    afg::check(cudaEventRecord(e1, f->stream), "event");
                    afg::check(cudaEventSynchronize(e1), "event");
                    float ms = 0.f;
                    afg::check(cudaEventElapsedTime(&ms, e0, e1), "event");
                    best = std::min(best, ms);
                }
                Row row{c, g.N, o.n_down, o.n_up, o.threads_per_box, 0, best, unknowns, 0.0, true};
                for (int t = 0; t < g.T; ++t) {
                    row.worst = std::max(row.worst, st[t].rel_residual);
                    row.max_cycles = std::max(row.max_cycles, st[t].cycles);
                }
                row.converged = row.worst <= o.rel_tol;
                rows.push_back(row);
            }
            cudaEventDestroy(e0);
            cudaEventDestroy(e1);
        }
    } catch (const std::exception &e) {
        return afg::api_fail(AFG_ERR_CUDA, e.what());
    }
    // objective: unknowns per second (time to the tolerance per unknown), so
    // forests of different box sizes -- different meshes at the same finest
    // spacing -- are compared per unknown; non-converged rows only if no row
    // converged
    int best = -1;
    for (int pass = 0; pass < 2 && best < 0; ++pass)
        for (size_t i = 0; i < rows.size(); ++i) {
            if (pass == 0 && !rows[i].converged) continue;
            if (best < 0 || rows[i].unknowns / rows[i].ms > rows[best].unknowns / rows[best].ms) best = (int)i;
        }
    auto row_json = [](const Row &r) {
        char b[512];
        std::snprintf(b, sizeof b,
                      "{\"candidate\": %d, \"box_n\": %d, \"n_down\": %d, \"n_up\": %d, \"threads_per_box\": %d, "
                      "\"ms\": %.6g, \"unknowns\": %.0f, \"unknowns_per_s\": %.6g, \"converged\": %s, "
                      "\"worst_rel_residual\": %.6g, \"max_cycles\": %d}",
                      r.cand, r.box_n, r.nd, r.nu, r.tpb, r.ms, r.unknowns, r.unknowns / (r.ms * 1e-3),
                      r.converged ? "true" : "false", r.worst, r.max_cycles);
        return std::string(b);
    };
    std::string js = "{\"objective\": \"unknowns_per_s\", \"best\": " + row_json(rows[best]) + ", \"table\": [";
    for (size_t i = 0; i < rows.size(); ++i) js += (i ? ", " : "") + row_json(rows[i]);
    js += "]}";
    if (js.size() + 1 > cap) return afg::api_fail(AFG_ERR_ARG, "json_out too small: needs " + std::to_string(js.size() + 1) + " bytes");
    std::memcpy(json_out, js.c_str(), js.size() + 1);
    return AFG_OK;
}
