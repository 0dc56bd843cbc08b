// Host harness for the fixed-point sums of csrc/fxsum.cuh: reads rows of K
// terms plus one centre value (raw doubles), writes for every row the sum
// sum_k x_k - C * centre and a flag (1 = handled, 0 = caller falls back).
#include <cstdio>
#include <cstdlib>
#include <vector>
#include "../paper_1701_04329_gb300/csrc/fxsum.cuh"

template <int K, int C>
static void run(const std::vector<double> &in, size_t rows, std::vector<double> &out, std::vector<unsigned char> &ok) {
    for (size_t i = 0; i < rows; ++i) {
        double x[K];
        for (int k = 0; k < K; ++k) x[k] = in[i * (K + 1) + k];
        double s = 0.0;
        ok[i] = afg::fx_sum<K, C>(x, in[i * (K + 1) + K], s) ? 1 : 0;
        out[i] = s;
    }
}

int main(int argc, char **argv) {
    if (argc != 5) return 2;
    const int K = atoi(argv[1]), C = atoi(argv[2]);
    FILE *f = fopen(argv[3], "rb");
    if (!f) return 3;
    std::vector<double> in;
    double v;
    while (fread(&v, 8, 1, f) == 1) in.push_back(v);
    fclose(f);
    const size_t rows = in.size() / (K + 1);
    std::vector<double> out(rows);
    std::vector<unsigned char> ok(rows);
    if (K == 2 && C == 0) run<2, 0>(in, rows, out, ok);
    else if (K == 3 && C == 0) run<3, 0>(in, rows, out, ok);
    else if (K == 4 && C == 0) run<4, 0>(in, rows, out, ok);
    else if (K == 6 && C == 0) run<6, 0>(in, rows, out, ok);
    else if (K == 4 && C == 4) run<4, 4>(in, rows, out, ok);
    else if (K == 6 && C == 6) run<6, 6>(in, rows, out, ok);
    else return 4;
    FILE *g = fopen(argv[4], "wb");
    if (!g) return 5;
    fwrite(out.data(), 8, rows, g);
    fwrite(ok.data(), 1, rows, g);
    fclose(g);
    return 0;
}
