// Sums of a few doubles formed exactly in 64-bit fixed point on the integer
// pipe, then rounded once.
//
// GB300 executes FP64 arithmetic at 2 FMA per clock per SM, 64 times below its
// FP32 / INT32 rate, so the FP64 stencil kernels are bound by the FP64 pipe,
// and most of their FP64 instructions are the additions of the neighbour sum
// of the (2D+1)-point operator (Eq. 5 and the relaxation of Sec. 3.1).  Here
// that sum is formed without FP64 instructions: every term's significand is
// aligned, as a 64-bit integer, to the largest exponent among the terms, with
// G guard bits below the 53-bit significand of the largest term and enough
// headroom above it for the total weight of the terms; the aligned integers
// are added exactly (two's complement) and the total is rounded once to
// nearest-even.  Besides that one rounding the only error is the truncation
// of bits lying more than 52 + G bits below the leading bit of the largest
// term: under one unit of 2^-G ulp(largest term) per unit of weight.
// Recursive FP64 summation rounds at every addition (up to half an ulp of each
// partial sum), so these sums are at least as accurate.  This is aligned
// (long-accumulator) summation in the manner of Kulisch & Miranker, cut to a
// 64-bit window.
//
// Range: the largest biased exponent E of the terms must lie in
// [kFxEmin, kFxEmax]; otherwise (every term zero or below 2^-959, a term near
// overflow, infinite or NaN) fx_sum returns false and the caller adds in FP64.
// Terms far below the largest one (zeros, subnormals) need no special case:
// their alignment shift exceeds the window and they contribute nothing.
#pragma once
#include <cstdint>
#include <cstring>

#ifdef __CUDACC__
#define AFG_HD __host__ __device__ __forceinline__
#else
#define AFG_HD inline
#endif
#ifdef __CUDA_ARCH__
#define AFG_FX_UNROLL _Pragma("unroll")
#else
#define AFG_FX_UNROLL
#endif

namespace afg {

constexpr int kFxEmin = 64, kFxEmax = 2040;

AFG_HD uint64_t fx_bits(double x) {
#ifdef __CUDA_ARCH__
    return (uint64_t)__double_as_longlong(x);
#else
    uint64_t b;
    std::memcpy(&b, &x, 8);
    return b;
#endif
}

AFG_HD double fx_double(uint64_t b) {
#ifdef __CUDA_ARCH__
    return __longlong_as_double((long long)b);
#else
    double x;
    std::memcpy(&x, &b, 8);
    return x;
#endif
}

AFG_HD int fx_clz(uint64_t a) {
#ifdef __CUDA_ARCH__
    return __clzll((long long)a);
#else
    return __builtin_clzll(a);
#endif
}

// Number of headroom bits for a total integer weight W (|sum| < W * 2^(63-h)).
constexpr int fx_headroom(int W) { return W <= 2 ? 1 : W <= 4 ? 2 : W <= 8 ? 3 : W <= 16 ? 4 : W <= 32 ? 5 : 6; }

// biased exponent field of x
AFG_HD int fx_exp(double x) { return (int)(fx_bits(x) >> 52) & 0x7FF; }

// Accumulator for terms of total |weight| at most W, aligned to E, the
// largest biased exponent among all terms (found by the caller first, with
// fx_exp).  add() the terms, then round().  Valid only when ok().
template <int W>
struct FxAcc {
    static constexpr int H = fx_headroom(W);
    static constexpr int G = 63 - H - 53;  // guard bits below the largest significand
    static_assert(G >= 4, "too many terms");
    int E;
    int64_t S;
    AFG_HD explicit FxAcc(int e) : E(e), S(0) {}
    AFG_HD bool ok() const { return E >= kFxEmin && E <= kFxEmax; }
    // S += w * x, w a small signed integer (sum of all |w| <= W)
    AFG_HD void add(double x, int w = 1) {
        const uint64_t b = fx_bits(x);
        // significand with its implicit bit (a zero or subnormal term gets a
        // spurious implicit bit, but its shift E - 0 >= 64 clears it)
        const uint64_t m = ((b & 0xFFFFFFFFFFFFFull) | (1ull << 52)) << G;
        const int s = E - ((int)(b >> 52) & 0x7FF);
        int64_t a = (int64_t)(s < 64 ? m >> s : 0);
        const int64_t neg = (int64_t)b >> 63;  // 0 or -1
        a = (a ^ neg) - neg;
        S += a * w;
    }
    // nearest-even rounding of S * 2^(E - 1075 - G)
    AFG_HD double round() const {
        if (S == 0) return 0.0;
        const uint64_t sg = (uint64_t)S & 0x8000000000000000ull;
        const uint64_t A = S < 0 ? (uint64_t)(-S) : (uint64_t)S;
        const int p = 63 - fx_clz(A);  // leading bit; p <= 62
        const int r = p - 52;
        uint64_t M;
        if (r > 0)  // round to nearest, ties to even: add half - 1 + lsb, then shift
            M = (A + ((1ull << (r - 1)) - 1) + ((A >> r) & 1)) >> r;
        else
            M = A << (-r);
        // biased exponent p + E - 52 - G.  M carries the implicit bit, so
        // (exponent - 1) << 52 + M also takes the carry of a round-up to 2^53
        // into the exponent.
        return fx_double((((uint64_t)(p + E - 53 - G) << 52) + M) | sg);
    }
};

// out = sum_k x[k] - C * c over x[0..K-1].  Returns false (out untouched)
// when the largest exponent is outside the handled range.
template <int K, int C = 0>
AFG_HD bool fx_sum(const double *x, double c, double &out) {
    int E = C ? fx_exp(c) : 0;
AFG_FX_UNROLL
    for (int k = 0; k < K; ++k) {
        const int e = fx_exp(x[k]);
        E = e > E ? e : E;
    }
    FxAcc<K + C> acc(E);
    if (!acc.ok()) return false;
AFG_FX_UNROLL
    for (int k = 0; k < K; ++k) acc.add(x[k]);
    if (C) acc.add(c, -C);
    out = acc.round();
    return true;
}

}  // namespace afg
