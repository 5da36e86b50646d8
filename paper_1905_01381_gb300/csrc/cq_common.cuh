// Shared device-side data structures of the Fock-build library.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "cq_df.cuh"

namespace cq {

constexpr int LMAX = 2;
constexpr int LTOT_MAX = 4 * LMAX;
constexpr int MAX_PRIM = 16;

__host__ __device__ constexpr int ncart(int L) { return (L + 1) * (L + 2) / 2; }

// Primitive pair data of one shell pair (a, b), la >= lb.
//   zeta = alpha + beta, oo2z = 1/(2 zeta), P = (alpha A + beta B)/zeta,
//   PA = P - A, K = c_a c_b exp(-alpha beta/zeta |A-B|^2) * sqrt(2) pi^{5/4} / zeta
// so that the (ss|ss)^(m) prefactor is K_ab K_cd / sqrt(zeta + eta).
template <typename R>
struct __align__(16) PrimPairT {
    R zeta, oo2z, P[3], PA[3], K;
    R pad[3];   // 12 values: loaded as three 16-byte (FP32) or six 16-byte (FP64) vectors
};
using PrimPair = PrimPairT<double>;
using PrimPairF = PrimPairT<float>;
using PrimPairX = PrimPairT<df>;     // double-float shadow

// Contracted shell pair header.
struct PairHdr {
    int a, b;        // shell indices (L[a] >= L[b])
    int bfa, bfb;    // first basis function of a and b within their molecule
    int nprim;       // number of primitive pairs
    int poff;        // offset into the primitive-pair arrays
    double AB[3];    // A - B
    int sa, sb;      // shell indices within the molecule
    long long mbase; // offset of the molecule's matrix slot (elements)
    long long smbase;// offset of the molecule's shell-block slot (density maxima)
};

// Per primitive quartet quantities consumed by the generated recurrences.
template <typename R>
struct PrimQuartet {
    R PA[3], QC[3], WP[3], WQ[3];
    R oo2z, oo2e, oo2ze, roz, roe;
    R S[LTOT_MAX + 1];   // [00|00]^(m) = prefactor * F_m(T)
};

template <int LA, int LB, int LC, int LD>
struct EriClass;  // specialisations are generated (gen_eri.py)

// ---------------------------------------------------------------- Boys
// Tabulated Taylor expansion around the nearest grid point T_k = k/16
// (|delta| <= 1/32), then downward recursion
//   F_m(T) = (2T F_{m+1}(T) + e^{-T}) / (2m+1),
// with e^{-T} = e^{-T_k} e^{-delta} (table column + Taylor).  For T >= 40
// the asymptotic F_0 = sqrt(pi/T)/2 and upward recursion
//   F_{m+1} = ((2m+1) F_m - e^{-T}) / (2T)
// are used.  The table is filled on the device by boys_table_kernel from the
// Kummer power series of the highest order and downward recursion.
constexpr int BOYS_NT = 40 * 16 + 2;     // grid rows, T in [0, 40]
constexpr double BOYS_TMAX = 40.0;
constexpr int BOYS_D_COLS = 18;          // m = 0..15, col 16 = e^{-T_k}
constexpr int BOYS_D_EXP = 16;
constexpr int BOYS_D_TAYLOR = 8;         // terms j = 0..7 (FP64)
constexpr int BOYS_F_COLS = 14;          // m = 0..12, col 13 = e^{-T_k}
constexpr int BOYS_F_EXP = 13;
constexpr int BOYS_F_TAYLOR = 5;         // terms j = 0..4 (FP32)
// double-float table, stored right after the FP32 one in the same array:
// m = 0..15, col 16 = e^{-T_k}, each as a (hi, lo) pair
constexpr int BOYS_X_COLS = 17;
constexpr int BOYS_X_EXP = 16;
constexpr int BOYS_X_TAYLOR = 8;         // terms j = 0..7
__host__ __device__ constexpr size_t boys_x_offset() { return (size_t)BOYS_NT * BOYS_F_COLS; }   // in floats

template <int L>
__device__ __forceinline__ void boys(double T, double* F, const double* __restrict__ tab)
{
    if (T < BOYS_TMAX) {
        const int k = __double2int_rn(T * 16.0);
        const double dl = T - 0.0625 * k;
        const double* row = tab + k * BOYS_D_COLS;
        double c[BOYS_D_TAYLOR];
#pragma unroll
        for (int j = 1; j < BOYS_D_TAYLOR; ++j) c[j] = -dl * (1.0 / j);
        double f = __ldg(row + L + BOYS_D_TAYLOR - 1);
#pragma unroll
        for (int j = BOYS_D_TAYLOR - 1; j >= 1; --j) f = fma(f, c[j], __ldg(row + L + j - 1));
        F[L] = f;
        if (L > 0) {
            double e = 1.0;
#pragma unroll
            for (int j = BOYS_D_TAYLOR - 1; j >= 1; --j) e = fma(e, c[j], 1.0);
            e *= __ldg(row + BOYS_D_EXP);
            const double t2 = T + T;
#pragma unroll
            for (int m = L - 1; m >= 0; --m) F[m] = fma(t2, F[m + 1], e) * (1.0 / (2 * m + 1));
        }
    } else {
        const double rs = rsqrt(T);
        F[0] = 0.88622692545275801365 * rs;   // sqrt(pi)/2
        if (L > 0) {
            const double e = exp(-T);
            const double o2t = 0.5 * rs * rs;
#pragma unroll
            for (int m = 0; m < L; ++m) F[m + 1] = fma((double)(2 * m + 1), F[m], -e) * o2t;
        }
    }
}

template <int L>
__device__ __forceinline__ void boys(float T, float* F, const float* __restrict__ tab)
{
    if (T < (float)BOYS_TMAX) {
        const int k = __float2int_rn(T * 16.0f);
        const float dl = T - 0.0625f * k;
        const float* row = tab + k * BOYS_F_COLS;
        float c[BOYS_F_TAYLOR];
#pragma unroll
        for (int j = 1; j < BOYS_F_TAYLOR; ++j) c[j] = -dl * (1.0f / j);
        float f = __ldg(row + L + BOYS_F_TAYLOR - 1);
#pragma unroll
        for (int j = BOYS_F_TAYLOR - 1; j >= 1; --j) f = fmaf(f, c[j], __ldg(row + L + j - 1));
        F[L] = f;
        if (L > 0) {
            float e = 1.0f;
#pragma unroll
            for (int j = BOYS_F_TAYLOR - 1; j >= 1; --j) e = fmaf(e, c[j], 1.0f);
            e *= __ldg(row + BOYS_F_EXP);
            const float t2 = T + T;
#pragma unroll
            for (int m = L - 1; m >= 0; --m) F[m] = fmaf(t2, F[m + 1], e) * (1.0f / (2 * m + 1));
        }
    } else {
        // correctly rounded 1/T and sqrt keep the upward recursion within a
        // few ulp of F_m over m <= 8
        const float it = 1.0f / T;
        F[0] = 0.886226925f * sqrtf(it);
        if (L > 0) {
            const float e = __expf(-T);
            const float o2t = 0.5f * it;
#pragma unroll
            for (int m = 0; m < L; ++m) F[m + 1] = fmaf((float)(2 * m + 1), F[m], -e) * o2t;
        }
    }
}

// ------------------------------------------------ J'/K' accumulation
// Order-independent accumulation.  Every contribution v is added to its
// element as the integer X = trunc(v 2^80), held in two signed 64-bit words:
// hi = trunc(X / 2^40) (units of 2^-40) and lo = X - hi 2^40 (units of
// 2^-80, |lo| < 2^40).  Integer addition is associative, so the sums --
// and the J, K built from them -- are the same bit for bit whatever the
// order of the adds (concurrent class kernels, warps, atomics).  Range:
// |element| < 2^22 and fewer than 2^23 adds per element; resolution 2^-80
// per add.  An element e occupies words 2e (hi) and 2e + 1 (lo).
using acc_t = unsigned long long;
constexpr double FX_HI_UNIT = 9.094947017729282379e-13;   // 2^-40
constexpr double FX_LO_UNIT = 8.271806125530276749e-25;   // 2^-80

__device__ __forceinline__ void fx_add(acc_t* __restrict__ acc, size_t e, double v)
{
    const unsigned long long u = (unsigned long long)__double_as_longlong(v);
    const int ex = (int)((u >> 52) & 0x7ff);
    int sh = ex - 1075 + 80;             // |v| 2^80 = man 2^sh
    if (ex == 0 || sh <= -53) return;    // zero, subnormal or below 2^-80
    if (sh > 49) sh = 49;                // |v| >= 2^22: outside the documented range (saturates)
    const unsigned long long man = (u & 0xfffffffffffffull) | (1ull << 52);
    const unsigned long long mask40 = (1ull << 40) - 1;
    unsigned long long mh, ml;
    if (sh < 0) {
        const unsigned long long m = man >> (-sh);
        mh = m >> 40;
        ml = m & mask40;
    } else if (sh < 40) {
        mh = man >> (40 - sh);
        ml = (man << sh) & mask40;
    } else {
        mh = man << (sh - 40);
        ml = 0;
    }
    const bool neg = (u >> 63) != 0;
    if (mh) atomicAdd(acc + 2 * e, neg ? (unsigned long long)(-(long long)mh) : mh);
    if (ml) atomicAdd(acc + 2 * e + 1, neg ? (unsigned long long)(-(long long)ml) : ml);
}

// Value of the integer sum (hi, lo) (signed words), rounded once to FP64.
__host__ __device__ __forceinline__ double fx_value(long long hi, long long lo)
{
    return (double)hi * FX_HI_UNIT + (double)lo * FX_LO_UNIT;
}

// Boys values of a primitive quartet in its kernel's precision.  FP32
// quartets keep FP64 near the small-T branch: below the first table interval
// (T < 1/32) the values come from the FP64 expansion around T = 0 and are
// rounded to FP32 once.
constexpr float BOYS_FP64_BELOW = 0.03125f;

template <int L>
__device__ __forceinline__ void boys_q(double T, double* F, const double* __restrict__ tabd,
                                       const float* __restrict__)
{
    boys<L>(T, F, tabd);
}

template <int L>
__device__ __forceinline__ void boys_q(float T, float* F, const double* __restrict__ tabd,
                                       const float* __restrict__ tabf)
{
    if (T < BOYS_FP64_BELOW) {
        double Fd[L + 1];
        boys<L>((double)T, Fd, tabd);
#pragma unroll
        for (int m = 0; m <= L; ++m) F[m] = (float)Fd[m];
    } else {
        boys<L>(T, F, tabf);
    }
}

// Double-float: the same tabulated Taylor expansion (8 terms, |delta| <=
// 1/32) and downward recursion in double-float arithmetic from the
// double-float table; for T >= 40 the asymptotic form with a double-float
// reciprocal and square root, and e^{-T} in FP32 (below 4.3e-18 there, its
// FP32 rounding is far below the double-float precision of the result).
template <int L>
__device__ __forceinline__ void boys_q(df T, df* F, const double* __restrict__, const float* __restrict__ tabf)
{
    const df* __restrict__ tab = reinterpret_cast<const df*>(tabf + boys_x_offset());
    if (T.hi < (float)BOYS_TMAX) {
        const int k = __float2int_rn(T.hi * 16.0f);
        const df d(T.hi - 0.0625f * (float)k, T.lo);      // T - T_k (the FP32 difference is exact)
        const df md = -d;
        const df* row = tab + k * BOYS_X_COLS;
        df c[BOYS_X_TAYLOR];
#pragma unroll
        for (int j = 1; j < BOYS_X_TAYLOR; ++j) c[j] = md * df(1.0 / j);
        df f = row[L + BOYS_X_TAYLOR - 1];
#pragma unroll
        for (int j = BOYS_X_TAYLOR - 1; j >= 1; --j) f = fma(f, c[j], row[L + j - 1]);
        F[L] = f;
        if (L > 0) {
            df e(1.f, 0.f);
#pragma unroll
            for (int j = BOYS_X_TAYLOR - 1; j >= 1; --j) e = fma(e, c[j], df(1.f, 0.f));
            e = e * row[BOYS_X_EXP];
            const df t2 = T + T;
#pragma unroll
            for (int m = L - 1; m >= 0; --m) F[m] = fma(t2, F[m + 1], e) * df(1.0 / (2 * m + 1));
        }
    } else {
        const df it = recip(T);
        F[0] = sqrt_df(it) * df(0.88622692545275801365);   // sqrt(pi)/2
        if (L > 0) {
            const df e(__expf(-T.hi), 0.f);
            const df o2t = it * df(0.5f, 0.f);
#pragma unroll
            for (int m = 0; m < L; ++m) F[m + 1] = (F[m] * df(2 * m + 1) - e) * o2t;
        }
    }
}

__device__ __forceinline__ double rsqrt_r(double x) { return rsqrt(x); }
__device__ __forceinline__ float rsqrt_r(float x) { return rsqrtf(x); }

}  // namespace cq
