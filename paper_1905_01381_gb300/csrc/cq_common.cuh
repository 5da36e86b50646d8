// Shared device-side data structures of the Fock-build library.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

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
struct PrimPairT {
    R zeta, oo2z, P[3], PA[3], K;
};
using PrimPair = PrimPairT<double>;
using PrimPairF = PrimPairT<float>;

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
        const float rs = rsqrtf(T);
        F[0] = 0.886226925f * rs;
        if (L > 0) {
            const float e = __expf(-T);
            const float o2t = 0.5f * rs * rs;
#pragma unroll
            for (int m = 0; m < L; ++m) F[m + 1] = fmaf((float)(2 * m + 1), F[m], -e) * o2t;
        }
    }
}

__device__ __forceinline__ double rsqrt_r(double x) { return rsqrt(x); }
__device__ __forceinline__ float rsqrt_r(float x) { return rsqrtf(x); }

}  // namespace cq
