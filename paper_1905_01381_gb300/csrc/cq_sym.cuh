// FP32 J/K kernel of the high angular-momentum classes: axis-permutation
// lane groups.  G lanes (G = 3: cyclic axis permutations, G = 6: all six)
// share one contracted quartet; each runs the same straight-line vertical
// recurrence (gen_sym.py) for the representative targets T0 on inputs whose
// vector components are permuted by its group element, over ALL primitive
// quartets of the quartet, accumulating |T0| values in registers.  The
// lanes' accumulators together are the quartet's contracted [e0|f0] block;
// the warp then takes the quartets of its groups one at a time through the
// warp-cooperative horizontal recurrence and output-stationary digestion
// (coop_hrr_digest) in shared memory.  Included by the generated class
// translation units after coop_tables.cuh and the class's SymClass
// specialisation.
#pragma once
#include "cq_coop_kernel.cuh"

namespace cq {

template <int LA, int LB, int LC, int LD, int G>
struct SymClass;   // specialisations are generated (gen_sym.py)
template <int LA, int LB, int LC, int LD, int G>
__device__ const unsigned short* sym_dst();

constexpr int SYM_THREADS = 128;   // 4 warps per CTA

template <typename R>
__host__ __device__ constexpr size_t sym_warp_bytes(int nslots)
{
    return (size_t)(nslots + 6 * 36 + 8) * sizeof(R);
}

// Primitive pair i with its vector components permuted: component x of the
// result is component p[x] of the stored pair.
// Primitive pair i with its vector components permuted: component x of the
// result is component p[x] of the stored pair (scalar loads at permuted
// offsets; cheaper here than vector loads followed by selects).
template <typename R>
__device__ __forceinline__ void load_prim_perm(const JKArgs& a, int i, int p0, int p1, int p2, PrimPairT<R>& o)
{
    const R* s;
    if constexpr (sizeof(R) == 4) s = reinterpret_cast<const R*>(a.primsf + i);
    else if constexpr (std::is_same<R, df>::value) s = reinterpret_cast<const R*>(a.primsx + i);
    else s = reinterpret_cast<const R*>(a.prims + i);
    o.zeta = ldg_r(s + 0);
    o.oo2z = ldg_r(s + 1);
    o.P[0] = ldg_r(s + 2 + p0); o.P[1] = ldg_r(s + 2 + p1); o.P[2] = ldg_r(s + 2 + p2);
    o.PA[0] = ldg_r(s + 5 + p0); o.PA[1] = ldg_r(s + 5 + p1); o.PA[2] = ldg_r(s + 5 + p2);
    o.K = ldg_r(s + 8);
}

// H > 1: each of the G frames of a quartet is further split over H lanes
// that take every H-th primitive quartet; their accumulators are summed
// with shuffles before the scatter (more, shorter work units for short
// lists).  Lane r of a group of G*H: frame k = r % G, primitive stride
// offset h = r / G.
template <int LA, int LB, int LC, int LD, typename R, int G, int H>
__global__ void __launch_bounds__(SYM_THREADS) jk_sym_kernel(const JKArgs a, int qc, int nslots)
{
    using S = SymClass<LA, LB, LC, LD, G>;
    constexpr int L = LA + LB + LC + LD;
    constexpr int GH = G * H;
    constexpr int NGRP = 32 / GH;                // groups per warp; lanes NGRP*GH..31 idle in the recurrence
    constexpr int WARPS = SYM_THREADS / 32;
    static_assert((H & (H - 1)) == 0 && NGRP >= 1, "H must be a power of two with G*H <= 32");
    const CoopClass C = COOP_CLASSES_D[qc];
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    const int grp = lane / GH, r = lane - (lane / GH) * GH;
    const int k = r % G, h = r / G;
    const bool lane_on = grp < NGRP;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    R* V = reinterpret_cast<R*>(smem_raw + (size_t)wib * sym_warp_bytes<R>(nslots));
    R* Db = V + nslots;
    R* hc = Db + 6 * 36;
    const int kk = lane_on ? k : 0;
    const int p0 = (int)((S::PERM >> (6 * kk)) & 3), p1 = (int)((S::PERM >> (6 * kk + 2)) & 3),
              p2 = (int)((S::PERM >> (6 * kk + 4)) & 3);
    const unsigned short* dst = sym_dst<LA, LB, LC, LD, G>() + kk * S::N0;
    const long long cnt = (long long)*a.qcount;
    const long long nw = (long long)gridDim.x * WARPS;
    unsigned long long nq = 0, np = 0;
    for (long long w = (long long)blockIdx.x * WARPS + wib; w * NGRP < cnt; w += nw) {
        const long long idx = w * NGRP + grp;
        const bool on = lane_on && idx < cnt;
        R acc[S::N0];
#pragma unroll
        for (int i = 0; i < S::N0; ++i) acc[i] = R(0);
        if (on) {
            const int2 e = a.qlist[(list_base(a) + idx) * a.qdir];
            const PairHdr B = a.pairs[e.x];
            const PairHdr K = a.pairs[e.y];
            if constexpr (H == 1) {
                for (int ip = 0; ip < B.nprim; ++ip) {
                    PrimPairT<R> bp;
                    load_prim_perm<R>(a, B.poff + ip, p0, p1, p2, bp);
                    for (int jp = 0; jp < K.nprim; ++jp) {
                        PrimPairT<R> kp;
                        load_prim_perm<R>(a, K.poff + jp, p0, p1, p2, kp);
                        PrimQuartet<R> q;
                        prim_setup<L, R>(bp, kp, a.boys_d, a.boys_f, q);
                        S::template prim<R>(q, acc);
                    }
                }
            } else {
                const int nkp = K.nprim, tot = B.nprim * nkp;
                int ip = 0, jp = h;
                while (jp >= nkp) { jp -= nkp; ++ip; }
                for (int pq = h; pq < tot; pq += H) {
                    PrimPairT<R> bp, kp;
                    load_prim_perm<R>(a, B.poff + ip, p0, p1, p2, bp);
                    load_prim_perm<R>(a, K.poff + jp, p0, p1, p2, kp);
                    PrimQuartet<R> q;
                    prim_setup<L, R>(bp, kp, a.boys_d, a.boys_f, q);
                    S::template prim<R>(q, acc);
                    jp += H;
                    while (jp >= nkp) { jp -= nkp; ++ip; }
                }
            }
            if (r == 0) { nq += 1; np += (unsigned long long)B.nprim * K.nprim; }
        }
        if constexpr (H > 1) {   // sum the H partial accumulators of each frame into h = 0
#pragma unroll
            for (int i = 0; i < S::N0; ++i) {
                R v = acc[i];
#pragma unroll
                for (int o = H / 2; o > 0; o >>= 1) v += shfl_down_r(v, G * o);
                acc[i] = v;
            }
        }
        // the warp's quartets, one at a time: scatter the group's
        // accumulators into the [e0|f0] block, HRR and digestion
        for (int g = 0; g < NGRP; ++g) {
            const long long gi = w * NGRP + g;
            if (gi >= cnt) break;                    // warp-uniform
            if (grp == g && h == 0) {
#pragma unroll
                for (int i = 0; i < S::N0; ++i) {
                    const int d = __ldg(dst + i);
                    if (d != 0xFFFF) V[C.N + d] = acc[i];
                }
            }
            __syncwarp();
            const int2 eg = a.qlist[(list_base(a) + gi) * a.qdir];
            const PairHdr B = a.pairs[eg.x];
            const PairHdr K = a.pairs[eg.y];
            coop_hrr_digest<R>(C, V, Db, hc, B, K, eg.x, eg.y, a, lane);
            __syncwarp();
        }
    }
    if (a.counters) {
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            nq += __shfl_xor_sync(0xffffffffu, nq, o);
            np += __shfl_xor_sync(0xffffffffu, np, o);
        }
        if (lane == 0 && nq) {
            atomicAdd(a.counters + 0, nq);
            atomicAdd(a.counters + 1, np);
        }
    }
}

}  // namespace cq
