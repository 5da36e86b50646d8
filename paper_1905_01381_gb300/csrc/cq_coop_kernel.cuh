// Kernel of the warp-cooperative path; included after coop_tables.cuh,
// which defines COOP_CLASSES_D.
#pragma once
#include "cq_coop.cuh"

namespace cq {

template <typename R>
__device__ __forceinline__ void boys_rt_any(int L, R T, R* F, const double* td, const float* tf)
{
    switch (L) {
        case 0: boys_q<0>(T, F, td, tf); break;
        case 1: boys_q<1>(T, F, td, tf); break;
        case 2: boys_q<2>(T, F, td, tf); break;
        case 3: boys_q<3>(T, F, td, tf); break;
        case 4: boys_q<4>(T, F, td, tf); break;
        case 5: boys_q<5>(T, F, td, tf); break;
        case 6: boys_q<6>(T, F, td, tf); break;
        case 7: boys_q<7>(T, F, td, tf); break;
        default: boys_q<8>(T, F, td, tf); break;
    }
}

// one vertical-recurrence node: returns the output slot, value in v
template <typename R>
__device__ __forceinline__ int coop_node(int shape, const int4 d, const R* __restrict__ cf, const R* V, R& v)
{
    const int x0 = d.x & 0xffff, x1 = (unsigned)d.x >> 16;
    const int cw = d.w;
    v = cf[cw & 63] * V[x0];
    v = fma(cf[(cw >> 6) & 63], V[x1], v);
    if (shape == 1 || shape == 3) {
        const int x2 = d.y & 0xffff, x3 = (unsigned)d.y >> 16;
        v = fma(cf[(cw >> 12) & 63], fma(-cf[(cw >> 18) & 63], V[x3], V[x2]), v);
    }
    if (shape >= 2) v = fma(cf[(cw >> 24) & 63], V[d.z & 0xffff], v);
    return (unsigned)d.z >> 16;
}

// Horizontal recurrence and output-stationary digestion of one contracted
// quartet whose [e0|f0] block sits in V[C.N + t] (t = ie |F| + jf): the
// warp walks the HRR table, then every lane owns whole J'/K' elements of the
// quartet's six blocks.  All 32 lanes take part.
template <typename R>
__device__ __forceinline__ void coop_hrr_digest(const CoopClass& C, R* __restrict__ V, R* __restrict__ Db,
                                                R* __restrict__ hc, const PairHdr& B, const PairHdr& K, int ib,
                                                int j, const JKArgs& a, int lane)
{
    const int NA = ncart(C.la), NB = ncart(C.lb), NC = ncart(C.lc), ND = ncart(C.ld);
    const int n = a.nbf;
    if (lane < 3) { hc[lane] = (R)B.AB[lane]; hc[3 + lane] = (R)K.AB[lane]; }
    __syncwarp();
    for (int g = 0; g < C.nhg; ++g) {
        const int4 G = __ldg(C.hgrp + g);
        if (lane < G.y) {
            const int4 d = __ldg(C.hdesc + G.z + lane);
            const int x0 = d.x & 0xffff, x1 = (unsigned)d.x >> 16;
            const R v = (G.x == 0) ? fma(hc[d.w & 63], V[x1], V[x0]) : V[x0];
            V[(unsigned)d.z >> 16] = v;
        }
        if (G.w) __syncwarp();
    }
    __syncwarp();

    // ---- output-stationary digestion
    R sdeg = R(1);
    if (B.a == B.b) sdeg *= R(0.5);
    if (K.a == K.b) sdeg *= R(0.5);
    if (j == ib) sdeg *= R(0.5);
    const int fa = B.bfa, fb = B.bfb, fc = K.bfa, fd = K.bfb;
    const long long mb = B.mbase;
    const int nJ = (a.want_j ? NA * NB + NC * ND : 0);
    const int nK = (a.want_k ? NA * NC + NA * ND + NB * NC + NB * ND : 0);
    for (int q = 0; q < a.nk; ++q) {
        if (q > 0 && !a.want_k) break;
        const double* Dq = a.D + (size_t)q * a.mstride;
        acc_t* Kq = a.K + 2 * (size_t)q * a.mstride;
        // density blocks: ab, cd, bd, bc, ad, ac (each <= 36)
        for (int e = lane; e < 216; e += 32) {
            const int blk = e / 36, r = e - blk * 36;
            int rr = 0, cc = 0, nr = 0, ncol = 0;
            switch (blk) {
                case 0: nr = NA; ncol = NB; rr = fa; cc = fb; break;
                case 1: nr = NC; ncol = ND; rr = fc; cc = fd; break;
                case 2: nr = NB; ncol = ND; rr = fb; cc = fd; break;
                case 3: nr = NB; ncol = NC; rr = fb; cc = fc; break;
                case 4: nr = NA; ncol = ND; rr = fa; cc = fd; break;
                default: nr = NA; ncol = NC; rr = fa; cc = fc; break;
            }
            if (r < nr * ncol) Db[e] = ldR<R>(Dq + mb + (size_t)(rr + r / ncol) * n + cc + r % ncol);
        }
        __syncwarp();
        const int nout = (q == 0 ? nJ : 0) + nK;
        for (int o = lane; o < nout; o += 32) {
            int kind = 0, oo = o;
            if (q != 0) kind = 2;
            if (q == 0 && oo >= nJ) { kind = 2; oo -= nJ; }
            R sum = R(0);
            acc_t* dst;
            size_t de;
            double f;
            if (kind == 0 && oo < NA * NB) {            // J'_ab
                const int m = oo / NB, k = oo % NB;
                for (int ls = 0; ls < NC * ND; ++ls) sum = fma(V[(m * NB + k) * NC * ND + ls], Db[36 + ls], sum);
                dst = a.J; de = mb + (size_t)(fa + m) * n + fb + k;
                f = 2.0 * (double)sdeg;
            } else if (kind == 0) {                       // J'_cd
                oo -= NA * NB;
                const int l = oo / ND, s = oo % ND;
                for (int mk = 0; mk < NA * NB; ++mk) sum = fma(V[mk * NC * ND + l * ND + s], Db[mk], sum);
                dst = a.J; de = mb + (size_t)(fc + l) * n + fd + s;
                f = 2.0 * (double)sdeg;
            } else if (oo < NA * NC) {                    // K'_ac += (ab|cd) D_bd
                const int m = oo / NC, l = oo % NC;
                for (int k = 0; k < NB; ++k)
                    for (int s = 0; s < ND; ++s)
                        sum = fma(V[((m * NB + k) * NC + l) * ND + s], Db[72 + k * ND + s], sum);
                dst = Kq; de = mb + (size_t)(fa + m) * n + fc + l;
                f = (double)sdeg;
            } else if (oo < NA * NC + NA * ND) {          // K'_ad += (ab|cd) D_bc
                oo -= NA * NC;
                const int m = oo / ND, s = oo % ND;
                for (int k = 0; k < NB; ++k)
                    for (int l = 0; l < NC; ++l)
                        sum = fma(V[((m * NB + k) * NC + l) * ND + s], Db[108 + k * NC + l], sum);
                dst = Kq; de = mb + (size_t)(fa + m) * n + fd + s;
                f = (double)sdeg;
            } else if (oo < NA * NC + NA * ND + NB * NC) {  // K'_bc += (ab|cd) D_ad
                oo -= NA * NC + NA * ND;
                const int k = oo / NC, l = oo % NC;
                for (int m = 0; m < NA; ++m)
                    for (int s = 0; s < ND; ++s)
                        sum = fma(V[((m * NB + k) * NC + l) * ND + s], Db[144 + m * ND + s], sum);
                dst = Kq; de = mb + (size_t)(fb + k) * n + fc + l;
                f = (double)sdeg;
            } else {                                       // K'_bd += (ab|cd) D_ac
                oo -= NA * NC + NA * ND + NB * NC;
                const int k = oo / ND, s = oo % ND;
                for (int m = 0; m < NA; ++m)
                    for (int l = 0; l < NC; ++l)
                        sum = fma(V[((m * NB + k) * NC + l) * ND + s], Db[180 + m * NC + l], sum);
                dst = Kq; de = mb + (size_t)(fb + k) * n + fd + s;
                f = (double)sdeg;
            }
            fx_add(dst, de, f * (double)sum);
        }
        __syncwarp();
    }
}

template <typename R>
struct CoopMinBlocks { static constexpr int v = sizeof(R) == 4 ? 8 : 6; };   // df: 8 bytes, as FP64

// Screening of a task of the candidate-task mode (list mode quartets are
// already screened): a molecule in all-FP64 mode sends every survivor to the
// FP64 half; a skipped molecule has none.
__device__ __forceinline__ bool coop_selected(const JKArgs& a, const PairHdr& B, const PairHdr& K, int ib, int j)
{
    const float* Dm = a.Dmax;
    const int ns = a.nsh;
    const float* Ds = Dm + B.smbase;
    float m = fmaxf(__ldg(Ds + B.sa * ns + B.sb), __ldg(Ds + K.sa * ns + K.sb));
    m = fmaxf(m, fmaxf(__ldg(Ds + B.sa * ns + K.sa), __ldg(Ds + B.sa * ns + K.sb)));
    m = fmaxf(m, fmaxf(__ldg(Ds + B.sb * ns + K.sa), __ldg(Ds + B.sb * ns + K.sb)));
    const float bound = __ldg(a.Q + ib) * __ldg(a.Q + j) * m;
    const int mode = a.mol_mode ? __ldg(a.mol_mode + B.smbase / a.lds2) : 1;
    const float tm = (mode & 1) ? a.tau_mixed : 0.f;
    bool sel = bound >= a.tau && !(mode & 2);
    if (a.prec_sel == 1) sel = sel && bound >= tm;
    else if (a.prec_sel == 2) sel = sel && bound < tm;
    return sel;
}

// One task: primitive quartets [p0, p1) of quartet (ib, j), their vertical
// recurrences, the contraction, HRR and digestion.  HRR and digestion are
// linear, so a chunk of primitive quartets is digested on its own and the
// J'/K' adds of all chunks sum to the quartet's.  coef, Sb and V lie one
// after the other in the warp's region, which the HRR and the digestion
// reuse from coef on once the vertical recurrences are done.
template <typename R>
__device__ __forceinline__ void coop_task(const JKArgs& a, const CoopClass& C, int ib, int j, int p0, int p1,
                                          const PairHdr& B, const PairHdr& K, R* coef,
                                          R* Sb, R* V, R* __restrict__ Db,
                                          R* __restrict__ hc, int lane, unsigned long long& nq,
                                          unsigned long long& np)
{
    // ---- primitive quartets: coefficients, VRR, accumulation
    R acc[COOP_MAXACC];
#pragma unroll
    for (int k = 0; k < COOP_MAXACC; ++k) acc[k] = R(0);
    const int nkp = K.nprim;
    for (int base = p0; base < p1; base += 32) {
        const int cnt = min(32, p1 - base);
        if (lane < cnt) {
            const int pq = base + lane;
            const int ip = pq / nkp, jp = pq - (pq / nkp) * nkp;
            PrimPairT<R> bp, kp;
            load_prim<R>(a, B.poff + ip, bp);
            load_prim<R>(a, K.poff + jp, kp);
            const R s = bp.zeta + kp.zeta;
            const R rs = rsqrt_r(s);
            const R is = rs * rs;
            const R PQx = bp.P[0] - kp.P[0], PQy = bp.P[1] - kp.P[1], PQz = bp.P[2] - kp.P[2];
            const R roz = kp.zeta * is, roe = bp.zeta * is;
            const R T = roz * bp.zeta * (PQx * PQx + PQy * PQy + PQz * PQz);
            R F[LTOT_MAX + 1];
            boys_rt_any<R>(C.L, T, F, a.boys_d, a.boys_f);
            const R pref = bp.K * kp.K * rs;
            R* cf = coef + lane * COOP_NCOEF;
            cf[0] = bp.PA[0]; cf[1] = bp.PA[1]; cf[2] = bp.PA[2];
            cf[3] = kp.PA[0]; cf[4] = kp.PA[1]; cf[5] = kp.PA[2];
            cf[6] = -roz * PQx; cf[7] = -roz * PQy; cf[8] = -roz * PQz;
            cf[9] = roe * PQx; cf[10] = roe * PQy; cf[11] = roe * PQz;
            cf[12] = roz; cf[13] = roe;
            const R o2ze = R(0.5) * is;
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                cf[14 + k] = R(k + 1) * bp.oo2z;
                cf[18 + k] = R(k + 1) * kp.oo2z;
                cf[22 + k] = R(k + 1) * o2ze;
            }
            R* sb = Sb + lane * (LTOT_MAX + 1);
            for (int m = 0; m <= C.L; ++m) sb[m] = pref * F[m];
        }
        __syncwarp();
        for (int q = 0; q < cnt; ++q) {
            if (lane <= C.L) V[lane] = Sb[q * (LTOT_MAX + 1) + lane];
            __syncwarp();
            const R* cf = coef + q * COOP_NCOEF;
            int4 Gn = __ldg(C.vgrp);
            for (int g = 0; g < C.nvg;) {
                const int4 G = Gn;
                // the next group of the same level is independent: evaluate both
                const bool pair = !G.w && g + 1 < C.nvg;
                const int4 G2 = pair ? __ldg(C.vgrp + g + 1) : G;
                const int gn = g + (pair ? 2 : 1);
                if (gn < C.nvg) Gn = __ldg(C.vgrp + gn);
                R v1 = R(0), v2 = R(0);
                int o1 = -1, o2 = -1;
                if (lane < G.y) o1 = coop_node<R>(G.x, __ldg(C.vdesc + G.z + lane), cf, V, v1);
                if (pair && lane < G2.y) o2 = coop_node<R>(G2.x, __ldg(C.vdesc + G2.z + lane), cf, V, v2);
                if (o1 >= 0) V[o1] = v1;
                if (o2 >= 0) V[o2] = v2;
                if ((pair ? G2.w : G.w)) __syncwarp();
                g = gn;
            }
#pragma unroll
            for (int k = 0; k < COOP_MAXACC; ++k) {
                const int tt = lane + 32 * k;
                if (tt < C.nacc) acc[k] += V[__ldg(C.tgt + tt)];
            }
            __syncwarp();
        }
        if (lane == 0) { nq += (base == 0); np += cnt; }
    }

    // ---- horizontal recurrence on the contracted block
#pragma unroll
    for (int k = 0; k < COOP_MAXACC; ++k) {
        const int tt = lane + 32 * k;
        if (tt < C.nacc) coef[C.N + tt] = acc[k];
    }
    coop_hrr_digest<R>(C, coef, Db, hc, B, K, ib, j, a, lane);
}

template <typename R>
__global__ void __launch_bounds__(COOP_THREADS, CoopMinBlocks<R>::v) jk_coop_kernel(const JKArgs a, int qc, int wslots)
{
    const CoopClass C = COOP_CLASSES_D[qc];
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    unsigned char* wbase = smem_raw + (size_t)wib * coop_warp_bytes<R>(wslots);
    R* coef = (R*)wbase;                                   // [32][NCOEF]; the HRR region from here
    R* Sb = coef + 32 * COOP_NCOEF;                        // [32][LTOT_MAX+1]
    R* V = Sb + 32 * (LTOT_MAX + 1);                       // VRR slots
    R* Db = coef + wslots;                                 // 6 density blocks of <= 36
    R* hc = Db + 6 * 36;                                   // AB, CD
    unsigned long long nq = 0, np = 0;
    if (a.coop_list) {
        // list mode: the warps stride over the screened quartets of the list,
        // each split into ranges of about a.coop_chunk primitive quartets
        // (at most a.coop_split ranges), one range per warp task: a deep
        // quartet (up to ~1300 primitive quartets) would otherwise hold one
        // warp for the whole build, and a short list of deep quartets would
        // leave most SMs idle.  Every range repeats the HRR and the
        // digestion, which bounds the useful split.
        const int split = a.coop_split;
        const long long cnt = (long long)*a.qcount * split;
        const long long nw = (long long)gridDim.x * COOP_WARPS;
        for (long long v = (long long)blockIdx.x * COOP_WARPS + wib; v < cnt; v += nw) {
            const long long q = v / split;
            const int k = (int)(v - q * split);
            const int2 e = a.qlist[(list_base(a) + q) * a.qdir];
            const PairHdr B = a.pairs[e.x];
            const PairHdr K = a.pairs[e.y];
            const int npq = B.nprim * K.nprim;
            const int nch = min(split, (npq + a.coop_chunk - 1) / a.coop_chunk);
            if (k >= nch) continue;
            const int chunk = (npq + nch - 1) / nch;
            const int p0 = k * chunk, p1 = min(npq, p0 + chunk);
            coop_task<R>(a, C, e.x, e.y, p0, p1, B, K, coef, Sb, V, Db, hc, lane, nq, np);
            __syncwarp();
        }
    } else {
        const int w = blockIdx.x * COOP_WARPS + wib;
        if (w < a.ntasks) {
            const int4 t = a.tasks[w];
            const PairHdr B = a.pairs[t.x];
            const PairHdr K = a.pairs[t.y];
            if (coop_selected(a, B, K, t.x, t.y))
                coop_task<R>(a, C, t.x, t.y, t.z, t.w, B, K, coef, Sb, V, Db, hc, lane, nq, np);
        }
    }
    if (a.counters) {
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            nq += __shfl_xor_sync(0xffffffffu, nq, o);
            np += __shfl_xor_sync(0xffffffffu, np, o);
        }
        if (lane == 0 && (nq || np)) {
            atomicAdd(a.counters + 0, nq);
            atomicAdd(a.counters + 1, np);
        }
    }
}

}  // namespace cq
