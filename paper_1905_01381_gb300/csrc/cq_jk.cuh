// J/K kernel template: one warp per (bra shell pair, range of ket shell
// pairs), one lane per contracted shell quartet.  Included by the generated
// per-class translation units after the class's EriClass specialisation.
#pragma once
#include <type_traits>

#include "cq_common.cuh"

namespace cq {

constexpr int JK_THREADS = 128;   // 4 warps per CTA
constexpr int JK_RANGE = 64;      // largest number of ket candidates per warp task

struct JKArgs {
    const PairHdr* pairs;
    const PrimPair* prims;
    const PrimPairF* primsf;
    const PrimPairX* primsx;      // double-float shadow of the pair data
    const int4* tasks;            // (bra pair, first ket candidate, end of candidates, 0)
    int ntasks;
    int ket_end;                  // end of the ket class range (exclusive)
    int same_class;               // bra and ket class equal: kets j <= bra
    const float* Q;               // Schwarz factor per pair
    const float* Dmax;            // nsh x nsh block maxima of |P| (all components)
    int nsh;
    float tau;                    // screening threshold
    float tau_mixed;              // precision split (FP32 below)
    int prec_sel;                 // 0: every surviving quartet; 1: bound >= tau_mixed; 2: bound < tau_mixed
    const double* D;              // nk scaled density matrices, nbf x nbf each
    int nk;
    int nbf;                      // leading dimension of every matrix slot
    long long mstride;            // elements of one matrix over all slots (density q at q * mstride)
    int want_j, want_k;
    acc_t* J;                     // J' accumulator nbf x nbf (fx_add words)
    acc_t* K;                     // K' accumulators nk x nbf x nbf (fx_add words)
    const double* boys_d;
    const float* boys_f;
    unsigned long long* counters; // [0] quartets, [1] primitive quartets
    const int2* qlist;            // compacted (bra, ket) quartets of this class and precision
    const unsigned int* qcount;   // number of entries (device)
    const unsigned int* qbase;    // optional device offset of the list's first entry (double-float
                                  // lists start after the FP64 list of their region); NULL: 0
    int qdir;                     // +1: entries qlist[i]; -1: entries qlist[-i] (list filled from the back)
    long long qmax;               // capacity of the list (candidate quartets of the class)
    const int* mol_mode;          // optional per-molecule mode (see ClassifyArgs), read by the
    long long lds2;               // cooperative kernel, which screens its own tasks
    int coop_list;                // cooperative kernel: 1 = quartets from qlist (already screened)
    int fp64_tier;                // the FP64 list of a three-tier build (short, deep quartets)
    int coop_split;               // cooperative kernel, list mode: warp tasks per quartet, at most
    int coop_chunk;               // ... and primitive quartets per task, about
};

template <typename R>
__device__ __forceinline__ R ldR(const double* p) { return (R)__ldg(p); }

// The pair data of a primitive pair in 16-byte vector loads (a lane reads
// its own pair, so the loads of a warp are scattered: fewer, wider loads
// cost fewer L1 wavefronts).
__device__ __forceinline__ void load_prim_v(const PrimPair* pd, int i, PrimPairT<double>& o)
{
    const double2* s = reinterpret_cast<const double2*>(pd + i);
    const double2 a = __ldg(s), b = __ldg(s + 1), c = __ldg(s + 2), d = __ldg(s + 3);
    o.zeta = a.x; o.oo2z = a.y;
    o.P[0] = b.x; o.P[1] = b.y; o.P[2] = c.x;
    o.PA[0] = c.y; o.PA[1] = d.x; o.PA[2] = d.y;
    o.K = __ldg(reinterpret_cast<const double*>(s + 4));
}

__device__ __forceinline__ void load_prim_v(const PrimPairF* pf, int i, PrimPairT<float>& o)
{
    const float4* s = reinterpret_cast<const float4*>(pf + i);
    const float4 a = __ldg(s), b = __ldg(s + 1);
    o.zeta = a.x; o.oo2z = a.y;
    o.P[0] = a.z; o.P[1] = a.w; o.P[2] = b.x;
    o.PA[0] = b.y; o.PA[1] = b.z; o.PA[2] = b.w;
    o.K = __ldg(reinterpret_cast<const float*>(s + 2));
}

__device__ __forceinline__ void load_prim_v(const PrimPairX* px, int i, PrimPairT<df>& o)
{
    const float4* s = reinterpret_cast<const float4*>(px + i);
    const float4 a = __ldg(s), b = __ldg(s + 1), c = __ldg(s + 2), d = __ldg(s + 3);
    const float2 e = __ldg(reinterpret_cast<const float2*>(s + 4));
    o.zeta = df(a.x, a.y); o.oo2z = df(a.z, a.w);
    o.P[0] = df(b.x, b.y); o.P[1] = df(b.z, b.w); o.P[2] = df(c.x, c.y);
    o.PA[0] = df(c.z, c.w); o.PA[1] = df(d.x, d.y); o.PA[2] = df(d.z, d.w);
    o.K = df(e.x, e.y);
}

template <typename R>
__device__ __forceinline__ void load_prim(const JKArgs& a, int i, PrimPairT<R>& o)
{
    if constexpr (sizeof(R) == 4) load_prim_v(a.primsf, i, o);
    else if constexpr (std::is_same<R, df>::value) load_prim_v(a.primsx, i, o);
    else load_prim_v(a.prims, i, o);
}

template <typename R>
__device__ __forceinline__ R ldg_r(const R* p)
{
    if constexpr (std::is_same<R, df>::value) {
        const float2 v = __ldg(reinterpret_cast<const float2*>(p));
        return df(v.x, v.y);
    } else {
        return __ldg(p);
    }
}

// the list offset of a kernel's entries (double-float lists start after the
// FP64 list of their class region)
__device__ __forceinline__ long long list_base(const JKArgs& a)
{
    return a.qbase ? (long long)*a.qbase : 0;
}

// Per-primitive-quartet quantities of the vertical recurrence: prefactor
// times Boys values, PA, QC, W-P, W-Q and the exponent ratios.
template <int L, typename R>
__device__ __forceinline__ void prim_setup(const PrimPairT<R>& bp, const PrimPairT<R>& kp,
                                           const double* __restrict__ boys_d, const float* __restrict__ boys_f,
                                           PrimQuartet<R>& q)
{
    const R s = bp.zeta + kp.zeta;
    const R rs = rsqrt_r(s);
    const R is = rs * rs;
    const R PQx = bp.P[0] - kp.P[0], PQy = bp.P[1] - kp.P[1], PQz = bp.P[2] - kp.P[2];
    const R roz = kp.zeta * is;   // rho/zeta = eta/(zeta+eta)
    const R roe = bp.zeta * is;   // rho/eta  = zeta/(zeta+eta)
    const R T = roz * bp.zeta * (PQx * PQx + PQy * PQy + PQz * PQz);
    R F[L + 1];
    boys_q<L>(T, F, boys_d, boys_f);
    const R pref = bp.K * kp.K * rs;
#pragma unroll
    for (int m = 0; m <= L; ++m) q.S[m] = pref * F[m];
#pragma unroll
    for (int x = 0; x < 3; ++x) { q.PA[x] = bp.PA[x]; q.QC[x] = kp.PA[x]; }
    q.WP[0] = -roz * PQx; q.WP[1] = -roz * PQy; q.WP[2] = -roz * PQz;
    q.WQ[0] = roe * PQx;  q.WQ[1] = roe * PQy;  q.WQ[2] = roe * PQz;
    q.oo2z = bp.oo2z; q.oo2e = kp.oo2z; q.oo2ze = R(0.5) * is;
    q.roz = roz; q.roe = roe;
}

// One primitive quartet: prefactor, Boys values and the class's vertical
// recurrence, accumulated into acc.
template <int LA, int LB, int LC, int LD, typename R>
__device__ __forceinline__ void prim_quartet(const PrimPairT<R>& bp, const PrimPairT<R>& kp,
                                             const double* __restrict__ boys_d, const float* __restrict__ boys_f,
                                             R* __restrict__ acc)
{
    using C = EriClass<LA, LB, LC, LD>;
    PrimQuartet<R> q;
    prim_setup<LA + LB + LC + LD, R>(bp, kp, boys_d, boys_f, q);
    C::template prim<R>(q, acc);
}

// Contracted quartet (ab|cd) over the primitive pairs of bra and ket.
template <int LA, int LB, int LC, int LD, typename R>
__device__ __forceinline__ void eri_quartet(const PairHdr& B, const PairHdr& K, const JKArgs& a,
                                            R* __restrict__ I)
{
    using C = EriClass<LA, LB, LC, LD>;
    R acc[C::NACC];
#pragma unroll
    for (int i = 0; i < C::NACC; ++i) acc[i] = R(0);
    for (int ip = 0; ip < B.nprim; ++ip) {
        PrimPairT<R> bp;
        load_prim<R>(a, B.poff + ip, bp);
        for (int jp = 0; jp < K.nprim; ++jp) {
            PrimPairT<R> kp;
            load_prim<R>(a, K.poff + jp, kp);
            prim_quartet<LA, LB, LC, LD, R>(bp, kp, a.boys_d, a.boys_f, acc);
        }
    }
    R ABv[3] = {(R)B.AB[0], (R)B.AB[1], (R)B.AB[2]};
    R CDv[3] = {(R)K.AB[0], (R)K.AB[1], (R)K.AB[2]};
    C::template hrr<R>(acc, ABv, CDv, I);
}

__device__ __forceinline__ float dmax6(const float* Dm, int nsh, int a, int b, int c, int d)
{
    float m = fmaxf(__ldg(Dm + a * nsh + b), __ldg(Dm + c * nsh + d));
    m = fmaxf(m, fmaxf(__ldg(Dm + a * nsh + c), __ldg(Dm + a * nsh + d)));
    m = fmaxf(m, fmaxf(__ldg(Dm + b * nsh + c), __ldg(Dm + b * nsh + d)));
    return m;
}

// Contract one quartet's integral block with the density blocks and add the
// resulting J'/K' blocks (see the Fock-build notes in cq_fock.cu for the
// half-accumulation convention: J = J' + J'^T, K = K' +/- K'^T).
template <int LA, int LB, int LC, int LD, typename R>
__device__ __forceinline__ void digest(const PairHdr& B, const PairHdr& K, const R* __restrict__ I,
                                       R sdeg, const JKArgs& a, double* __restrict__ jq)
{
    constexpr int NA = ncart(LA), NB = ncart(LB), NC = ncart(LC), ND = ncart(LD);
    const int n = a.nbf;
    const int fa = B.bfa, fb = B.bfb, fc = K.bfa, fd = K.bfb;
    const long long mb = B.mbase;
    if (a.want_j) {
        const double* D0 = a.D;
        R dab[NA * NB], dcd[NC * ND], jcd[NC * ND];
#pragma unroll
        for (int m = 0; m < NA; ++m)
#pragma unroll
            for (int k = 0; k < NB; ++k) dab[m * NB + k] = ldR<R>(D0 + mb + (size_t)(fa + m) * n + fb + k);
#pragma unroll
        for (int l = 0; l < NC; ++l)
#pragma unroll
            for (int s = 0; s < ND; ++s) {
                dcd[l * ND + s] = ldR<R>(D0 + mb + (size_t)(fc + l) * n + fd + s);
                jcd[l * ND + s] = R(0);
            }
#pragma unroll
        for (int mn = 0; mn < NA * NB; ++mn) {
            R t = R(0);
#pragma unroll
            for (int ls = 0; ls < NC * ND; ++ls) {
                const R v = I[mn * NC * ND + ls];
                t = fma(v, dcd[ls], t);
                jcd[ls] = fma(v, dab[mn], jcd[ls]);
            }
            jq[mn] = 2.0 * (double)sdeg * (double)t;
        }
        const double f = 2.0 * (double)sdeg;
#pragma unroll
        for (int l = 0; l < NC; ++l)
#pragma unroll
            for (int s = 0; s < ND; ++s)
                fx_add(a.J, mb + (size_t)(fc + l) * n + fd + s, f * (double)jcd[l * ND + s]);
    }
    if (a.want_k) {
#pragma unroll 1
        for (int q = 0; q < a.nk; ++q) {
            const double* Dq = a.D + (size_t)q * a.mstride;
            acc_t* Kq = a.K + 2 * (size_t)q * a.mstride;
            R dbd[NB * ND], dbc[NB * NC], dad[NA * ND], dac[NA * NC];
            R kac[NA * NC], kad[NA * ND], kbc[NB * NC], kbd[NB * ND];
#pragma unroll
            for (int k = 0; k < NB; ++k) {
#pragma unroll
                for (int s = 0; s < ND; ++s) { dbd[k * ND + s] = ldR<R>(Dq + mb + (size_t)(fb + k) * n + fd + s); kbd[k * ND + s] = R(0); }
#pragma unroll
                for (int l = 0; l < NC; ++l) { dbc[k * NC + l] = ldR<R>(Dq + mb + (size_t)(fb + k) * n + fc + l); kbc[k * NC + l] = R(0); }
            }
#pragma unroll
            for (int m = 0; m < NA; ++m) {
#pragma unroll
                for (int s = 0; s < ND; ++s) { dad[m * ND + s] = ldR<R>(Dq + mb + (size_t)(fa + m) * n + fd + s); kad[m * ND + s] = R(0); }
#pragma unroll
                for (int l = 0; l < NC; ++l) { dac[m * NC + l] = ldR<R>(Dq + mb + (size_t)(fa + m) * n + fc + l); kac[m * NC + l] = R(0); }
            }
#pragma unroll
            for (int m = 0; m < NA; ++m)
#pragma unroll
                for (int k = 0; k < NB; ++k)
#pragma unroll
                    for (int l = 0; l < NC; ++l)
#pragma unroll
                        for (int s = 0; s < ND; ++s) {
                            const R v = I[((m * NB + k) * NC + l) * ND + s];
                            kac[m * NC + l] = fma(v, dbd[k * ND + s], kac[m * NC + l]);
                            kad[m * ND + s] = fma(v, dbc[k * NC + l], kad[m * ND + s]);
                            kbc[k * NC + l] = fma(v, dad[m * ND + s], kbc[k * NC + l]);
                            kbd[k * ND + s] = fma(v, dac[m * NC + l], kbd[k * ND + s]);
                        }
            const double f = (double)sdeg;
#pragma unroll
            for (int m = 0; m < NA; ++m) {
#pragma unroll
                for (int l = 0; l < NC; ++l) fx_add(Kq, mb + (size_t)(fa + m) * n + fc + l, f * (double)kac[m * NC + l]);
#pragma unroll
                for (int s = 0; s < ND; ++s) fx_add(Kq, mb + (size_t)(fa + m) * n + fd + s, f * (double)kad[m * ND + s]);
            }
#pragma unroll
            for (int k = 0; k < NB; ++k) {
#pragma unroll
                for (int l = 0; l < NC; ++l) fx_add(Kq, mb + (size_t)(fb + k) * n + fc + l, f * (double)kbc[k * NC + l]);
#pragma unroll
                for (int s = 0; s < ND; ++s) fx_add(Kq, mb + (size_t)(fb + k) * n + fd + s, f * (double)kbd[k * ND + s]);
            }
        }
    }
}

// Digestion of the integral subset owned by one lane of a G-lane group
// (bra function pairs mn = sub, sub+G, ...).  Adds the lane's partial J'_cd
// and K' blocks to jcd / kblk (zeroed by the caller) and adds its J'_ab elements.
template <int LA, int LB, int LC, int LD, typename R, int G>
__device__ __forceinline__ void digest_part(const PairHdr& B, const PairHdr& K, const R* __restrict__ I,
                                            R sdeg, const JKArgs& a, int q, int sub,
                                            R* __restrict__ jcd, R* __restrict__ kblk)
{
    constexpr int NA = ncart(LA), NB = ncart(LB), NC = ncart(LC), ND = ncart(LD);
    constexpr int NCD = NC * ND;
    R* kac = kblk;
    R* kad = kac + NA * NC;
    R* kbc = kad + NA * ND;
    R* kbd = kbc + NB * NC;
    const int n = a.nbf;
    const int fa = B.bfa, fb = B.bfb, fc = K.bfa, fd = K.bfb;
    const long long mb = B.mbase;
    const double* Dq = a.D + (size_t)q * a.mstride;
    if (q == 0 && a.want_j) {
        R dcd[NCD];
#pragma unroll
        for (int l = 0; l < NC; ++l)
#pragma unroll
            for (int s = 0; s < ND; ++s) dcd[l * ND + s] = ldR<R>(Dq + mb + (size_t)(fc + l) * n + fd + s);
#pragma unroll 1
        for (int mn = sub; mn < NA * NB; mn += G) {
            const int m = mn / NB, k = mn - (mn / NB) * NB;
            const R dab = ldR<R>(Dq + mb + (size_t)(fa + m) * n + fb + k);
            R t = R(0);
#pragma unroll
            for (int ls = 0; ls < NCD; ++ls) {
                const R v = I[mn * NCD + ls];
                t = fma(v, dcd[ls], t);
                jcd[ls] = fma(v, dab, jcd[ls]);
            }
            fx_add(a.J, mb + (size_t)(fa + m) * n + fb + k, 2.0 * (double)sdeg * (double)t);
        }
    }
    if (a.want_k) {
#pragma unroll 1
        for (int mn = sub; mn < NA * NB; mn += G) {
            const int m = mn / NB, k = mn - (mn / NB) * NB;
            R dbd[ND], dbc[NC], dad[ND], dac[NC];
#pragma unroll
            for (int s = 0; s < ND; ++s) {
                dbd[s] = ldR<R>(Dq + mb + (size_t)(fb + k) * n + fd + s);
                dad[s] = ldR<R>(Dq + mb + (size_t)(fa + m) * n + fd + s);
            }
#pragma unroll
            for (int l = 0; l < NC; ++l) {
                dbc[l] = ldR<R>(Dq + mb + (size_t)(fb + k) * n + fc + l);
                dac[l] = ldR<R>(Dq + mb + (size_t)(fa + m) * n + fc + l);
            }
#pragma unroll
            for (int l = 0; l < NC; ++l)
#pragma unroll
                for (int s = 0; s < ND; ++s) {
                    const R v = I[mn * NCD + l * ND + s];
                    kac[m * NC + l] = fma(v, dbd[s], kac[m * NC + l]);
                    kad[m * ND + s] = fma(v, dbc[l], kad[m * ND + s]);
                    kbc[k * NC + l] = fma(v, dad[s], kbc[k * NC + l]);
                    kbd[k * ND + s] = fma(v, dac[l], kbd[k * ND + s]);
                }
        }
    }
}

template <typename T, int G>
__device__ __forceinline__ T group_sum(T v)
{
#pragma unroll
    for (int o = G / 2; o > 0; o >>= 1) v += shfl_xor_r(v, o);
    return v;
}

// Screening and precision split of every candidate quartet (one warp per
// static task of candidates): survivors are appended, warp-aggregated, to the
// class's FP64 list (from the front of its region) or FP32 list (from the
// back).  cls_task_off/cls_qoff: per-class offsets of tasks and list regions.
struct ClassifyArgs {
    const PairHdr* pairs;
    const int4* tasks;
    int ntasks;
    const int* cls_task_off;      // NQC + 1
    const long long* cls_qoff;    // NQC + 1
    const float* Q;
    const float* Dmax;
    int nsh;
    float tau, tau_mixed;
    float tau_64;                 // double-float tier for bounds in [tau_mixed, tau_64) (off if <= tau_mixed)
    int split;                    // 0: every survivor to the FP64 list
    // optional per-molecule mode (batched drivers): bit 0 allows the FP32
    // list for the molecule's quartets, bit 1 skips the molecule; NULL: every
    // molecule follows `split`
    const int* mol_mode;
    long long lds2;               // shell-block slot size (smbase / lds2 = molecule)
    int2* qlist;
    unsigned int* qcount;         // [NQC][3] survivors per precision: FP64, FP32, double-float
};

// Largest grid (CTAs) of a lane-group launch on the current device: the
// kernels stride over their list, so longer lists reuse resident warps
// instead of launching warps that find nothing to do.
int jk_grid_cap();

// Lane-group evaluation of list chunk w: a group of G lanes evaluates one
// contracted quartet, its lanes splitting the primitive quartets;
// accumulators and digested blocks are summed across the group with
// shuffles.  The chunk is list entries [w*S, w*S + S), S = 32/G.
template <int LA, int LB, int LC, int LD, typename R, int G>
__device__ __forceinline__ void jk_chunk(const JKArgs& a, const long long w, const long long cnt)
{
    constexpr int NA = ncart(LA), NB = ncart(LB), NC = ncart(LC), ND = ncart(LD);
    constexpr int NKB = NA * NC + NA * ND + NB * NC + NB * ND;
    constexpr int S = 32 / G;
    using C = EriClass<LA, LB, LC, LD>;
    const int lane = threadIdx.x & 31;
    const int grp = lane / G, sub = lane - (lane / G) * G;
    if (w * S >= cnt) return;
    const long long idx = w * S + grp;
    const bool on = idx < cnt;
    const int2 e = a.qlist[(list_base(a) + (on ? idx : w * S)) * a.qdir];
    const PairHdr B = a.pairs[e.x];
    const PairHdr K = a.pairs[e.y];
    R acc[C::NACC];
#pragma unroll
    for (int i = 0; i < C::NACC; ++i) acc[i] = R(0);
    unsigned long long nq = 0, np = 0;
    if (on) {
        const int nkp = K.nprim, tot = B.nprim * K.nprim;
        if constexpr (G == 1) {
            for (int ip = 0; ip < B.nprim; ++ip) {
                PrimPairT<R> bp;
                load_prim<R>(a, B.poff + ip, bp);
                for (int jp = 0; jp < nkp; ++jp) {
                    PrimPairT<R> kp;
                    load_prim<R>(a, K.poff + jp, kp);
                    prim_quartet<LA, LB, LC, LD, R>(bp, kp, a.boys_d, a.boys_f, acc);
                }
            }
        } else {
            // primitive quartets sub, sub + G, ... of the ip-major order
            int ip = 0, jp = sub;
            while (jp >= nkp) { jp -= nkp; ++ip; }
            for (int pq = sub; pq < tot; pq += G) {
                PrimPairT<R> bp, kp;
                load_prim<R>(a, B.poff + ip, bp);
                load_prim<R>(a, K.poff + jp, kp);
                prim_quartet<LA, LB, LC, LD, R>(bp, kp, a.boys_d, a.boys_f, acc);
                jp += G;
                while (jp >= nkp) { jp -= nkp; ++ip; }
            }
        }
        if (sub == 0) { nq = 1; np = (unsigned long long)tot; }
    }
    if constexpr (G > 1) {
#pragma unroll
        for (int i = 0; i < C::NACC; ++i) acc[i] = group_sum<R, G>(acc[i]);
    }
    R sdeg = R(1);
    if (B.a == B.b) sdeg *= R(0.5);
    if (K.a == K.b) sdeg *= R(0.5);
    if (e.x == e.y) sdeg *= R(0.5);
    if constexpr (G == 1) {
        double jq[NA * NB];
#pragma unroll
        for (int i = 0; i < NA * NB; ++i) jq[i] = 0.0;
        if (on) {
            R I[C::N];
            R ABv[3] = {(R)B.AB[0], (R)B.AB[1], (R)B.AB[2]};
            R CDv[3] = {(R)K.AB[0], (R)K.AB[1], (R)K.AB[2]};
            C::template hrr<R>(acc, ABv, CDv, I);
            digest<LA, LB, LC, LD, R>(B, K, I, sdeg, a, jq);
        }
        if (a.want_j) {
            // J'_ab: segmented warp sum over runs of lanes with the same bra
            // pair (list entries of one bra are contiguous), one add per run
            const int my = on ? e.x : -1;
            const int prev = __shfl_up_sync(0xffffffffu, my, 1);
            const bool head = lane == 0 || prev != my;
            const unsigned heads = __ballot_sync(0xffffffffu, head);
            const int seg = __popc(heads & (0xffffffffu >> (31 - lane)));
            bool same[5];
#pragma unroll
            for (int k = 0; k < 5; ++k) {
                const int o = 1 << k;
                const int so = __shfl_down_sync(0xffffffffu, seg, o);
                same[k] = (lane + o < 32) && so == seg;
            }
#pragma unroll
            for (int i = 0; i < NA * NB; ++i) {
                double v = jq[i];
#pragma unroll
                for (int k = 0; k < 5; ++k) {
                    const double u = __shfl_down_sync(0xffffffffu, v, 1 << k);
                    if (same[k]) v += u;
                }
                if (head && on && v != 0.0)
                    fx_add(a.J, B.mbase + (size_t)(B.bfa + i / NB) * a.nbf + B.bfb + i % NB, v);
            }
        }
    } else {
        R I[C::N];
        if (on) {
            R ABv[3] = {(R)B.AB[0], (R)B.AB[1], (R)B.AB[2]};
            R CDv[3] = {(R)K.AB[0], (R)K.AB[1], (R)K.AB[2]};
            C::template hrr<R>(acc, ABv, CDv, I);
        }
        const int n = a.nbf;
        const int fa = B.bfa, fb = B.bfb, fc = K.bfa, fd = K.bfb;
    const long long mb = B.mbase;
#pragma unroll 1
        for (int q = 0; q < a.nk; ++q) {
            if (q > 0 && !a.want_k) break;
            R jcd[NC * ND], kb[NKB];
#pragma unroll
            for (int i = 0; i < NC * ND; ++i) jcd[i] = R(0);
#pragma unroll
            for (int i = 0; i < NKB; ++i) kb[i] = R(0);
            if (on) digest_part<LA, LB, LC, LD, R, G>(B, K, I, sdeg, a, q, sub, jcd, kb);
            if (q == 0 && a.want_j) {
                const double f = 2.0 * (double)sdeg;
#pragma unroll
                for (int l = 0; l < NC; ++l)
#pragma unroll
                    for (int s = 0; s < ND; ++s) {
                        const R v = group_sum<R, G>(jcd[l * ND + s]);
                        if (on && ((l * ND + s) % G) == sub)
                            fx_add(a.J, mb + (size_t)(fc + l) * n + fd + s, f * (double)v);
                    }
            }
            if (a.want_k) {
                acc_t* Kq = a.K + 2 * (size_t)q * a.mstride;
                const double f = (double)sdeg;
                int e2 = 0;
#pragma unroll
                for (int m = 0; m < NA; ++m)
#pragma unroll
                    for (int l = 0; l < NC; ++l, ++e2) {
                        const R v = group_sum<R, G>(kb[m * NC + l]);
                        if (on && (e2 % G) == sub) fx_add(Kq, mb + (size_t)(fa + m) * n + fc + l, f * (double)v);
                    }
#pragma unroll
                for (int m = 0; m < NA; ++m)
#pragma unroll
                    for (int s = 0; s < ND; ++s, ++e2) {
                        const R v = group_sum<R, G>(kb[NA * NC + m * ND + s]);
                        if (on && (e2 % G) == sub) fx_add(Kq, mb + (size_t)(fa + m) * n + fd + s, f * (double)v);
                    }
#pragma unroll
                for (int k = 0; k < NB; ++k)
#pragma unroll
                    for (int l = 0; l < NC; ++l, ++e2) {
                        const R v = group_sum<R, G>(kb[NA * NC + NA * ND + k * NC + l]);
                        if (on && (e2 % G) == sub) fx_add(Kq, mb + (size_t)(fb + k) * n + fc + l, f * (double)v);
                    }
#pragma unroll
                for (int k = 0; k < NB; ++k)
#pragma unroll
                    for (int s = 0; s < ND; ++s, ++e2) {
                        const R v = group_sum<R, G>(kb[NA * NC + NA * ND + NB * NC + k * ND + s]);
                        if (on && (e2 % G) == sub) fx_add(Kq, mb + (size_t)(fb + k) * n + fd + s, f * (double)v);
                    }
            }
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

// Lane-group kernel over a compacted quartet list: warp w evaluates chunks
// w, w + W, w + 2W, ... (W warps in the grid) until the device-side count.
template <int LA, int LB, int LC, int LD, typename R, int G>
__global__ void __launch_bounds__(JK_THREADS) jk_kernel(const JKArgs a)
{
    constexpr int S = 32 / G;
    const long long cnt = (long long)*a.qcount;
    const long long nw = ((long long)gridDim.x * JK_THREADS) >> 5;
    for (long long w = ((long long)blockIdx.x * JK_THREADS + threadIdx.x) >> 5; w * S < cnt; w += nw)
        jk_chunk<LA, LB, LC, LD, R, G>(a, w, cnt);
}

// Schwarz factors of the pairs [begin, end) of class (LA LB): a group of G
// lanes per pair splits its primitive quartets (ab|ab), the group sums the
// accumulators with shuffles and its first lane runs the HRR and takes the
// largest diagonal element, all in FP64.
template <int LA, int LB, int G>
__global__ void __launch_bounds__(JK_THREADS) schwarz_kernel(const JKArgs a, int begin, int end, float* Qf, double* Qd)
{
    constexpr int NA = ncart(LA), NB = ncart(LB);
    using C = EriClass<LA, LB, LA, LB>;
    const int lane = threadIdx.x & 31;
    const int grp = lane / G, sub = lane - (lane / G) * G;
    const long long w = ((long long)blockIdx.x * JK_THREADS + threadIdx.x) >> 5;
    const long long p0 = begin + w * (32 / G);
    if (p0 >= end) return;                       // whole warp past the end
    const long long p = p0 + grp;
    const bool on = p < end;
    const PairHdr B = a.pairs[on ? p : p0];
    double acc[C::NACC];
#pragma unroll
    for (int i = 0; i < C::NACC; ++i) acc[i] = 0.0;
    if (on) {
        const int tot = B.nprim * B.nprim;
        for (int pq = sub; pq < tot; pq += G) {
            const int ip = pq / B.nprim, jp = pq - (pq / B.nprim) * B.nprim;
            PrimPairT<double> bp, kp;
            load_prim<double>(a, B.poff + ip, bp);
            load_prim<double>(a, B.poff + jp, kp);
            prim_quartet<LA, LB, LA, LB, double>(bp, kp, a.boys_d, a.boys_f, acc);
        }
    }
    if constexpr (G > 1) {
#pragma unroll
        for (int i = 0; i < C::NACC; ++i) acc[i] = group_sum<double, G>(acc[i]);
    }
    if (!on || sub != 0) return;
    double I[C::N];
    const double ABv[3] = {B.AB[0], B.AB[1], B.AB[2]};
    C::template hrr<double>(acc, ABv, ABv, I);
    double mx = 0.0;
#pragma unroll
    for (int m = 0; m < NA; ++m)
#pragma unroll
        for (int k = 0; k < NB; ++k) {
            const double v = fabs(I[((m * NB + k) * NA + m) * NB + k]);
            mx = v > mx ? v : mx;
        }
    const double q = sqrt(mx);
    Qd[p] = q;
    Qf[p] = (float)q * 1.0000005f;   // round up: a bound must not shrink in FP32
}

}  // namespace cq
