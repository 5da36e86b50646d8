// Direct Fock build J, K <- P (Eq. 2c_fock), over unique shell quartets.
//
// Conventions.  The integral kernels evaluate (ab|cd) for the x^L
// normalisation of every shell; the Cartesian component factors s_m are
// applied to the density on the way in (P'_{mn} = s_m s_n P_{mn}) and to J
// and K on the way out.  Each unique quartet (a>=b, c>=d, ab>=cd) carries the
// degeneracy factor sdeg = (1/2 if a==b)(1/2 if c==d)(1/2 if ab==cd) and adds
//     J'_ab += 2 sdeg (ab|cd) D_cd,   J'_cd += 2 sdeg (ab|cd) D_ab,
//     K'_ac += sdeg (ab|cd) D_bd,  K'_ad += sdeg (ab|cd) D_bc,
//     K'_bc += sdeg (ab|cd) D_ad,  K'_bd += sdeg (ab|cd) D_ac,
// after which J = J' + J'^T and K = K' + K'^T for a symmetric density or
// K = K' - K'^T for an antisymmetric one (the eight index permutations of a
// real integral folded into four accumulations and one transpose).
//
// A Hermitian P = P_R + i P_I has P_R symmetric and P_I antisymmetric, so
// J[P] = J[P_R] and K[P] = K[P_R] + i K[P_I]; the Pauli case applies this
// to P^0..P^3 (eight real K matrices, J from Re P^0).
#include <cstring>

#include <algorithm>
#include <climits>
#include <vector>

#include "cq_internal.h"
#include "cq_jk.cuh"

namespace cq {

// Matrices are stored as one slot per molecule: element (r, c) of molecule
// m at m*ld*ld + r*ld + c, ld = the largest molecule's function count (for a
// single molecule ld = nbf and the layout is the plain row-major matrix).
// P (layout by kind) -> nk scaled real matrices; padding elements -> 0.
__global__ void density_prep_kernel(int kind, int nmol, int ld, const int* __restrict__ mol_n,
                                    const int* __restrict__ mol_bfo, const double* __restrict__ P,
                                    const double* __restrict__ sc, double* __restrict__ Dp)
{
    const size_t slot = (size_t)ld * ld, ms = slot * nmol;
    const size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= ms) return;
    const int m = (int)(i / slot);
    const int r = (int)((i / ld) % ld), c = (int)(i % ld);
    const int nm = mol_n[m];
    const double f = (r < nm && c < nm) ? sc[mol_bfo[m] + r] * sc[mol_bfo[m] + c] : 0.0;
    if (kind == CQ_DENS_REAL_SYM) {
        Dp[i] = f * P[i];
    } else if (kind == CQ_DENS_COMPLEX_HERM) {
        Dp[i] = f * P[2 * i];
        Dp[ms + i] = f * P[2 * i + 1];
    } else if (kind == CQ_DENS_REAL_GENERAL) {
        // symmetric and antisymmetric parts, handled as Re and Im of S + iA
        const size_t t = (size_t)m * slot + (size_t)c * ld + r;
        Dp[i] = 0.5 * f * (P[i] + P[t]);
        Dp[ms + i] = 0.5 * f * (P[i] - P[t]);
    } else {
        for (int I = 0; I < 4; ++I) {
            Dp[(2 * I) * ms + i] = f * P[2 * (I * ms + i)];
            Dp[(2 * I + 1) * ms + i] = f * P[2 * (I * ms + i) + 1];
        }
    }
}

// Shell-block maxima of |P'| over all nk matrices, one slot of lds x lds
// per molecule (lds = the largest molecule's shell count).
__global__ void dmax_kernel(int nmol, int ld, int lds, const int* __restrict__ mol_nsh, const int* __restrict__ mol_sho,
                            const int* __restrict__ mol_bfo, const int* __restrict__ bfo, int nk,
                            const double* __restrict__ Dp, const int* __restrict__ mol_mode, float* __restrict__ Dmax)
{
    const size_t sslot = (size_t)lds * lds;
    const size_t p = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= sslot * nmol) return;
    const int m = (int)(p / sslot);
    const int sa = (int)((p / lds) % lds), sb = (int)(p % lds);
    if (sa >= mol_nsh[m] || sb >= mol_nsh[m] || (mol_mode && (mol_mode[m] & 2))) { Dmax[p] = 0.f; return; }
    const int a = mol_sho[m] + sa, b = mol_sho[m] + sb, f0 = mol_bfo[m];
    const size_t slot = (size_t)ld * ld, ms = slot * nmol;
    double mx = 0.0;
    for (int q = 0; q < nk; ++q)
        for (int i = bfo[a]; i < bfo[a + 1]; ++i)
            for (int j = bfo[b]; j < bfo[b + 1]; ++j)
                mx = fmax(mx, fabs(Dp[(size_t)q * ms + m * slot + (size_t)(i - f0) * ld + (j - f0)]));
    Dmax[p] = (float)mx * 1.0000005f;
}

// X'_i + sgn X'_t of two fixed-point accumulator elements, summed as integers
// and rounded once to FP64.
__device__ __forceinline__ double fx_pair(const acc_t* __restrict__ X, size_t i, size_t t, bool minus)
{
    const long long hi_i = (long long)X[2 * i], lo_i = (long long)X[2 * i + 1];
    const long long hi_t = (long long)X[2 * t], lo_t = (long long)X[2 * t + 1];
    return minus ? fx_value(hi_i - hi_t, lo_i - lo_t) : fx_value(hi_i + hi_t, lo_i + lo_t);
}

// J = s s (J' + J'^T); K_q = s s (K'_q +/- K'_q^T), per slot, in the output layout.
__global__ void finalize_kernel(int kind, int nmol, int ld, const int* __restrict__ mol_n,
                                const int* __restrict__ mol_bfo, const double* __restrict__ sc,
                                const acc_t* __restrict__ Jp, const acc_t* __restrict__ Kp, double* __restrict__ J,
                                double* __restrict__ K, int want_j, int want_k)
{
    const size_t slot = (size_t)ld * ld, ms = slot * nmol;
    const size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= ms) return;
    const int m = (int)(i / slot);
    const int r = (int)((i / ld) % ld), c = (int)(i % ld);
    const size_t t = (size_t)m * slot + (size_t)c * ld + r;
    const int nm = mol_n[m];
    const double f = (r < nm && c < nm) ? sc[mol_bfo[m] + r] * sc[mol_bfo[m] + c] : 0.0;
    if (want_j) J[i] = f * fx_pair(Jp, i, t, false);
    if (!want_k) return;
    if (kind == CQ_DENS_REAL_SYM) {
        K[i] = f * fx_pair(Kp, i, t, false);
    } else if (kind == CQ_DENS_COMPLEX_HERM) {
        K[2 * i] = f * fx_pair(Kp, i, t, false);
        K[2 * i + 1] = f * fx_pair(Kp + 2 * ms, i, t, true);
    } else if (kind == CQ_DENS_REAL_GENERAL) {
        K[i] = f * (fx_pair(Kp, i, t, false) + fx_pair(Kp + 2 * ms, i, t, true));   // K[S] + K[A]
    } else {
        for (int I = 0; I < 4; ++I) {
            const acc_t* Kr = Kp + 2 * (2 * I) * ms;
            const acc_t* Ki = Kp + 2 * (2 * I + 1) * ms;
            K[2 * (I * ms + i)] = f * fx_pair(Kr, i, t, false);
            K[2 * (I * ms + i) + 1] = f * fx_pair(Ki, i, t, true);
        }
    }
}

__global__ void counter_total_kernel(unsigned long long* c)
{
    if (threadIdx.x < 6) {
        unsigned long long t = 0;
        for (int q = 0; q < NQC; ++q) t += c[6 + 6 * q + threadIdx.x];
        // [0] fp64 quartets [1] fp64 prims [2] fp32 quartets [3] fp32 prims
        // [4] double-float quartets [5] double-float prims
        c[threadIdx.x] = t;
    }
}

static int nk_of(int kind) { return dens_nk(kind); }

int ensure_scratch(cq_basis* b, int nk)
{
    if (nk <= b->nk_cap) return CQ_OK;
    const size_t nn = b->mstride;
    if (b->d_Dp) cudaFree(b->d_Dp);
    if (b->d_Kp) cudaFree(b->d_Kp);
    b->d_Dp = nullptr;
    b->d_Kp = nullptr;
    int rc;
    if ((rc = dalloc(&b->d_Dp, nn * nk))) return rc;
    if ((rc = dalloc(&b->d_Kp, 2 * nn * nk))) return rc;
    if (!b->d_Jp && (rc = dalloc(&b->d_Jp, 2 * nn))) return rc;
    if (!b->d_Dmax && (rc = dalloc(&b->d_Dmax, (size_t)b->nmol * b->lds * b->lds))) return rc;
    b->nk_cap = nk;
    return CQ_OK;
}

// Screening and precision split of the candidates of one static task:
// returns this lane's class of candidate j0 + lane (-1 rejected, 0 FP64,
// 1 FP32, 2 double-float).
__device__ __forceinline__ int classify_one(const ClassifyArgs& c, const float* Dm, int j, int jend, int ba, int bb,
                                            float Qb, float dab, int mode)
{
    if (j >= jend || (mode & 2)) return -1;
    const int ns = c.nsh;
    const int kc = __ldg(&c.pairs[j].sa), kd = __ldg(&c.pairs[j].sb);
    float m = fmaxf(dab, __ldg(Dm + kc * ns + kd));
    m = fmaxf(m, fmaxf(__ldg(Dm + ba * ns + kc), __ldg(Dm + ba * ns + kd)));
    m = fmaxf(m, fmaxf(__ldg(Dm + bb * ns + kc), __ldg(Dm + bb * ns + kd)));
    const float bound = Qb * __ldg(c.Q + j) * m;
    if (!(bound >= c.tau)) return -1;
    if (!(mode & 1)) return 0;
    if (bound < c.tau_mixed) return 1;
    return bound < c.tau_64 ? 2 : 0;
}

// Pass 1 (write = 0): survivors per task and precision -> tcount[3t + p].
// Pass 3 (write = 1): survivors written at the scanned offsets, in task
// order and, within a task, in ket order, so that a warp of the integral
// kernels gets consecutive kets of mostly one bra with similar primitive
// counts.  FP64 entries fill a class's region from the front, FP32 entries
// from the back, double-float entries follow the FP64 ones (their base is
// the class's FP64 total from the scan).
__global__ void classify_kernel(const ClassifyArgs c, int nqc, int write, unsigned int* __restrict__ tcount,
                                const unsigned int* __restrict__ toff)
{
    const int lane = threadIdx.x & 31;
    const int w = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (w >= c.ntasks) return;
    int qc = 0;
    while (qc + 1 < nqc && c.cls_task_off[qc + 1] <= w) ++qc;
    const int4 t = c.tasks[w];
    const int ib = t.x;
    const int ba = __ldg(&c.pairs[ib].sa), bb = __ldg(&c.pairs[ib].sb);
    const float Qb = __ldg(c.Q + ib);
    const long long smb = __ldg(&c.pairs[ib].smbase);
    const float* Dm = c.Dmax + smb;
    const float dab = __ldg(Dm + ba * c.nsh + bb);
    const int mode = c.mol_mode ? (__ldg(c.mol_mode + smb / c.lds2) & (c.split ? 3 : 2)) : (c.split ? 1 : 0);
    const long long base = c.cls_qoff[qc], top = c.cls_qoff[qc + 1];
    unsigned int n0 = 0, n1 = 0, n2 = 0;
    unsigned int o0 = write ? toff[3 * w] : 0, o1 = write ? toff[3 * w + 1] : 0;
    unsigned int o2 = write ? toff[3 * w + 2] + c.qcount[3 * qc] : 0;
    // a skipped molecule's task has no survivors (the whole warp agrees)
    const int jend = (mode & 2) ? t.y : t.z;
    for (int j0 = t.y; j0 < jend; j0 += 32) {
        const int j = j0 + lane;
        const int prec = classify_one(c, Dm, j, t.z, ba, bb, Qb, dab, mode);
        const unsigned m0 = __ballot_sync(0xffffffffu, prec == 0);
        const unsigned m1 = __ballot_sync(0xffffffffu, prec == 1);
        const unsigned m2 = __ballot_sync(0xffffffffu, prec == 2);
        if (write) {
            const unsigned below = (1u << lane) - 1u;
            if (prec == 0) c.qlist[base + o0 + n0 + __popc(m0 & below)] = make_int2(ib, j);
            if (prec == 1) c.qlist[top - 1 - (o1 + n1 + __popc(m1 & below))] = make_int2(ib, j);
            if (prec == 2) c.qlist[base + o2 + n2 + __popc(m2 & below)] = make_int2(ib, j);
        }
        n0 += __popc(m0);
        n1 += __popc(m1);
        n2 += __popc(m2);
    }
    if (!write && lane == 0) {
        tcount[3 * w] = n0;
        tcount[3 * w + 1] = n1;
        tcount[3 * w + 2] = n2;
    }
}

// Exclusive scan (one CTA) of the per-task survivor counts of tasks
// [t0, t1) into offsets within their list region, and the list lengths.
__device__ __forceinline__ void scan_range(int t0, int t1, const unsigned int* __restrict__ tcount,
                                          unsigned int* __restrict__ toff, unsigned int* __restrict__ qcount)
{
    __shared__ unsigned int part[3][1024];
    const int n = t1 - t0;
    const int per = (n + blockDim.x - 1) / blockDim.x;
    const int b0 = t0 + threadIdx.x * per, b1 = min(t1, b0 + per);
    unsigned int sp[3] = {0, 0, 0};
    for (int t = b0; t < b1; ++t)
        for (int p = 0; p < 3; ++p) sp[p] += tcount[3 * t + p];
    for (int p = 0; p < 3; ++p) part[p][threadIdx.x] = sp[p];
    __syncthreads();
    if (threadIdx.x < 3) {
        const int p = threadIdx.x;
        unsigned int acc = 0;
        for (int i = 0; i < (int)blockDim.x; ++i) {
            const unsigned int x = part[p][i];
            part[p][i] = acc;
            acc += x;
        }
        qcount[p] = acc;
    }
    __syncthreads();
    unsigned int ap[3] = {part[0][threadIdx.x], part[1][threadIdx.x], part[2][threadIdx.x]};
    for (int t = b0; t < b1; ++t)
        for (int p = 0; p < 3; ++p) {
            toff[3 * t + p] = ap[p];
            ap[p] += tcount[3 * t + p];
        }
}

// Pass 2: per class (one CTA each), the scan over the class's tasks.
__global__ void scan_tasks_kernel(const int* __restrict__ cls_task_off, const unsigned int* __restrict__ tcount,
                                  unsigned int* __restrict__ toff, unsigned int* __restrict__ qcount)
{
    const int qc = blockIdx.x;
    scan_range(cls_task_off[qc], cls_task_off[qc + 1], tcount, toff, qcount + 3 * qc);
}

// The same over the n tasks of one pass (one CTA).
__global__ void scan_pass_kernel(int n, const unsigned int* __restrict__ tcount, unsigned int* __restrict__ toff,
                                 unsigned int* __restrict__ qcount)
{
    scan_range(0, n, tcount, toff, qcount);
}

// Precisions a build evaluates: FP64 only, FP64 + FP32, or FP64 + FP32 +
// double-float (mixed builds with fp64_tol above mixed_tol).
static int n_precisions(const cq_fock_opts& o)
{
    if (o.prec == CQ_PREC_FP64) return 1;
    return o.fp64_tol > o.mixed_tol ? 3 : 2;
}

// List and screening arguments of precision pp of one class: FP64 entries
// from the front of the class's region, FP32 from the back, double-float
// after the FP64 ones; qcnt points at the class's three survivor counts.
static void set_precision(JKArgs& a, const cq_fock_opts& o, int pp, int2* region, int2* region_last,
                          unsigned int* qcnt)
{
    const bool three = n_precisions(o) == 3;
    a.prec_sel = (o.prec == CQ_PREC_FP64) ? 0 : (pp == 0 ? 1 : 2);   // cooperative kernel's own screening
    a.tau_mixed = (float)((pp == 0 && three) ? o.fp64_tol : o.mixed_tol);
    a.qlist = pp == 1 ? region_last : region;
    a.qdir = pp == 1 ? -1 : 1;
    a.qcount = qcnt + pp;
    a.qbase = pp == 2 ? qcnt : nullptr;
    a.fp64_tier = three && pp == 0;
}

static const int CLASS_ORDER[NQC] = {20, 19, 18, 17, 16, 14, 13, 15, 12, 11, 10, 9, 8, 7, 5, 6, 4, 3, 2, 1, 0};

// Large bases: per class, runs of whole tasks whose candidates fit the list
// are screened into it and drained by the class kernel(s) in turn, on one
// stream.  The cooperative kernel reads its quartets from the list.
static int launch_passes(const cq_basis* b, JKArgs& a, ClassifyArgs c, const cq_fock_opts& o, bool profile,
                         cudaStream_t s)
{
    cq_basis* bm = const_cast<cq_basis*>(b);
    const long long cap = std::min<long long>(b->list_cap, 1LL << 30);
    c.cls_qoff = b->d_pass_qoff;   // FP64 (then double-float) entries from the front, FP32 from the back
    const int npp = n_precisions(o);
    for (int oi = 0; oi < NQC; ++oi) {
        const int qc = CLASS_ORDER[oi];
        const int t0 = b->task_off[qc], t1 = b->task_off[qc + 1];
        if (t0 == t1) continue;
        int X = 0;
        while ((X + 1) * (X + 2) / 2 <= qc) ++X;
        const int Y = qc - X * (X + 1) / 2;
        a.ket_end = b->cls_off[Y + 1];
        a.same_class = (X == Y);
        for (int ta = t0; ta < t1;) {
            const long long base = b->task_cand[ta];
            int tb = (int)(std::upper_bound(b->task_cand.begin() + ta + 1, b->task_cand.begin() + t1 + 1, base + cap) -
                           b->task_cand.begin()) - 1;
            if (tb <= ta) {
                set_error("cq_fock_build: one bra pair has more candidate quartets than the list capacity");
                return CQ_ERR_UNSUPPORTED;
            }
            const long long cand = b->task_cand[tb] - base;
            c.tasks = b->d_tasks + ta;
            c.ntasks = tb - ta;
            const int blocks = (int)(((long long)c.ntasks * 32 + 255) / 256);
            c.qcount = b->d_qcount + 3 * qc;   // the pass's counts (read as class 0 of one)
            classify_kernel<<<blocks, 256, 0, s>>>(c, 1, 0, b->d_tcount + 3 * (size_t)ta, nullptr);
            scan_pass_kernel<<<1, 1024, 0, s>>>(c.ntasks, b->d_tcount + 3 * (size_t)ta, b->d_toff + 3 * (size_t)ta,
                                                b->d_qcount + 3 * qc);
            classify_kernel<<<blocks, 256, 0, s>>>(c, 1, 1, nullptr, b->d_toff + 3 * (size_t)ta);
            a.tasks = c.tasks;
            a.ntasks = c.ntasks;
            a.qmax = cand;
            for (int pp = 0; pp < npp; ++pp) {
                set_precision(a, o, pp, b->d_qlist, b->d_qlist + (b->list_cap - 1), b->d_qcount + 3 * qc);
                unsigned long long* base_cnt = a.counters;
                a.counters = base_cnt + 6 * qc + 2 * pp;
                cudaEvent_t* ev = nullptr;
                if (profile) {   // one event pair per pass, summed by cq_fock_class_stats
                    auto& v = bm->pev_pass[qc][pp];
                    const int k = bm->pev_npass[qc][pp]++;
                    while ((int)v.size() < 2 * (k + 1)) {
                        cudaEvent_t e;
                        CQ_CUDA(cudaEventCreate(&e));
                        v.push_back(e);
                    }
                    ev = &v[2 * k];
                    CQ_CUDA(cudaEventRecord(ev[0], s));
                }
                launch_jk_class(b, a, qc, pp, s);
                if (profile) {
                    CQ_CUDA(cudaEventRecord(ev[1], s));
                    bm->pev_used[qc][pp] = true;
                }
                a.counters = base_cnt;
            }
            CQ_CUDA(cudaGetLastError());
            ta = tb;
        }
    }
    return CQ_OK;
}

// Screen and split every candidate quartet into the per-class lists (one
// kernel), then launch every class kernel, heaviest classes first.
int classify_and_launch(const cq_basis* b, JKArgs& a, const cq_fock_opts& o, bool profile, cudaStream_t s,
                        const int* mol_mode)
{
    ClassifyArgs c;
    c.mol_mode = mol_mode;
    c.lds2 = (long long)b->lds * b->lds;
    c.pairs = b->d_pairs; c.tasks = b->d_tasks; c.ntasks = b->task_off[NQC];
    c.cls_task_off = b->d_task_off; c.cls_qoff = b->d_qoff;
    c.Q = a.Q; c.Dmax = a.Dmax; c.nsh = b->lds;
    c.tau = a.tau; c.tau_mixed = (float)o.mixed_tol; c.split = o.prec == CQ_PREC_MIXED;
    c.tau_64 = n_precisions(o) == 3 ? (float)o.fp64_tol : 0.f;
    c.qlist = b->d_qlist; c.qcount = b->d_qcount;
    if (b->passes) return launch_passes(b, a, c, o, profile, s);
    if (c.ntasks > 0) {
        const int blocks = (c.ntasks * 32 + 255) / 256;
        classify_kernel<<<blocks, 256, 0, s>>>(c, NQC, 0, b->d_tcount, nullptr);
        scan_tasks_kernel<<<NQC, 1024, 0, s>>>(b->d_task_off, b->d_tcount, b->d_toff, b->d_qcount);
        classify_kernel<<<blocks, 256, 0, s>>>(c, NQC, 1, nullptr, b->d_toff);
    }
    CQ_CUDA(cudaGetLastError());
    const int* order = CLASS_ORDER;
    cq_basis* bm = const_cast<cq_basis*>(b);
    // fork: the class kernels are independent (they only add into J'/K'), so
    // they run on side streams that wait for the classification; the main
    // stream joins them before finalisation.  A profiled build stays on one
    // stream so that each class's events time that class alone.
    const bool fork = !profile;
    if (fork) CQ_CUDA(cudaEventRecord(bm->fork_ev, s));
    if (fork)
        for (int k = 0; k < cq_basis::NSIDE; ++k) CQ_CUDA(cudaStreamWaitEvent(bm->side[k], bm->fork_ev, 0));
    int launched = 0;
    for (int oi = 0; oi < NQC; ++oi) {
        const int qc = order[oi];
        int X = 0;
        while ((X + 1) * (X + 2) / 2 <= qc) ++X;
        const int Y = qc - X * (X + 1) / 2;
        a.tasks = b->d_tasks + b->task_off[qc];
        a.ntasks = b->task_off[qc + 1] - b->task_off[qc];
        a.qmax = b->qoff[qc + 1] - b->qoff[qc];
        if (a.ntasks == 0 || a.qmax == 0) continue;
        a.ket_end = b->cls_off[Y + 1];
        a.same_class = (X == Y);
        for (int pp = 0; pp < n_precisions(o); ++pp) {
            set_precision(a, o, pp, b->d_qlist + b->qoff[qc], b->d_qlist + (b->qoff[qc + 1] - 1),
                          b->d_qcount + 3 * qc);
            unsigned long long* base_cnt = a.counters;
            a.counters = base_cnt + 6 * qc + 2 * pp;
            if (profile) {
                for (int e = 0; e < 2; ++e)
                    if (!bm->pev[qc][pp][e]) CQ_CUDA(cudaEventCreate(&bm->pev[qc][pp][e]));
                CQ_CUDA(cudaEventRecord(bm->pev[qc][pp][0], s));
            }
            cudaStream_t ks = fork ? bm->side[launched % cq_basis::NSIDE] : s;
            ++launched;
            launch_jk_class(b, a, qc, pp, ks);
            if (profile) {
                CQ_CUDA(cudaEventRecord(bm->pev[qc][pp][1], s));
                bm->pev_used[qc][pp] = true;
            }
            a.counters = base_cnt;
        }
    }
    if (fork)
        for (int k = 0; k < cq_basis::NSIDE; ++k) {
            CQ_CUDA(cudaEventRecord(bm->join_ev[k], bm->side[k]));
            CQ_CUDA(cudaStreamWaitEvent(s, bm->join_ev[k], 0));
        }
    return CQ_OK;
}

// Cooperative kernel on the screened list, split per the basis's list_split
// and list_chunk.  The FP64 pipe of an SM runs at 1/62 of its FP32 rate, so
// the deep quartets of short FP64 lists pay to be spread over many warps
// (SMs); every task repeats the HRR and the digestion, which bounds the
// useful split.
static void launch_coop_list(const cq_basis* b, const JKArgs& a, int qc, int prec, cudaStream_t s)
{
    JKArgs c = a;
    c.coop_list = 1;
    c.coop_split = b->list_split[prec];
    c.coop_chunk = b->list_chunk[prec];
    c.ntasks = (int)std::min<long long>(a.qmax, INT_MAX);
    if (c.ntasks > 0) launch_coop(c, qc, prec, s);
}

// Whether class qc has kernel variant v at precision prec (0 FP64, 1 FP32,
// 2 double-float).  The cooperative kernel's task mode screens inside the
// kernel against one bound, so the double-float band takes it on the
// screened list only.
bool variant_exists(int qc, int prec, int v)
{
    switch (v) {
    case VARIANT_LANES: return prec != PREC_DF || LANE_DF[qc];
    case VARIANT_COOP: return prec != PREC_DF;
    case VARIANT_SYM: return SYM_LAUNCH[qc] != nullptr && (prec == 1 || SYM_F64[qc]);
    case VARIANT_COOP_LIST: return true;
    default: return false;
    }
}

void launch_jk_class(const cq_basis* b, const JKArgs& a, int qc, int prec, cudaStream_t s)
{
    int v = b->variant[qc][prec];
    // the FP64 list of a three-tier build holds the few quartets of the
    // largest bounds, mostly deep contractions: spread over the GPU, each
    // split into primitive ranges (the per-SM FP64 rate is 1/62 of FP32's)
    if (!variant_exists(qc, prec, v) || a.fp64_tier) v = VARIANT_COOP_LIST;
    if (v == VARIANT_SYM) {
        SYM_LAUNCH[qc](a, prec, s);
    } else if (v == VARIANT_LANES) {
        JK_LAUNCH[qc](a, prec, s);
    } else if (v == VARIANT_COOP_LIST || (b->coop_list && !b->coop_dirty)) {
        // the screened list (large bases always), each quartet split over up
        // to four warps
        launch_coop_list(b, a, qc, prec, s);
    } else if (!b->coop_dirty) {
        JKArgs c = a;
        c.tasks = b->d_coop_tasks + b->coop_off[qc];
        c.ntasks = b->coop_off[qc + 1] - b->coop_off[qc];
        if (c.ntasks > 0) launch_coop(c, qc, prec, s);
    } else {
        // a class switched to the cooperative kernel uses it once its task
        // list has been rebuilt (by the next cq_fock_build); until then, lane groups
        JK_LAUNCH[qc](a, prec, s);
    }
}

}  // namespace cq

using namespace cq;

namespace cq {
long long g_list_capacity = 3000000000LL;

int jk_grid_cap()
{
    static int cap[64] = {0};
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return 1 << 20;
    if (!cap[dev]) {
        int sms = 0;
        if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || sms <= 0) sms = 152;
        cap[dev] = sms * 16;
    }
    return cap[dev];
}
}

extern "C" int cq_set_list_capacity(long long entries)
{
    if (entries < 1024) {
        set_error("cq_set_list_capacity: capacity below 1024 entries");
        return CQ_ERR_INVALID_ARG;
    }
    g_list_capacity = entries;
    return CQ_OK;
}

extern "C" long long cq_get_list_capacity(void) { return g_list_capacity; }

extern "C" int cq_fock_set_variant(cq_basis* b, int qc, int prec, int variant)
{
    if (!b || qc < 0 || qc >= NQC || prec < 0 || prec > 2 || variant < 0 || variant >= NVARIANT) {
        set_error("cq_fock_set_variant: bad argument");
        return CQ_ERR_INVALID_ARG;
    }
    if (!variant_exists(qc, prec, variant)) {
        set_error("cq_fock_set_variant: this class and precision have no such kernel variant");
        return CQ_ERR_UNSUPPORTED;
    }
    if (b->variant[qc][prec] != variant) b->coop_dirty = true;
    b->variant[qc][prec] = variant;
    return CQ_OK;
}

extern "C" int cq_fock_set_list_split(cq_basis* b, int prec, int split, int chunk)
{
    if (!b || prec < 0 || prec > 2 || split < 1 || split > 64 || chunk < 1) {
        set_error("cq_fock_set_list_split: bad argument");
        return CQ_ERR_INVALID_ARG;
    }
    b->list_split[prec] = split;
    b->list_chunk[prec] = chunk;
    return CQ_OK;
}

extern "C" int cq_fock_get_variant(const cq_basis* b, int qc, int prec, int* variant)
{
    if (!b || !variant || qc < 0 || qc >= NQC || prec < 0 || prec > 2) {
        set_error("cq_fock_get_variant: bad argument");
        return CQ_ERR_INVALID_ARG;
    }
    *variant = b->variant[qc][prec];
    return CQ_OK;
}

// Adds the six totals (quartets and primitive quartets in FP64, FP32 and
// double-float) of a build into a running accumulator.
namespace cq {
__global__ void counter_accumulate_kernel(const unsigned long long* __restrict__ c, unsigned long long* __restrict__ acc)
{
    if (threadIdx.x < 6) acc[threadIdx.x] += c[threadIdx.x];
}
}  // namespace cq

int cq::fock_build_modes(cq_basis* b, int kind, const void* P, double* J, void* K, const cq_fock_opts* opts,
                     cq_fock_stats* stats, cudaStream_t s, const int* mol_mode, unsigned long long* acc)
{
    if (!b || !P) { set_error("cq_fock_build: NULL basis or density"); return CQ_ERR_INVALID_ARG; }
    if (kind < CQ_DENS_REAL_SYM || kind > CQ_DENS_REAL_GENERAL) {
        set_error("cq_fock_build: unknown density kind");
        return CQ_ERR_INVALID_ARG;
    }
    cq_fock_opts o{1e-14, 1e-5, CQ_PREC_FP64, 1, 1, 0.0};
    if (opts) o = *opts;
    if ((o.want_J && !J) || (o.want_K && !K)) {
        set_error("cq_fock_build: requested output pointer is NULL");
        return CQ_ERR_INVALID_ARG;
    }
    if (o.prec != CQ_PREC_FP64 && o.prec != CQ_PREC_MIXED) {
        set_error("cq_fock_build: unknown precision mode");
        return CQ_ERR_INVALID_ARG;
    }
    if (!(o.schwarz_tol >= 0.0) || !(o.mixed_tol >= 0.0) || !(o.fp64_tol >= 0.0)) {
        set_error("cq_fock_build: negative threshold");
        return CQ_ERR_INVALID_ARG;
    }
    const int nk = nk_of(kind);
    int rc = ensure_scratch(b, nk);
    if (rc) return rc;
    if ((rc = ensure_coop_tasks(b))) return rc;
    const int n = b->ld;
    const size_t nn = b->mstride;
    const int nb = (int)((nn + 255) / 256);
    if (stats) CQ_CUDA(cudaEventRecord(b->ev0, s));
    density_prep_kernel<<<nb, 256, 0, s>>>(kind, b->nmol, n, b->d_mol_n, b->d_mol_bfo, (const double*)P, b->d_scale,
                                           b->d_Dp);
    const size_t nsl = (size_t)b->nmol * b->lds * b->lds;
    dmax_kernel<<<(unsigned)((nsl + 127) / 128), 128, 0, s>>>(b->nmol, n, b->lds, b->d_mol_nsh, b->d_mol_sho,
                                                              b->d_mol_bfo, b->d_bfo, nk, b->d_Dp, mol_mode,
                                                              b->d_Dmax);
    CQ_CUDA(cudaMemsetAsync(b->d_Jp, 0, 2 * nn * sizeof(acc_t), s));
    CQ_CUDA(cudaMemsetAsync(b->d_Kp, 0, 2 * nn * nk * sizeof(acc_t), s));
    CQ_CUDA(cudaMemsetAsync(b->d_cnt, 0, CNT_WORDS * sizeof(unsigned long long), s));
    if (b->profile) {
        memset(b->pev_used, 0, sizeof b->pev_used);
        memset(b->pev_npass, 0, sizeof b->pev_npass);
    }
    JKArgs a;
    memset(&a, 0, sizeof a);
    a.pairs = b->d_pairs; a.prims = b->d_prims; a.primsf = b->d_primsf;
    a.Q = b->d_Qf; a.Dmax = b->d_Dmax; a.nsh = b->lds;
    a.mstride = (long long)nn;
    a.tau = (float)o.schwarz_tol;
    a.tau_mixed = (float)o.mixed_tol;
    a.D = b->d_Dp; a.nk = nk; a.nbf = n;
    a.want_j = o.want_J; a.want_k = o.want_K;
    a.J = b->d_Jp; a.K = b->d_Kp;
    a.boys_d = b->d_boys; a.boys_f = b->d_boysf;
    a.counters = b->d_cnt + 6;
    a.primsx = b->d_primsx;
    a.mol_mode = mol_mode;
    a.lds2 = (long long)b->lds * b->lds;
    rc = classify_and_launch(b, a, o, b->profile != 0, s, mol_mode);
    if (rc) return rc;
    CQ_CUDA(cudaGetLastError());
    counter_total_kernel<<<1, 32, 0, s>>>(b->d_cnt);
    if (acc) counter_accumulate_kernel<<<1, 32, 0, s>>>(b->d_cnt, acc);
    finalize_kernel<<<nb, 256, 0, s>>>(kind, b->nmol, n, b->d_mol_n, b->d_mol_bfo, b->d_scale, b->d_Jp, b->d_Kp, J,
                                       (double*)K, o.want_J, o.want_K);
    CQ_CUDA(cudaGetLastError());
    if (stats) {
        CQ_CUDA(cudaEventRecord(b->ev1, s));
        unsigned long long c[6];
        CQ_CUDA(cudaMemcpyAsync(c, b->d_cnt, sizeof c, cudaMemcpyDeviceToHost, s));
        CQ_CUDA(cudaStreamSynchronize(s));
        float ms = 0.f;
        CQ_CUDA(cudaEventElapsedTime(&ms, b->ev0, b->ev1));
        stats->quartets_fp64 = c[0];
        stats->prim_fp64 = c[1];
        stats->quartets_fp32 = c[2];
        stats->prim_fp32 = c[3];
        stats->quartets_df = c[4];
        stats->prim_df = c[5];
        stats->ms = ms;
    }
    return CQ_OK;
}

extern "C" int cq_fock_build(cq_basis* b, int kind, const void* P, double* J, void* K,
                             const cq_fock_opts* opts, cq_fock_stats* stats, void* stream)
{
    return fock_build_modes(b, kind, P, J, K, opts, stats, (cudaStream_t)stream, nullptr, nullptr);
}

extern "C" int cq_fock_profile(cq_basis* b, int enable)
{
    if (!b) { set_error("cq_fock_profile: NULL basis"); return CQ_ERR_INVALID_ARG; }
    b->profile = enable ? 1 : 0;
    return CQ_OK;
}

extern "C" int cq_fock_class_stats(cq_basis* b, int qc, int fp32, double* ms, unsigned long long* quartets,
                                   unsigned long long* prims)
{
    if (!b || qc < 0 || qc >= NQC || fp32 < 0 || fp32 > 2) {
        set_error("cq_fock_class_stats: bad argument");
        return CQ_ERR_INVALID_ARG;
    }
    CQ_CUDA(cudaDeviceSynchronize());
    unsigned long long c[2];
    CQ_CUDA(cudaMemcpy(c, b->d_cnt + 6 + 6 * qc + 2 * fp32, sizeof c, cudaMemcpyDeviceToHost));
    if (quartets) *quartets = c[0];
    if (prims) *prims = c[1];
    if (ms) {
        float t = 0.f;
        double tot = 0.0;
        if (b->profile && b->pev_used[qc][fp32]) {
            if (b->passes) {
                for (int k = 0; k < b->pev_npass[qc][fp32]; ++k) {
                    CQ_CUDA(cudaEventElapsedTime(&t, b->pev_pass[qc][fp32][2 * k], b->pev_pass[qc][fp32][2 * k + 1]));
                    tot += t;
                }
            } else {
                CQ_CUDA(cudaEventElapsedTime(&t, b->pev[qc][fp32][0], b->pev[qc][fp32][1]));
                tot = t;
            }
        }
        *ms = tot;
    }
    return CQ_OK;
}

// Autotuner: time every kernel variant of every class on the caller's
// density (profiled builds run on one stream, so each class kernel is timed
// alone), keep the fastest per class and precision, then refine on whole
// (concurrent) builds.  The axis-permutation kernel exists for the classes
// listed in SYM_LAUNCH (FP64 and double-float where SYM_F64).
extern "C" int cq_autotune(cq_basis* b, int kind, const void* P, const cq_fock_opts* opts, int* table,
                           double* ms_out, void* stream)
{
    if (!b || !P) { set_error("cq_autotune: NULL argument"); return CQ_ERR_INVALID_ARG; }
    cq_fock_opts o{1e-14, 1e-3, CQ_PREC_MIXED, 1, 1, 0.0};
    if (opts) o = *opts;
    const size_t nn = b->mstride;
    const int nk = nk_of(kind);
    // precisions the build uses: FP64 alone, FP64 + FP32, or all three tiers
    // (whose FP64 tier always takes the cooperative kernel on the list)
    const int np = o.prec == CQ_PREC_FP64 ? 1 : n_precisions(o);
    const int p0 = np == 3 ? 1 : 0;
    double *J = nullptr, *K = nullptr;
    int rc;
    if ((rc = dalloc(&J, nn))) return rc;
    if ((rc = dalloc(&K, nn * (nk == 1 ? 1 : nk == 2 ? 2 : 8)))) { cudaFree(J); return rc; }
    const int old_profile = b->profile;
    b->profile = 1;
    double t[NQC][3][NVARIANT];
    for (int q = 0; q < NQC; ++q)
        for (int p = 0; p < 3; ++p)
            for (int v = 0; v < NVARIANT; ++v) t[q][p][v] = 1e300;
    auto allowed = [&](int q, int p, int v) { return variant_exists(q, p, v); };
    // one round of builds per variant: every class that has the variant
    // runs it, the others their default
    for (int v = 0; v < NVARIANT && rc == CQ_OK; ++v) {
        for (int q = 0; q < NQC; ++q)
            for (int p = p0; p < np; ++p) {
                const int want = allowed(q, p, v) ? v : DEFAULT_VARIANT[q][p];
                if (b->variant[q][p] != want) b->coop_dirty = true;
                b->variant[q][p] = want;
            }
        // a warm-up build, then the faster of two profiled builds per class
        for (int rep = 0; rep < 3 && rc == CQ_OK; ++rep) {
            cq_fock_stats st;
            if ((rc = cq_fock_build(b, kind, P, J, K, &o, &st, stream))) break;
            if (rep == 0) continue;
            for (int q = 0; q < NQC && rc == CQ_OK; ++q)
                for (int p = p0; p < np; ++p) {
                    if (!allowed(q, p, v)) continue;
                    double ms = 0.0;
                    unsigned long long nq = 0, npr = 0;
                    if ((rc = cq_fock_class_stats(b, q, p, &ms, &nq, &npr))) break;
                    t[q][p][v] = std::min(t[q][p][v], ms);
                }
        }
    }
    b->profile = old_profile;
    if (rc) {
        cudaFree(J);
        cudaFree(K);
        return rc;
    }
    int best[NQC][3], second[NQC][3];
    for (int q = 0; q < NQC; ++q)
        for (int p = p0; p < np; ++p) {
            best[q][p] = DEFAULT_VARIANT[q][p];
            second[q][p] = -1;
            for (int v = 0; v < NVARIANT; ++v)
                if (t[q][p][v] < t[q][p][best[q][p]]) best[q][p] = v;
            for (int v = 0; v < NVARIANT; ++v)
                if (v != best[q][p] && t[q][p][v] < 1e299 &&
                    (second[q][p] < 0 || t[q][p][v] < t[q][p][second[q][p]]))
                    second[q][p] = v;
            if (b->variant[q][p] != best[q][p]) b->coop_dirty = true;
            b->variant[q][p] = best[q][p];
        }
    // Refinement on the whole build: the class kernels of a build run
    // concurrently, so a variant that wins alone can lose beside the others.
    // For the costliest classes, try the runner-up variant and keep it only
    // if the median time of three complete builds improves by more than 1 %.
    auto build_ms = [&](double* out) -> int {
        double tt[3];
        for (int r = 0; r < 3; ++r) {
            cq_fock_stats st;
            const int e = cq_fock_build(b, kind, P, J, K, &o, &st, stream);
            if (e) return e;
            tt[r] = st.ms;
        }
        std::sort(tt, tt + 3);
        *out = tt[1];
        return CQ_OK;
    };
    std::vector<std::pair<double, int>> cand;
    for (int q = 0; q < NQC; ++q)
        for (int p = p0; p < np; ++p)
            if (second[q][p] >= 0) cand.push_back({t[q][p][best[q][p]], 3 * q + p});
    std::sort(cand.begin(), cand.end(), [](const std::pair<double, int>& x, const std::pair<double, int>& y) {
        return x.first > y.first;
    });
    if (cand.size() > 8) cand.resize(8);
    double cur = 0.0;
    rc = build_ms(&cur);
    for (size_t i = 0; i < cand.size() && rc == CQ_OK; ++i) {
        const int q = cand[i].second / 3, p = cand[i].second % 3;
        const int keep = b->variant[q][p];
        b->variant[q][p] = second[q][p];
        b->coop_dirty = true;
        double tb = 0.0;
        if ((rc = build_ms(&tb))) break;
        if (tb < 0.99 * cur) {
            cur = tb;
        } else {
            b->variant[q][p] = keep;
            b->coop_dirty = true;
        }
    }
    cudaFree(J);
    cudaFree(K);
    if (rc) return rc;
    for (int q = 0; q < NQC; ++q)
        for (int p = 0; p < 3; ++p) {
            const double ms = (p >= p0 && p < np) ? t[q][p][best[q][p]] : 1e300;
            if (table) table[3 * q + p] = b->variant[q][p];
            if (ms_out) ms_out[3 * q + p] = ms < 1e299 ? ms : 0.0;
        }
    return ensure_coop_tasks(b);
}
