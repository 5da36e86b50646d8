// Batched RHF SCF over the molecules of a batched basis (cq_basis_create_batch):
// every iteration runs one Fock build for all molecules and the dense steps
// of every molecule as strided-batched GEMMs and one batched symmetric
// eigensolver call, on ld x ld slots (ld = largest molecule).  Padding rows and
// columns, and overlap directions dropped by canonical orthogonalisation,
// are pushed to the top of each Fock spectrum by a large diagonal shift, so
// that they are never occupied.  Each molecule has its own DIIS subspace and
// convergence flag; a converged molecule keeps its density.
#include <cublas_v2.h>
#include <cusolverDn.h>

#include <cmath>
#include <cstring>
#include <vector>

#include "cq_internal.h"

namespace cq {

#define CQ_BLAS_B(call)                                                   \
    do {                                                                  \
        cublasStatus_t _s = (call);                                       \
        if (_s != CUBLAS_STATUS_SUCCESS) {                                \
            set_error(std::string("cuBLAS failure in ") + #call);         \
            return CQ_ERR_CUDA;                                           \
        }                                                                 \
    } while (0)
#define CQ_SOLVER_B(call)                                                 \
    do {                                                                  \
        cusolverStatus_t _s = (call);                                     \
        if (_s != CUSOLVER_STATUS_SUCCESS) {                              \
            set_error(std::string("cuSOLVER failure in ") + #call);       \
            return CQ_ERR_CUDA;                                           \
        }                                                                 \
    } while (0)

constexpr int BDIIS = 8;
constexpr double BATCH_SHIFT = 1.0e6;

// C_m = alpha op(A_m) op(B_m) + beta C_m for every slot (row-major ld x ld)
static cublasStatus_t gemm_batch(cublasHandle_t h, bool ta, bool tb, int ld, int nmol, double alpha,
                                 const double* A, const double* B, double beta, double* C)
{
    const long long st = (long long)ld * ld;
    return cublasDgemmStridedBatched(h, tb ? CUBLAS_OP_T : CUBLAS_OP_N, ta ? CUBLAS_OP_T : CUBLAS_OP_N, ld, ld, ld,
                                     &alpha, B, ld, st, A, ld, st, &beta, C, ld, st, nmol);
}

__global__ void slot_axpby_kernel(size_t n, double a, const double* __restrict__ x, double b,
                                  const double* __restrict__ y, double* __restrict__ z)
{
    const size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) z[i] = a * x[i] + b * y[i];
}

// S with zero padding diagonal (so padding eigenvalues are 0 and dropped)
__global__ void pad_overlap_kernel(int nmol, int ld, const int* __restrict__ mol_n, const double* __restrict__ S,
                                   double* __restrict__ out)
{
    const size_t slot = (size_t)ld * ld;
    const size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= slot * nmol) return;
    out[i] = S[i];
}

// X_m columns: eigenvector k / sqrt(w_k) when w_k >= 1e-8, else zero; shift
// 0 for kept columns, BATCH_SHIFT for the rest.  Rows of V hold eigenvectors.
__global__ void batch_ortho_kernel(int nmol, int ld, const double* __restrict__ V, const double* __restrict__ w,
                                   double* __restrict__ X, double* __restrict__ shift)
{
    const size_t slot = (size_t)ld * ld;
    const size_t t = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= slot * nmol) return;
    const int m = (int)(t / slot), i = (int)((t / ld) % ld), j = (int)(t % ld);
    const double wj = w[(size_t)m * ld + j];
    const bool keep = wj >= 1e-8;
    X[t] = keep ? V[(size_t)m * slot + (size_t)j * ld + i] * rsqrt(wj) : 0.0;
    if (i == 0) shift[(size_t)m * ld + j] = keep ? 0.0 : BATCH_SHIFT;
}

__global__ void add_diag_kernel(int nmol, int ld, const double* __restrict__ shift, double* __restrict__ A)
{
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= nmol * ld) return;
    const int m = t / ld, j = t % ld;
    A[(size_t)m * ld * ld + (size_t)j * ld + j] += shift[t];
}

// G = 2J - K, F = H + G
__global__ void batch_fock_kernel(size_t n, const double* __restrict__ H, const double* __restrict__ J,
                                  const double* __restrict__ K, double* __restrict__ F)
{
    const size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) F[i] = H[i] + 2.0 * J[i] - K[i];
}

// Iteration state kept on the device, so that an iteration is the same
// sequence of launches every time (and can be captured once as a graph):
// the iteration number, the DIIS ring (insertions so far, newest slot,
// subspace size and the slots from oldest to newest), the number of
// molecules open at the start of the iteration and the number still open
// after its convergence test.
struct BatchState {
    int it;
    int kd;
    int slot, nvec;
    int order[BDIIS];
    int nact;
    unsigned int nopen;
};

// per-molecule mode bits read by the Fock build (ClassifyArgs::mol_mode)
constexpr int MODE_FP32 = 1;
constexpr int MODE_SKIP = 2;

// Start of an iteration: the open molecules, in order, become the compact
// slots 0..nact-1 of the dense steps (one block; slots nact..kb-1 repeat a
// valid molecule and are never written back).
__global__ void batch_begin_kernel(int nmol, int kb, const int* __restrict__ conv, const int* __restrict__ nocc,
                                   BatchState* st, int* __restrict__ act, int* __restrict__ nocc_c)
{
    __shared__ int part[1024];
    const int per = (nmol + blockDim.x - 1) / blockDim.x;
    const int m0 = threadIdx.x * per, m1 = min(nmol, m0 + per);
    int c = 0;
    for (int m = m0; m < m1; ++m) c += conv[m] ? 0 : 1;
    part[threadIdx.x] = c;
    __syncthreads();
    if (threadIdx.x == 0) {
        int a = 0;
        for (int i = 0; i < (int)blockDim.x; ++i) {
            const int x = part[i];
            part[i] = a;
            a += x;
        }
        st->it += 1;
        st->nopen = 0u;
        st->nact = min(a, kb);
    }
    __syncthreads();
    int k = part[threadIdx.x];
    for (int m = m0; m < m1; ++m)
        if (!conv[m]) {
            if (k < kb) { act[k] = m; nocc_c[k] = nocc[m]; }
            ++k;
        }
    __syncthreads();
    const int na = st->nact;
    const int dummy = na > 0 ? act[0] : 0;
    for (int i = na + threadIdx.x; i < kb; i += blockDim.x) {
        act[i] = dummy;
        nocc_c[i] = nocc[dummy];
    }
}

// dst slot k <- src slot act[k] (slot = n elements), for up to three arrays
struct Gather3 {
    const double* src[3];
    double* dst[3];
};
__global__ void batch_gather_kernel(int kb, size_t n, const int* __restrict__ act, Gather3 g)
{
    const size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= (size_t)kb * n) return;
    const size_t k = i / n, r = i - k * n;
    const size_t from = (size_t)act[k] * n + r;
    for (int q = 0; q < 3; ++q)
        if (g.src[q]) g.dst[q][i] = g.src[q][from];
}

// per open molecule (compact slot k, one block each): E = sum (H + F) D + Enuc
// over its full slot; rms of its orthogonal-basis error (compact)
__global__ void batch_energy_rms_kernel(int ld, const int* __restrict__ act, const BatchState* st,
                                        const double* __restrict__ H, const double* __restrict__ F,
                                        const double* __restrict__ D, const double* __restrict__ Epc,
                                        const double* __restrict__ enuc, const int* __restrict__ mol_n,
                                        double* __restrict__ E, double* __restrict__ rms)
{
    __shared__ double r0[256], r1[256];
    const int k = blockIdx.x;
    if (k >= st->nact) return;
    const int m = act[k];
    const size_t slot = (size_t)ld * ld, o = (size_t)m * slot, oc = (size_t)k * slot;
    double e = 0.0, q = 0.0;
    for (size_t i = threadIdx.x; i < slot; i += blockDim.x) {
        e += (H[o + i] + F[o + i]) * D[o + i];
        q += Epc[oc + i] * Epc[oc + i];
    }
    r0[threadIdx.x] = e;
    r1[threadIdx.x] = q;
    __syncthreads();
    for (int s = blockDim.x / 2; s > 0; s >>= 1) {
        if ((int)threadIdx.x < s) { r0[threadIdx.x] += r0[threadIdx.x + s]; r1[threadIdx.x] += r1[threadIdx.x + s]; }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        E[m] = r0[0] + enuc[m];
        const double nm = (double)mol_n[m];
        rms[m] = sqrt(r1[0] / (nm * nm));
    }
}

__global__ void batch_antisym_kernel(int nmol, int ld, const double* __restrict__ T, double* __restrict__ E)
{
    const size_t slot = (size_t)ld * ld;
    const size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= slot * nmol) return;
    const size_t m = i / slot;
    const int r = (int)((i / ld) % ld), c = (int)(i % ld);
    E[i] = T[i] - T[m * slot + (size_t)c * ld + r];
}

// Convergence test per molecule (one thread each).  A molecule is tested
// from the second iteration on, and only on an energy from an all-FP64
// build; a molecule built in mixed precision moves to FP64 builds once its
// orthogonal-basis error falls below switch_tol.  A converged molecule is
// skipped by later builds and dense steps; the open count goes to the state
// and to the host-visible history (one entry per iteration).  A molecule
// still open at iteration restart_iter (> 0) restarts from the fallback
// density: the flag is read by the DIIS solve (fresh subspace) and the
// density update.
__global__ void batch_conv_kernel(int nmol, const double* __restrict__ E, const double* __restrict__ Eold,
                                  const double* __restrict__ rms, double e_tol, double d_tol, double switch_tol,
                                  int restart_iter, int mode0, int* __restrict__ conv, int* __restrict__ iters,
                                  int* __restrict__ mode, int* __restrict__ restart, BatchState* st)
{
    const int m = blockIdx.x * blockDim.x + threadIdx.x;
    if (m >= nmol || conv[m]) return;
    const int it = st->it;
    restart[m] = 0;
    const int md = mode[m];
    if (it > 1 && !(md & MODE_FP32) && fabs(E[m] - Eold[m]) < e_tol && rms[m] < d_tol) {
        conv[m] = 1;
        iters[m] = it;
        mode[m] = md | MODE_SKIP;
        return;
    }
    if (it == restart_iter) {
        restart[m] = 1;
        mode[m] = mode0;
    } else if ((md & MODE_FP32) && rms[m] < switch_tol) {
        mode[m] = md & ~MODE_FP32;
    }
    atomicAdd(&st->nopen, 1u);
}

__global__ void batch_publish_kernel(const BatchState* st, unsigned int* open_hist, int hist_len)
{
    if (threadIdx.x == 0 && st->it < hist_len) open_hist[st->it] = st->nopen;
}

// next DIIS slot: the ring holds the last ds error vectors
__global__ void batch_diis_index_kernel(BatchState* st, int ds)
{
    if (threadIdx.x != 0) return;
    const int kd = st->kd;
    const int slot = kd % ds;
    const int nvec = kd + 1 < ds ? kd + 1 : ds;
    st->slot = slot;
    st->nvec = nvec;
    for (int k = 0; k < nvec; ++k) st->order[k] = (slot + 1 - nvec + k + ds) % ds;
    st->kd = kd + 1;
}

struct SlotPtrs {
    double* p[BDIIS];
};

// F and E' of the open molecules (compact slots) into the newest ring slot
// (ring kept per molecule)
__global__ void batch_store_slot_kernel(int kb, int ld, SlotPtrs Fs, SlotPtrs Es, const BatchState* st,
                                        const int* __restrict__ act, const double* __restrict__ Fc,
                                        const double* __restrict__ Epc)
{
    const size_t slot = (size_t)ld * ld;
    const size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= slot * kb) return;
    const size_t k = i / slot, r = i - k * slot;
    if ((int)k >= st->nact) return;
    const size_t to = (size_t)act[k] * slot + r;
    const int q = st->slot;
    Fs.p[q][to] = Fc[i];
    Es.p[q][to] = Epc[i];
}

// B[m][slot][j] = e_slot . e_j for the ring slots j (grid: compact slots x BDIIS)
__global__ void batch_dot_kernel(int ld, SlotPtrs Es, const BatchState* st, const int* __restrict__ act,
                                 double* __restrict__ Bm)
{
    __shared__ double red[256];
    const int k = blockIdx.x, p = blockIdx.y;
    if (k >= st->nact || p >= st->nvec) return;
    const int m = act[k];
    const int pi = st->slot, pj = st->order[p];
    const size_t slot = (size_t)ld * ld, o = (size_t)m * slot;
    const double* a = Es.p[pi] + o;
    const double* b = Es.p[pj] + o;
    double s = 0.0;
    for (size_t i = threadIdx.x; i < slot; i += blockDim.x) s += a[i] * b[i];
    red[threadIdx.x] = s;
    __syncthreads();
    for (int q = blockDim.x / 2; q > 0; q >>= 1) {
        if ((int)threadIdx.x < q) red[threadIdx.x] += red[threadIdx.x + q];
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        Bm[(size_t)m * BDIIS * BDIIS + pi * BDIIS + pj] = red[0];
        Bm[(size_t)m * BDIIS * BDIIS + pj * BDIIS + pi] = red[0];
    }
}

// Per open molecule: the DIIS coefficients over its newest nv ring slots
// (nv = its insertions since its last restart, at most the ring's size) from
// the bordered system [B -1; -1 0][c; l] = [0; -1], by Gaussian elimination
// with partial pivoting; one vector gives c = 1.  nv is kept in kdm.
__global__ void batch_diis_solve_kernel(int nmol, const BatchState* st, const int* __restrict__ conv,
                                        const int* __restrict__ restart, int* __restrict__ kdm,
                                        const double* __restrict__ Bm, double* __restrict__ coef)
{
    const int mol = blockIdx.x * blockDim.x + threadIdx.x;
    if (mol >= nmol || conv[mol]) return;
    double* c = coef + (size_t)mol * BDIIS;
    if (restart[mol]) {   // this iteration's density is replaced: start a fresh subspace
        kdm[mol] = 0;
        c[0] = 1.0;
        return;
    }
    const int m = min(kdm[mol] + 1, st->nvec), N = m + 1;
    kdm[mol] = m;
    const int off = st->nvec - m;
    if (m < 2) {
        c[0] = 1.0;
        return;
    }
    double A[BDIIS + 1][BDIIS + 2];
    const double* B = Bm + (size_t)mol * BDIIS * BDIIS;
    for (int i = 0; i < m; ++i) {
        for (int j = 0; j < m; ++j) A[i][j] = B[st->order[off + i] * BDIIS + st->order[off + j]];
        A[i][m] = -1.0;
        A[i][m + 1] = 0.0;
    }
    for (int j = 0; j < m; ++j) A[m][j] = -1.0;
    A[m][m] = 0.0;
    A[m][m + 1] = -1.0;
    for (int col = 0; col < N; ++col) {
        int piv = col;
        for (int r = col + 1; r < N; ++r)
            if (fabs(A[r][col]) > fabs(A[piv][col])) piv = r;
        if (piv != col)
            for (int k = 0; k <= N; ++k) { const double t = A[col][k]; A[col][k] = A[piv][k]; A[piv][k] = t; }
        if (fabs(A[col][col]) < 1e-300) {
            for (int i = 0; i < m; ++i) c[i] = (i == m - 1) ? 1.0 : 0.0;
            return;
        }
        for (int r = col + 1; r < N; ++r) {
            const double f = A[r][col] / A[col][col];
            for (int k = col; k <= N; ++k) A[r][k] -= f * A[col][k];
        }
    }
    double x[BDIIS + 1];
    for (int r = N - 1; r >= 0; --r) {
        double s = A[r][N];
        for (int k = r + 1; k < N; ++k) s -= A[r][k] * x[k];
        x[r] = s / A[r][r];
    }
    for (int i = 0; i < m; ++i) c[i] = x[i];
}

// extrapolated Fock matrices of the compact slots (a molecule that has just
// converged, restarts or fills a padding slot takes its current F)
__global__ void batch_diis_combine_kernel(int kb, int ld, SlotPtrs F, const BatchState* st,
                                          const int* __restrict__ act, const int* __restrict__ conv,
                                          const int* __restrict__ kdm, const double* __restrict__ coef,
                                          const double* __restrict__ Fc, double* __restrict__ out)
{
    const size_t slot = (size_t)ld * ld;
    const size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= slot * kb) return;
    const size_t k = i / slot, r = i - k * slot;
    const int m = act[k];
    const int nv = kdm[m];
    if ((int)k >= st->nact || conv[m] || nv < 1) {
        out[i] = Fc[i];
        return;
    }
    const int off = st->nvec - nv;
    const size_t from = (size_t)m * slot + r;
    double s = 0.0;
    for (int q = 0; q < nv; ++q) s += coef[(size_t)m * BDIIS + q] * F.p[st->order[off + q]][from];
    out[i] = s;
}

__global__ void fill_int_kernel(int n, int v, int* __restrict__ x)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) x[i] = v;
}

// keep the first nocc[k] columns of C (the occupied orbitals)
__global__ void occ_mask_kernel(int nmol, int ld, const int* __restrict__ nocc, double* __restrict__ C)
{
    const size_t slot = (size_t)ld * ld;
    const size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= slot * nmol) return;
    const int m = (int)(i / slot), c = (int)(i % ld);
    if (c >= nocc[m]) C[i] = 0.0;
}

// dst slot act[k] <- the new density of compact slot k, for the molecules
// still open (the fallback density for a molecule restarting this
// iteration); conv and restart may be NULL (every slot taken)
__global__ void batch_scatter_kernel(int kb, int ld, const int* __restrict__ act, const BatchState* st,
                                     const int* __restrict__ conv, const int* __restrict__ restart,
                                     const double* __restrict__ Dnc, const double* __restrict__ Dfall,
                                     double* __restrict__ dst)
{
    const size_t slot = (size_t)ld * ld;
    const size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= slot * kb) return;
    const size_t k = i / slot, r = i - k * slot;
    if ((int)k >= st->nact) return;
    const int m = act[k];
    if (conv && conv[m]) return;
    const size_t to = (size_t)m * slot + r;
    dst[to] = (restart && restart[m]) ? Dfall[to] : Dnc[i];
}

static int nb256(size_t n) { return (int)((n + 255) / 256); }

}  // namespace cq

using namespace cq;

extern "C" int cq_scf_batch(cq_basis* b, const int* nocc, const cq_scf_opts* opts, const double* D_in, double* D_out,
                            double* E_out, int* iters_out, cq_scf_stats* stats, void* stream)
{
    if (!b || !nocc || !D_out) { set_error("cq_scf_batch: NULL argument"); return CQ_ERR_INVALID_ARG; }
    cq_scf_opts o{1e-10, 1e-8, 128, 8, CQ_PREC_FP64, 1e-5, 1e-14, 0, 8, 1e-5, 1, 0, 0.0};
    if (opts) o = *opts;
    // the core-guess fallback applies to a supplied starting density only
    const int restart_iter = (D_in && o.guess_fallback > 1) ? o.guess_fallback : 0;
    if (o.diis_size < 1 || o.diis_size > BDIIS || o.max_iter <= 0) {
        set_error("cq_scf_batch: diis_size must be 1..8 and max_iter > 0");
        return CQ_ERR_INVALID_ARG;
    }
    if (o.prec != CQ_PREC_FP64 && o.prec != CQ_PREC_MIXED) {
        set_error("cq_scf_batch: unknown precision mode");
        return CQ_ERR_INVALID_ARG;
    }
    const int nmol = b->nmol, ld = b->ld;
    for (int m = 0; m < nmol; ++m)
        if (nocc[m] <= 0 || nocc[m] > b->mol_n[m]) {
            set_error("cq_scf_batch: nocc out of range for molecule " + std::to_string(m));
            return CQ_ERR_INVALID_ARG;
        }
    // The iterations run on a private non-blocking stream (graphs are not
    // captured on the legacy default stream), ordered after the caller's
    // stream on entry; the call returns after that stream has drained.
    const cudaStream_t caller = (cudaStream_t)stream;
    if (!b->batch_stream) {
        CQ_CUDA(cudaStreamCreateWithFlags(&b->batch_stream, cudaStreamNonBlocking));
        CQ_CUDA(cudaEventCreateWithFlags(&b->batch_ev, cudaEventDisableTiming));
    }
    const cudaStream_t s = b->batch_stream;
    CQ_CUDA(cudaEventRecord(b->batch_ev, caller));
    CQ_CUDA(cudaStreamWaitEvent(s, b->batch_ev, 0));
    if (!b->blas) {
        cublasHandle_t h;
        CQ_BLAS_B(cublasCreate(&h));
        b->blas = h;
    }
    if (!b->solver) {
        cusolverDnHandle_t h;
        CQ_SOLVER_B(cusolverDnCreate(&h));
        b->solver = h;
    }
    cublasHandle_t blas = (cublasHandle_t)b->blas;
    cusolverDnHandle_t sol = (cusolverDnHandle_t)b->solver;
    CQ_BLAS_B(cublasSetStream(blas, s));
    CQ_SOLVER_B(cusolverDnSetStream(sol, s));
    const size_t ms = (size_t)b->mstride;
    const size_t slot = (size_t)ld * ld;
    const int ds = o.diis_size;
    std::vector<void*> bufs;
    int rc = CQ_OK;
    auto get = [&](auto** p, size_t n) -> int {
        int r = dalloc(p, n);
        if (!r) bufs.push_back((void*)*p);
        return r;
    };
    // per molecule (slot = molecule): one-electron data, X, shift, density,
    // J/K/F, DIIS ring, scalars; compact (slot k = k-th open molecule): the
    // dense steps' operands
    double *S, *T, *V, *H, *X, *shift, *D, *J, *K, *F, *Bm, *coef, *E, *Eold, *rms, *enuc, *Dcore = nullptr;
    double *Fc, *Dc, *Sc, *Xc, *shc, *T1, *T2, *Epc, *Fdc, *Dnc, *w;
    int *conv, *iters, *d_nocc, *info, *mode, *kdm, *restart, *act, *nocc_c;
    unsigned long long* acc;
    BatchState* bst;
    SlotPtrs Fs{}, Es{};
    cusolverDnParams_t prm = nullptr;
    void* dwork = nullptr;
    std::vector<char> hwork;
    unsigned int* open_hist = nullptr;   // mapped host memory, one entry per iteration
    unsigned int* open_dev = nullptr;
    struct Graphs {
        int kb;
        cudaGraphExec_t full, a, b;
    };
    std::vector<Graphs> graphs;
    cudaEvent_t iev[2] = {nullptr, nullptr}, e0 = nullptr, e1 = nullptr;
    const int hist_len = o.max_iter + 2;
    auto fail = [&](int r) {
        if (r != CQ_OK) cudaStreamSynchronize(s);
        for (Graphs& g : graphs)
            for (cudaGraphExec_t x : {g.full, g.a, g.b})
                if (x) cudaGraphExecDestroy(x);
        for (cudaEvent_t e : {iev[0], iev[1], e0, e1})
            if (e) cudaEventDestroy(e);
        if (prm) cusolverDnDestroyParams(prm);
        if (dwork) cudaFree(dwork);
        if (open_hist) cudaFreeHost(open_hist);
        for (void* p : bufs) cudaFree(p);
        return r;
    };
#define GETB(p, n)                          \
    if ((rc = get(&(p), (n)))) return fail(rc);
    GETB(S, ms) GETB(T, ms) GETB(V, ms) GETB(H, ms) GETB(X, ms) GETB(shift, (size_t)nmol * ld) GETB(D, ms)
    GETB(J, ms) GETB(K, ms) GETB(F, ms) GETB(Bm, (size_t)nmol * BDIIS * BDIIS) GETB(coef, (size_t)nmol * BDIIS)
    GETB(E, nmol) GETB(Eold, nmol) GETB(rms, nmol) GETB(enuc, nmol)
    GETB(Fc, ms) GETB(Dc, ms) GETB(Sc, ms) GETB(Xc, ms) GETB(shc, (size_t)nmol * ld) GETB(T1, ms) GETB(T2, ms)
    GETB(Epc, ms) GETB(Fdc, ms) GETB(Dnc, ms) GETB(w, (size_t)nmol * ld)
    for (int k = 0; k < ds; ++k) { GETB(Fs.p[k], ms) GETB(Es.p[k], ms) }
    GETB(conv, nmol) GETB(iters, nmol) GETB(d_nocc, nmol) GETB(info, nmol) GETB(mode, nmol) GETB(acc, 6)
    GETB(bst, 1) GETB(kdm, nmol) GETB(restart, nmol) GETB(act, nmol) GETB(nocc_c, nmol)
    if (restart_iter) GETB(Dcore, ms)
#undef GETB
    if (cudaHostAlloc((void**)&open_hist, hist_len * sizeof(unsigned int), cudaHostAllocMapped) != cudaSuccess ||
        cudaHostGetDevicePointer((void**)&open_dev, open_hist, 0) != cudaSuccess) {
        open_hist = nullptr;
        set_error("cq_scf_batch: mapped host allocation failed");
        return fail(CQ_ERR_OOM);
    }
    for (int i = 0; i < hist_len; ++i) open_hist[i] = 0xffffffffu;
    for (cudaEvent_t* e : {&iev[0], &iev[1]})
        if (cudaEventCreateWithFlags(e, cudaEventDisableTiming) != cudaSuccess) return fail(CQ_ERR_CUDA);
    if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) return fail(CQ_ERR_CUDA);
    // ---- one-electron data, orthogonalisers
    if ((rc = cq_one_electron(b, S, T, V, nullptr, nullptr, s))) return fail(rc);
    slot_axpby_kernel<<<nb256(ms), 256, 0, s>>>(ms, 1.0, T, 1.0, V, H);
    {
        std::vector<double> en(nmol);
        if ((rc = cq_nuclear_repulsion_batch(b, en.data()))) return fail(rc);
        if (cudaMemcpyAsync(enuc, en.data(), nmol * sizeof(double), cudaMemcpyHostToDevice, s) ||
            cudaMemcpyAsync(d_nocc, nocc, nmol * sizeof(int), cudaMemcpyHostToDevice, s) ||
            cudaStreamSynchronize(s))
            return fail(CQ_ERR_CUDA);
    }
    if (cusolverDnCreateParams(&prm) != CUSOLVER_STATUS_SUCCESS) return fail(CQ_ERR_CUDA);
    size_t dws = 0, hws = 0;
    if (cusolverDnXsyevBatched_bufferSize(sol, prm, CUSOLVER_EIG_MODE_VECTOR, CUBLAS_FILL_MODE_LOWER, ld, CUDA_R_64F, T1,
                                          ld, CUDA_R_64F, w, CUDA_R_64F, &dws, &hws, nmol) != CUSOLVER_STATUS_SUCCESS) {
        set_error("cusolverDnXsyevBatched_bufferSize failed");
        return fail(CQ_ERR_CUDA);
    }
    if (cudaMalloc(&dwork, dws > 0 ? dws : 1) != cudaSuccess) { set_error("cq_scf_batch: OOM"); return fail(CQ_ERR_OOM); }
    hwork.resize(hws > 0 ? hws : 1);
    // eigenpairs of the first kb slots of A (the workspace is sized for nmol)
    auto eig = [&](double* A, int kb) -> int {
        if (cusolverDnXsyevBatched(sol, prm, CUSOLVER_EIG_MODE_VECTOR, CUBLAS_FILL_MODE_LOWER, ld, CUDA_R_64F, A, ld,
                                   CUDA_R_64F, w, CUDA_R_64F, dwork, dws, hwork.data(), hws, info,
                                   kb) != CUSOLVER_STATUS_SUCCESS) {
            set_error("cusolverDnXsyevBatched failed");
            return CQ_ERR_CUDA;
        }
        return CQ_OK;
    };
    pad_overlap_kernel<<<nb256(ms), 256, 0, s>>>(nmol, ld, b->d_mol_n, S, T1);
    if ((rc = eig(T1, nmol))) return fail(rc);
    batch_ortho_kernel<<<nb256(ms), 256, 0, s>>>(nmol, ld, T1, w, X, shift);
    auto gather = [&](int kb, size_t n, const double* s0, double* d0, const double* s1, double* d1,
                      const double* s2, double* d2) {
        Gather3 g{{s0, s1, s2}, {d0, d1, d2}};
        batch_gather_kernel<<<nb256((size_t)kb * n), 256, 0, s>>>(kb, n, act, g);
    };
    // orthogonal-basis Fock matrices Xc^T Fm Xc of the compact slots, shifted, into T2
    auto ortho_fock = [&](int kb, const double* Fm) -> int {
        CQ_BLAS_B(gemm_batch(blas, true, false, ld, kb, 1.0, Xc, Fm, 0.0, T1));
        CQ_BLAS_B(gemm_batch(blas, false, false, ld, kb, 1.0, T1, Xc, 0.0, T2));
        add_diag_kernel<<<nb256((size_t)kb * ld), 256, 0, s>>>(kb, ld, shc, T2);
        return CQ_OK;
    };
    // rows of T2 are eigenvectors: C = Xc T2^T, occupied columns kept, Dnc = C C^T
    auto density_c = [&](int kb) -> int {
        CQ_BLAS_B(gemm_batch(blas, false, true, ld, kb, 1.0, Xc, T2, 0.0, T1));
        occ_mask_kernel<<<nb256((size_t)kb * slot), 256, 0, s>>>(kb, ld, nocc_c, T1);
        CQ_BLAS_B(gemm_batch(blas, false, true, ld, kb, 1.0, T1, T1, 0.0, Dnc));
        return CQ_OK;
    };
    if (cudaMemsetAsync(conv, 0, nmol * sizeof(int), s) || cudaMemsetAsync(iters, 0, nmol * sizeof(int), s) ||
        cudaMemsetAsync(Eold, 0, nmol * sizeof(double), s) || cudaMemsetAsync(E, 0, nmol * sizeof(double), s) ||
        cudaMemsetAsync(acc, 0, 6 * sizeof(unsigned long long), s) || cudaMemsetAsync(bst, 0, sizeof(BatchState), s) ||
        cudaMemsetAsync(kdm, 0, nmol * sizeof(int), s) || cudaMemsetAsync(restart, 0, nmol * sizeof(int), s))
        return fail(CQ_ERR_CUDA);
    const int mode0 = o.prec == CQ_PREC_MIXED ? MODE_FP32 : 0;
    fill_int_kernel<<<(nmol + 127) / 128, 128, 0, s>>>(nmol, mode0, mode);
    // core-guess density of every molecule into dst (the starting density, or
    // the fallback of a supplied one)
    auto core_guess = [&](double* dst) -> int {
        batch_begin_kernel<<<1, 1024, 0, s>>>(nmol, nmol, conv, d_nocc, bst, act, nocc_c);
        gather(nmol, slot, H, Fdc, X, Xc, nullptr, nullptr);
        gather(nmol, ld, shift, shc, nullptr, nullptr, nullptr, nullptr);
        int r;
        if ((r = ortho_fock(nmol, Fdc)) || (r = eig(T2, nmol)) || (r = density_c(nmol))) return r;
        batch_scatter_kernel<<<nb256(ms), 256, 0, s>>>(nmol, ld, act, bst, nullptr, nullptr, Dnc, nullptr, dst);
        return cudaGetLastError() == cudaSuccess ? CQ_OK : CQ_ERR_CUDA;
    };
    if (restart_iter && (rc = core_guess(Dcore))) return fail(rc);
    if (D_in) {
        if (cudaMemcpyAsync(D, D_in, ms * sizeof(double), cudaMemcpyDeviceToDevice, s)) return fail(CQ_ERR_CUDA);
    } else if ((rc = core_guess(D))) {
        return fail(rc);
    }
    // the set-up passes above advanced the iteration counter
    if (cudaMemsetAsync(bst, 0, sizeof(BatchState), s)) return fail(CQ_ERR_CUDA);
    // Phase A of an iteration over kb compact slots (kb >= open molecules):
    // compaction, Fock build for the open molecules, energy, orthogonal-basis
    // error, convergence test, DIIS extrapolation (not on the first iteration
    // from a supplied density, which need not be idempotent), Xc^T F Xc.  Then
    // the eigensolver, then phase B (density, written back per molecule).
    auto phase_a = [&](int kb, bool first) -> int {
        batch_begin_kernel<<<1, 1024, 0, s>>>(nmol, kb, conv, d_nocc, bst, act, nocc_c);
        cq_fock_opts fo{o.schwarz_tol, o.mixed_tol, o.prec, 1, 1, o.fp64_tol};
        int r = fock_build_modes(b, CQ_DENS_REAL_SYM, D, J, K, &fo, nullptr, s, mode, acc);
        if (r) return r;
        batch_fock_kernel<<<nb256(ms), 256, 0, s>>>(ms, H, J, K, F);
        const size_t nc = (size_t)kb * slot;
        gather(kb, slot, F, Fc, D, Dc, S, Sc);
        gather(kb, slot, X, Xc, nullptr, nullptr, nullptr, nullptr);
        gather(kb, ld, shift, shc, nullptr, nullptr, nullptr, nullptr);
        CQ_BLAS_B(gemm_batch(blas, false, false, ld, kb, 1.0, Fc, Dc, 0.0, T1));
        CQ_BLAS_B(gemm_batch(blas, false, false, ld, kb, 1.0, T1, Sc, 0.0, T2));
        batch_antisym_kernel<<<nb256(nc), 256, 0, s>>>(kb, ld, T2, Fdc);
        CQ_BLAS_B(gemm_batch(blas, true, false, ld, kb, 1.0, Xc, Fdc, 0.0, T1));
        CQ_BLAS_B(gemm_batch(blas, false, false, ld, kb, 1.0, T1, Xc, 0.0, Epc));
        batch_energy_rms_kernel<<<kb, 256, 0, s>>>(ld, act, bst, H, F, D, Epc, enuc, b->d_mol_n, E, rms);
        batch_conv_kernel<<<(nmol + 127) / 128, 128, 0, s>>>(nmol, E, Eold, rms, o.e_tol, o.d_tol, o.switch_tol,
                                                             restart_iter, mode0, conv, iters, mode, restart, bst);
        batch_publish_kernel<<<1, 32, 0, s>>>(bst, open_dev, hist_len);
        if (cudaMemcpyAsync(Eold, E, nmol * sizeof(double), cudaMemcpyDeviceToDevice, s)) return CQ_ERR_CUDA;
        const double* Fuse = Fc;
        if (!first) {
            batch_diis_index_kernel<<<1, 32, 0, s>>>(bst, ds);
            batch_store_slot_kernel<<<nb256(nc), 256, 0, s>>>(kb, ld, Fs, Es, bst, act, Fc, Epc);
            batch_dot_kernel<<<dim3(kb, BDIIS), 256, 0, s>>>(ld, Es, bst, act, Bm);
            batch_diis_solve_kernel<<<(nmol + 127) / 128, 128, 0, s>>>(nmol, bst, conv, restart, kdm, Bm, coef);
            batch_diis_combine_kernel<<<nb256(nc), 256, 0, s>>>(kb, ld, Fs, bst, act, conv, kdm, coef, Fc, Fdc);
            Fuse = Fdc;
        }
        if ((r = ortho_fock(kb, Fuse))) return r;
        return cudaGetLastError() == cudaSuccess ? CQ_OK : CQ_ERR_CUDA;
    };
    auto phase_b = [&](int kb) -> int {
        int r = density_c(kb);
        if (r) return r;
        batch_scatter_kernel<<<nb256((size_t)kb * slot), 256, 0, s>>>(kb, ld, act, bst, conv, restart, Dnc, Dcore, D);
        return cudaGetLastError() == cudaSuccess ? CQ_OK : CQ_ERR_CUDA;
    };
    auto capture = [&](auto&& fn, cudaGraphExec_t* out) -> bool {
        cudaGraph_t g = nullptr;
        *out = nullptr;
        if (cudaStreamBeginCapture(s, cudaStreamCaptureModeRelaxed) != cudaSuccess) {
            cudaGetLastError();
            return false;
        }
        const int r = fn();
        const cudaError_t ce = cudaStreamEndCapture(s, &g);
        bool ok = r == CQ_OK && ce == cudaSuccess && g != nullptr;
        if (ok && cudaGraphInstantiate(out, g, 0) != cudaSuccess) ok = false;
        if (g) cudaGraphDestroy(g);
        if (!ok) {
            if (*out) cudaGraphExecDestroy(*out);
            *out = nullptr;
            cudaGetLastError();
        }
        return ok;
    };
    // graphs per compact size kb, captured on first use: the whole iteration
    // (level 2) or the two phases around an eager eigensolver call (level 1)
    int graph_level = o.graph && !b->profile ? 2 : 0;
    auto graphs_for = [&](int kb) -> Graphs* {
        for (Graphs& g : graphs)
            if (g.kb == kb) return &g;
        Graphs g{kb, nullptr, nullptr, nullptr};
        if (graph_level == 2 &&
            !capture([&]() {
                int r = phase_a(kb, false);
                if (!r) r = eig(T2, kb);
                if (!r) r = phase_b(kb);
                return r;
            }, &g.full))
            graph_level = 1;
        if (graph_level == 1 && !g.full) {
            if (!capture([&]() { return phase_a(kb, false); }, &g.a) || !capture([&]() { return phase_b(kb); }, &g.b)) {
                if (g.a) cudaGraphExecDestroy(g.a);
                g.a = nullptr;
                graph_level = 0;
            }
        }
        graphs.push_back(g);
        return &graphs.back();
    };
    auto run_iter = [&](int kb, bool first, bool eager) -> int {
        Graphs* g = eager || graph_level == 0 ? nullptr : graphs_for(kb);
        if (g && g->full) return cudaGraphLaunch(g->full, s) == cudaSuccess ? CQ_OK : CQ_ERR_CUDA;
        int r;
        if (g && g->a) {
            if (cudaGraphLaunch(g->a, s) != cudaSuccess) return CQ_ERR_CUDA;
            if ((r = eig(T2, kb))) return r;
            return cudaGraphLaunch(g->b, s) == cudaSuccess ? CQ_OK : CQ_ERR_CUDA;
        }
        if ((r = phase_a(kb, first)) || (r = eig(T2, kb))) return r;
        return phase_b(kb);
    };
    // compact size for a known number of open molecules: the next power of
    // two, at most nmol (so a handful of graphs covers the whole run)
    auto bucket = [&](int open) {
        int kb = 1;
        while (kb < open) kb <<= 1;
        return kb < nmol ? kb : nmol;
    };
    // Iteration 1 runs eagerly (it also sizes the build's scratch); later
    // iterations replay the graph of their compact size.  The host reads the
    // open count of iteration k-1 while iteration k runs (so the compact size
    // of iteration k+1 bounds its open molecules); iterations after the last
    // molecule converged skip every quartet and every dense step.
    cudaEventRecord(e0, s);
    int done = 0, known_open = nmol;
    for (int it = 1; it <= o.max_iter; ++it) {
        const int kb = bucket(known_open);
        if ((rc = run_iter(kb, it == 1 && D_in != nullptr, it == 1))) return fail(rc);
        if (cudaEventRecord(iev[it & 1], s) != cudaSuccess) return fail(CQ_ERR_CUDA);
        done = it;
        if (it >= 2) {
            if (cudaEventSynchronize(iev[(it - 1) & 1]) != cudaSuccess) return fail(CQ_ERR_CUDA);
            known_open = (int)open_hist[it - 1];
            if (known_open == 0) {
                done = it - 1;
                break;
            }
        }
    }
    cudaEventRecord(e1, s);
    if (cudaMemcpyAsync(D_out, D, ms * sizeof(double), cudaMemcpyDeviceToDevice, s)) return fail(CQ_ERR_CUDA);
    std::vector<double> hE(nmol);
    std::vector<int> hit(nmol), hconv(nmol);
    unsigned long long hacc[6];
    if (cudaMemcpyAsync(hE.data(), E, nmol * sizeof(double), cudaMemcpyDeviceToHost, s) ||
        cudaMemcpyAsync(hit.data(), iters, nmol * sizeof(int), cudaMemcpyDeviceToHost, s) ||
        cudaMemcpyAsync(hconv.data(), conv, nmol * sizeof(int), cudaMemcpyDeviceToHost, s) ||
        cudaMemcpyAsync(hacc, acc, sizeof hacc, cudaMemcpyDeviceToHost, s) || cudaStreamSynchronize(s))
        return fail(CQ_ERR_CUDA);
    float msf = 0.f;
    cudaEventElapsedTime(&msf, e0, e1);
    cq_scf_stats st;
    memset(&st, 0, sizeof st);
    int nconv = 0;
    double esum = 0.0;
    for (int m = 0; m < nmol; ++m) {
        if (E_out) E_out[m] = hE[m];
        if (iters_out) iters_out[m] = hconv[m] ? hit[m] : o.max_iter;
        nconv += hconv[m];
        esum += hE[m];
    }
    st.energy = esum;
    st.iterations = done;
    st.converged = nconv;
    st.quartets_fp64 = hacc[0];
    st.quartets_fp32 = hacc[2];
    st.quartets_df = hacc[4];
    st.ms = msf;
    st.graph = o.graph && !b->profile ? graph_level : 0;
    if (stats) *stats = st;
    fail(CQ_OK);
    if (nconv < nmol) {
        set_error("cq_scf_batch: " + std::to_string(nmol - nconv) + " molecule(s) not converged");
        return CQ_ERR_NOT_CONVERGED;
    }
    return CQ_OK;
}
