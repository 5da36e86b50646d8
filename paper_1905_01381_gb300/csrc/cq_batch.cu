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
// subspace size and the slots from oldest to newest) and the number of
// molecules still open after the iteration's convergence test.
struct BatchState {
    int it;
    int kd;
    int slot, nvec;
    int order[BDIIS];
    unsigned int nopen;
};

// per-molecule mode bits read by the Fock build (ClassifyArgs::mol_mode)
constexpr int MODE_FP32 = 1;
constexpr int MODE_SKIP = 2;

__global__ void batch_iter_begin_kernel(BatchState* st)
{
    if (threadIdx.x == 0) {
        st->it += 1;
        st->nopen = 0u;
    }
}

// per open molecule (one block each): E = sum (H + F) D + Enuc; rms of E'
__global__ void batch_energy_rms_kernel(int ld, const double* __restrict__ H, const double* __restrict__ F,
                                        const double* __restrict__ D, const double* __restrict__ Ep,
                                        const double* __restrict__ enuc, const int* __restrict__ mol_n,
                                        const int* __restrict__ conv, double* __restrict__ E, double* __restrict__ rms)
{
    __shared__ double r0[256], r1[256];
    const int m = blockIdx.x;
    if (conv[m]) return;
    const size_t slot = (size_t)ld * ld, o = (size_t)m * slot;
    double e = 0.0, q = 0.0;
    for (size_t i = threadIdx.x; i < slot; i += blockDim.x) {
        e += (H[o + i] + F[o + i]) * D[o + i];
        q += Ep[o + i] * Ep[o + i];
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
// skipped by later builds; the open count goes to the state and to the
// host-visible history (one entry per iteration).
__global__ void batch_conv_kernel(int nmol, const double* __restrict__ E, const double* __restrict__ Eold,
                                  const double* __restrict__ rms, double e_tol, double d_tol, double switch_tol,
                                  int* __restrict__ conv, int* __restrict__ iters, int* __restrict__ mode,
                                  BatchState* st)
{
    const int m = blockIdx.x * blockDim.x + threadIdx.x;
    if (m >= nmol || conv[m]) return;
    const int it = st->it;
    const int md = mode[m];
    if (it > 1 && !(md & MODE_FP32) && fabs(E[m] - Eold[m]) < e_tol && rms[m] < d_tol) {
        conv[m] = 1;
        iters[m] = it;
        mode[m] = md | MODE_SKIP;
        return;
    }
    if ((md & MODE_FP32) && rms[m] < switch_tol) mode[m] = md & ~MODE_FP32;
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

// F and E' of the open molecules into the newest ring slot
__global__ void batch_store_slot_kernel(int nmol, int ld, SlotPtrs Fs, SlotPtrs Es, const BatchState* st,
                                        const int* __restrict__ conv, const double* __restrict__ F,
                                        const double* __restrict__ Ep)
{
    const size_t slot = (size_t)ld * ld;
    const size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= slot * nmol || conv[i / slot]) return;
    const int k = st->slot;
    Fs.p[k][i] = F[i];
    Es.p[k][i] = Ep[i];
}

// B[m][slot][k] = e_slot . e_k for the ring slots k (grid: molecules x BDIIS)
__global__ void batch_dot_kernel(int ld, SlotPtrs Es, const BatchState* st, const int* __restrict__ conv,
                                 double* __restrict__ Bm)
{
    __shared__ double red[256];
    const int m = blockIdx.x, p = blockIdx.y;
    if (p >= st->nvec || conv[m]) return;
    const int pi = st->slot, pj = st->order[p];
    const size_t slot = (size_t)ld * ld, o = (size_t)m * slot;
    const double* a = Es.p[pi] + o;
    const double* b = Es.p[pj] + o;
    double s = 0.0;
    for (size_t i = threadIdx.x; i < slot; i += blockDim.x) s += a[i] * b[i];
    red[threadIdx.x] = s;
    __syncthreads();
    for (int k = blockDim.x / 2; k > 0; k >>= 1) {
        if ((int)threadIdx.x < k) red[threadIdx.x] += red[threadIdx.x + k];
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        Bm[(size_t)m * BDIIS * BDIIS + pi * BDIIS + pj] = red[0];
        Bm[(size_t)m * BDIIS * BDIIS + pj * BDIIS + pi] = red[0];
    }
}

// Per open molecule: the DIIS coefficients over the ring slots (oldest to
// newest) from the bordered system [B -1; -1 0][c; l] = [0; -1], by
// Gaussian elimination with partial pivoting; one vector gives c = 1.
__global__ void batch_diis_solve_kernel(int nmol, const BatchState* st, const int* __restrict__ conv,
                                        const double* __restrict__ Bm, double* __restrict__ coef)
{
    const int mol = blockIdx.x * blockDim.x + threadIdx.x;
    if (mol >= nmol || conv[mol]) return;
    const int m = st->nvec, N = m + 1;
    double* c = coef + (size_t)mol * BDIIS;
    if (m < 2) {
        c[0] = 1.0;
        return;
    }
    double A[BDIIS + 1][BDIIS + 2];
    const double* B = Bm + (size_t)mol * BDIIS * BDIIS;
    for (int i = 0; i < m; ++i) {
        for (int j = 0; j < m; ++j) A[i][j] = B[st->order[i] * BDIIS + st->order[j]];
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

// extrapolated Fock matrices (a converged molecule, whose build was
// skipped, takes its current F so that its slot stays finite)
__global__ void batch_diis_combine_kernel(int nmol, int ld, SlotPtrs F, const BatchState* st,
                                          const int* __restrict__ conv, const double* __restrict__ coef,
                                          const double* __restrict__ Fcur, double* __restrict__ out)
{
    const size_t slot = (size_t)ld * ld;
    const size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= slot * nmol) return;
    const int m = (int)(i / slot);
    if (conv[m]) {
        out[i] = Fcur[i];
        return;
    }
    const int nvec = st->nvec;
    double s = 0.0;
    for (int k = 0; k < nvec; ++k) s += coef[(size_t)m * BDIIS + k] * F.p[st->order[k]][i];
    out[i] = s;
}

__global__ void fill_int_kernel(int n, int v, int* __restrict__ x)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) x[i] = v;
}

// keep the first nocc[m] columns of C (the occupied orbitals)
__global__ void occ_mask_kernel(int nmol, int ld, const int* __restrict__ nocc, double* __restrict__ C)
{
    const size_t slot = (size_t)ld * ld;
    const size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= slot * nmol) return;
    const int m = (int)(i / slot), c = (int)(i % ld);
    if (c >= nocc[m]) C[i] = 0.0;
}

// D <- Dnew for molecules still iterating
__global__ void freeze_update_kernel(int nmol, int ld, const int* __restrict__ conv, const double* __restrict__ Dnew,
                                     double* __restrict__ D)
{
    const size_t slot = (size_t)ld * ld;
    const size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= slot * nmol) return;
    if (!conv[i / slot]) D[i] = Dnew[i];
}

static int nb256(size_t n) { return (int)((n + 255) / 256); }

}  // namespace cq

using namespace cq;

extern "C" int cq_scf_batch(cq_basis* b, const int* nocc, const cq_scf_opts* opts, const double* D_in, double* D_out,
                            double* E_out, int* iters_out, cq_scf_stats* stats, void* stream)
{
    if (!b || !nocc || !D_out) { set_error("cq_scf_batch: NULL argument"); return CQ_ERR_INVALID_ARG; }
    cq_scf_opts o{1e-10, 1e-8, 128, 8, CQ_PREC_FP64, 1e-5, 1e-14, 0, 8, 1e-5, 1};
    if (opts) o = *opts;
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
    const int ds = o.diis_size;
    std::vector<void*> bufs;
    int rc = CQ_OK;
    auto get = [&](auto** p, size_t n) -> int {
        int r = dalloc(p, n);
        if (!r) bufs.push_back((void*)*p);
        return r;
    };
    double *S, *T, *V, *H, *X, *shift, *w, *D, *Dn, *J, *K, *F, *T1, *T2, *Err, *Ep, *Fd, *Bm, *coef, *E, *Eold,
        *rms, *enuc;
    int *conv, *iters, *d_nocc, *info, *mode;
    unsigned long long* acc;
    BatchState* bst;
    SlotPtrs Fs{}, Es{};
    cusolverDnParams_t prm = nullptr;
    void* dwork = nullptr;
    std::vector<char> hwork;
    unsigned int* open_hist = nullptr;   // mapped host memory, one entry per iteration
    unsigned int* open_dev = nullptr;
    cudaGraphExec_t gx_full = nullptr, gx_a = nullptr, gx_b = nullptr;
    cudaEvent_t iev[2] = {nullptr, nullptr}, e0 = nullptr, e1 = nullptr;
    const int hist_len = o.max_iter + 2;
    auto fail = [&](int r) {
        if (r != CQ_OK) cudaStreamSynchronize(s);
        if (gx_full) cudaGraphExecDestroy(gx_full);
        if (gx_a) cudaGraphExecDestroy(gx_a);
        if (gx_b) cudaGraphExecDestroy(gx_b);
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
    GETB(S, ms) GETB(T, ms) GETB(V, ms) GETB(H, ms) GETB(X, ms) GETB(shift, (size_t)nmol * ld) GETB(w, (size_t)nmol * ld)
    GETB(D, ms) GETB(Dn, ms) GETB(J, ms) GETB(K, ms) GETB(F, ms) GETB(T1, ms) GETB(T2, ms) GETB(Err, ms) GETB(Ep, ms)
    GETB(Fd, ms) GETB(Bm, (size_t)nmol * BDIIS * BDIIS) GETB(coef, (size_t)nmol * BDIIS) GETB(E, nmol) GETB(Eold, nmol)
    GETB(rms, nmol) GETB(enuc, nmol)
    for (int k = 0; k < ds; ++k) { GETB(Fs.p[k], ms) GETB(Es.p[k], ms) }
    GETB(conv, nmol) GETB(iters, nmol) GETB(d_nocc, nmol) GETB(info, nmol) GETB(mode, nmol) GETB(acc, 4)
    GETB(bst, 1)
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
    auto eig = [&](double* A) -> int {
        if (cusolverDnXsyevBatched(sol, prm, CUSOLVER_EIG_MODE_VECTOR, CUBLAS_FILL_MODE_LOWER, ld, CUDA_R_64F, A, ld,
                                   CUDA_R_64F, w, CUDA_R_64F, dwork, dws, hwork.data(), hws, info,
                                   nmol) != CUSOLVER_STATUS_SUCCESS) {
            set_error("cusolverDnXsyevBatched failed");
            return CQ_ERR_CUDA;
        }
        return CQ_OK;
    };
    pad_overlap_kernel<<<nb256(ms), 256, 0, s>>>(nmol, ld, b->d_mol_n, S, T1);
    if ((rc = eig(T1))) return fail(rc);
    batch_ortho_kernel<<<nb256(ms), 256, 0, s>>>(nmol, ld, T1, w, X, shift);
    // orthogonal-basis Fock matrix X^T F X, shifted, into T2 (diagonalised in place)
    auto ortho_fock = [&](const double* Fm) -> int {
        CQ_BLAS_B(gemm_batch(blas, true, false, ld, nmol, 1.0, X, Fm, 0.0, T1));
        CQ_BLAS_B(gemm_batch(blas, false, false, ld, nmol, 1.0, T1, X, 0.0, T2));
        add_diag_kernel<<<nb256((size_t)nmol * ld), 256, 0, s>>>(nmol, ld, shift, T2);
        return CQ_OK;
    };
    // rows of T2 are eigenvectors: C = X T2^T, occupied columns kept,
    // D = C C^T taken by the molecules still open
    auto new_density = [&]() -> int {
        CQ_BLAS_B(gemm_batch(blas, false, true, ld, nmol, 1.0, X, T2, 0.0, T1));
        occ_mask_kernel<<<nb256(ms), 256, 0, s>>>(nmol, ld, d_nocc, T1);
        CQ_BLAS_B(gemm_batch(blas, false, true, ld, nmol, 1.0, T1, T1, 0.0, Dn));
        freeze_update_kernel<<<nb256(ms), 256, 0, s>>>(nmol, ld, conv, Dn, D);
        return cudaGetLastError() == cudaSuccess ? CQ_OK : CQ_ERR_CUDA;
    };
    if (cudaMemsetAsync(conv, 0, nmol * sizeof(int), s) || cudaMemsetAsync(iters, 0, nmol * sizeof(int), s) ||
        cudaMemsetAsync(Eold, 0, nmol * sizeof(double), s) || cudaMemsetAsync(E, 0, nmol * sizeof(double), s) ||
        cudaMemsetAsync(acc, 0, 4 * sizeof(unsigned long long), s) || cudaMemsetAsync(bst, 0, sizeof(BatchState), s))
        return fail(CQ_ERR_CUDA);
    fill_int_kernel<<<(nmol + 127) / 128, 128, 0, s>>>(nmol, o.prec == CQ_PREC_MIXED ? MODE_FP32 : 0, mode);
    if (D_in) {
        if (cudaMemcpyAsync(D, D_in, ms * sizeof(double), cudaMemcpyDeviceToDevice, s)) return fail(CQ_ERR_CUDA);
    } else {
        if ((rc = ortho_fock(H)) || (rc = eig(T2)) || (rc = new_density())) return fail(rc);
    }
    // Phase A of an iteration: Fock build for the open molecules, energy,
    // orthogonal-basis error, convergence test, DIIS extrapolation (not on
    // the first iteration from a supplied density, which need not be
    // idempotent), X^T F X.  Then the eigensolver, then phase B (density).
    auto phase_a = [&](bool first) -> int {
        batch_iter_begin_kernel<<<1, 32, 0, s>>>(bst);
        cq_fock_opts fo{o.schwarz_tol, o.mixed_tol, o.prec, 1, 1};
        int r = fock_build_modes(b, CQ_DENS_REAL_SYM, D, J, K, &fo, nullptr, s, mode, acc);
        if (r) return r;
        batch_fock_kernel<<<nb256(ms), 256, 0, s>>>(ms, H, J, K, F);
        CQ_BLAS_B(gemm_batch(blas, false, false, ld, nmol, 1.0, F, D, 0.0, T1));
        CQ_BLAS_B(gemm_batch(blas, false, false, ld, nmol, 1.0, T1, S, 0.0, T2));
        batch_antisym_kernel<<<nb256(ms), 256, 0, s>>>(nmol, ld, T2, Err);
        CQ_BLAS_B(gemm_batch(blas, true, false, ld, nmol, 1.0, X, Err, 0.0, T1));
        CQ_BLAS_B(gemm_batch(blas, false, false, ld, nmol, 1.0, T1, X, 0.0, Ep));
        batch_energy_rms_kernel<<<nmol, 256, 0, s>>>(ld, H, F, D, Ep, enuc, b->d_mol_n, conv, E, rms);
        batch_conv_kernel<<<(nmol + 127) / 128, 128, 0, s>>>(nmol, E, Eold, rms, o.e_tol, o.d_tol, o.switch_tol, conv,
                                                             iters, mode, bst);
        batch_publish_kernel<<<1, 32, 0, s>>>(bst, open_dev, hist_len);
        if (cudaMemcpyAsync(Eold, E, nmol * sizeof(double), cudaMemcpyDeviceToDevice, s)) return CQ_ERR_CUDA;
        const double* Fuse = F;
        if (!first) {
            batch_diis_index_kernel<<<1, 32, 0, s>>>(bst, ds);
            batch_store_slot_kernel<<<nb256(ms), 256, 0, s>>>(nmol, ld, Fs, Es, bst, conv, F, Ep);
            batch_dot_kernel<<<dim3(nmol, BDIIS), 256, 0, s>>>(ld, Es, bst, conv, Bm);
            batch_diis_solve_kernel<<<(nmol + 127) / 128, 128, 0, s>>>(nmol, bst, conv, Bm, coef);
            batch_diis_combine_kernel<<<nb256(ms), 256, 0, s>>>(nmol, ld, Fs, bst, conv, coef, F, Fd);
            Fuse = Fd;
        }
        if ((r = ortho_fock(Fuse))) return r;
        return cudaGetLastError() == cudaSuccess ? CQ_OK : CQ_ERR_CUDA;
    };
    auto whole = [&]() -> int {
        int r = phase_a(false);
        if (!r) r = eig(T2);
        if (!r) r = new_density();
        return r;
    };
    auto capture = [&](auto&& fn, cudaGraphExec_t* out) -> bool {
        cudaGraph_t g = nullptr;
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
            *out = nullptr;
            cudaGetLastError();
        }
        return ok;
    };
    int graph_used = 0;
    auto run_iter = [&](bool first) -> int {
        if (gx_full) return cudaGraphLaunch(gx_full, s) == cudaSuccess ? CQ_OK : CQ_ERR_CUDA;
        int r;
        if (gx_a) {
            if (cudaGraphLaunch(gx_a, s) != cudaSuccess) return CQ_ERR_CUDA;
            if ((r = eig(T2))) return r;
            return cudaGraphLaunch(gx_b, s) == cudaSuccess ? CQ_OK : CQ_ERR_CUDA;
        }
        if ((r = phase_a(first)) || (r = eig(T2))) return r;
        return new_density();
    };
    // Iteration 1 runs eagerly (it also sizes the build's scratch); the
    // later iterations are one launch sequence, captured once as a graph
    // (the eigensolver left outside it if it cannot be captured) and
    // replayed.  The host reads the open count of iteration k-1 while
    // iteration k runs; iterations after the last molecule converged skip
    // every quartet and leave every density as it is.
    cudaEventRecord(e0, s);
    int done = 0;
    for (int it = 1; it <= o.max_iter; ++it) {
        if (it == 2 && o.graph && !b->profile) {
            if (capture(whole, &gx_full)) {
                graph_used = 2;
            } else if (capture([&]() { return phase_a(false); }, &gx_a) && capture(new_density, &gx_b)) {
                graph_used = 1;
            } else {
                if (gx_a) cudaGraphExecDestroy(gx_a);
                gx_a = nullptr;
            }
        }
        if ((rc = run_iter(it == 1 && D_in != nullptr))) return fail(rc);
        if (cudaEventRecord(iev[it & 1], s) != cudaSuccess) return fail(CQ_ERR_CUDA);
        done = it;
        if (it >= 2) {
            if (cudaEventSynchronize(iev[(it - 1) & 1]) != cudaSuccess) return fail(CQ_ERR_CUDA);
            if (open_hist[it - 1] == 0u) {
                done = it - 1;
                break;
            }
        }
    }
    cudaEventRecord(e1, s);
    if (cudaMemcpyAsync(D_out, D, ms * sizeof(double), cudaMemcpyDeviceToDevice, s)) return fail(CQ_ERR_CUDA);
    std::vector<double> hE(nmol);
    std::vector<int> hit(nmol), hconv(nmol);
    unsigned long long hacc[4];
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
    st.ms = msf;
    st.graph = graph_used;
    if (stats) *stats = st;
    fail(CQ_OK);
    if (nconv < nmol) {
        set_error("cq_scf_batch: " + std::to_string(nmol - nconv) + " molecule(s) not converged");
        return CQ_ERR_NOT_CONVERGED;
    }
    return CQ_OK;
}
