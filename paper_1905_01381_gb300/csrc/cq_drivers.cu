// Dense drivers on the GPU: RHF direct SCF (Sec. "Self-Consistent Field
// Optimization": DIIS extrapolation of the Fock matrix) and one RT-TDHF
// step (Sec. "Real-Time Electronic Dynamics": MMUT leap-frog with EM2 seed
// and restart steps).  Dense algebra goes through cuBLAS (FP64 GEMM) and
// cuSOLVER (symmetric eigensolver); every other step is a kernel here.
#include <cublas_v2.h>
#include <cuComplex.h>
#include <cusolverDn.h>

#include <cmath>
#include <cstring>
#include <vector>

#include "cq_internal.h"

namespace cq {

#define CQ_BLAS(call)                                                        \
    do {                                                                     \
        cublasStatus_t _s = (call);                                          \
        if (_s != CUBLAS_STATUS_SUCCESS) {                                   \
            set_error(std::string("cuBLAS failure in ") + #call);            \
            return CQ_ERR_CUDA;                                              \
        }                                                                    \
    } while (0)
#define CQ_SOLVER(call)                                                      \
    do {                                                                     \
        cusolverStatus_t _s = (call);                                        \
        if (_s != CUSOLVER_STATUS_SUCCESS) {                                 \
            set_error(std::string("cuSOLVER failure in ") + #call);          \
            return CQ_ERR_CUDA;                                              \
        }                                                                    \
    } while (0)

// Row-major GEMM: C(MxN) = alpha op(A)(MxK) op(B)(KxN) + beta C, expressed as
// the column-major product C^T = op(B)^T op(A)^T.
static cublasStatus_t dgemm_rm(cublasHandle_t h, bool ta, bool tb, int M, int N, int K, double alpha,
                               const double* A, int lda, const double* B, int ldb, double beta, double* C, int ldc)
{
    return cublasDgemm(h, tb ? CUBLAS_OP_T : CUBLAS_OP_N, ta ? CUBLAS_OP_T : CUBLAS_OP_N, N, M, K, &alpha, B, ldb,
                       A, lda, &beta, C, ldc);
}

// op: 'N', 'T' or 'C' (conjugate transpose)
static cublasOperation_t zop(char c)
{
    return c == 'T' ? CUBLAS_OP_T : c == 'C' ? CUBLAS_OP_C : CUBLAS_OP_N;
}

static cublasStatus_t zgemm_rm(cublasHandle_t h, char ta, char tb, int M, int N, int K, cuDoubleComplex alpha,
                               const cuDoubleComplex* A, int lda, const cuDoubleComplex* B, int ldb,
                               cuDoubleComplex beta, cuDoubleComplex* C, int ldc)
{
    return cublasZgemm(h, zop(tb), zop(ta), N, M, K, &alpha, B, ldb, A, lda, &beta, C, ldc);
}

template <typename T>
static int scratch(cq_basis* b, T** p, size_t n)
{
    int rc = dalloc(p, n);
    if (rc) return rc;
    b->dense_bufs.push_back((void*)*p);
    return CQ_OK;
}

// ------------------------------------------------------------------ kernels

// X from the eigenpairs of S: row k of V holds eigenvector k (ascending w).
// Loewdin X = V w^{-1/2} V^T when nothing is dropped, else canonical
// X = V_keep w_keep^{-1/2}.  This kernel writes Y = V^T-columns / sqrt(w)
// restricted to kept eigenvectors: Y[i][j] = V[k0 + j][i] / sqrt(w[k0 + j]).
__global__ void ortho_y_kernel(int n, int m, int k0, const double* __restrict__ V, const double* __restrict__ w,
                               double* __restrict__ Y)
{
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= n * m) return;
    const int i = t / m, j = t % m;
    Y[t] = V[(size_t)(k0 + j) * n + i] * rsqrt(w[k0 + j]);
}

__global__ void add_kernel(size_t n, double a, const double* __restrict__ x, double b, const double* __restrict__ y,
                           double* __restrict__ z)
{
    const size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) z[i] = a * x[i] + b * y[i];
}

// G (=) 2J - K (optionally accumulated), F = h + G
__global__ void fock_real_kernel(size_t nn, int accumulate, const double* __restrict__ h, const double* __restrict__ J,
                                 const double* __restrict__ K, double* __restrict__ G, double* __restrict__ F)
{
    const size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= nn) return;
    const double g = 2.0 * J[i] - K[i] + (accumulate ? G[i] : 0.0);
    G[i] = g;
    F[i] = h[i] + g;
}

// out = sum_i A_i B_i (fixed-order block reduction, one block)
__global__ void dot_kernel(size_t n, const double* __restrict__ A, const double* __restrict__ B, double add,
                           double scale, int take_sqrt, double* __restrict__ out)
{
    __shared__ double red[256];
    double s = 0.0;
    for (size_t i = threadIdx.x; i < n; i += blockDim.x) s += A[i] * (B ? B[i] : A[i]);
    red[threadIdx.x] = s;
    __syncthreads();
    for (int o = blockDim.x / 2; o > 0; o >>= 1) {
        if ((int)threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        const double v = red[0] * scale + add;
        *out = take_sqrt ? sqrt(v) : v;
    }
}

// E = sum_ij (h + F)_ij D_ij + Enuc (D symmetric)
__global__ void rhf_energy_kernel(size_t nn, const double* __restrict__ h, const double* __restrict__ F,
                                  const double* __restrict__ D, double enuc, double* __restrict__ out)
{
    __shared__ double red[256];
    double s = 0.0;
    for (size_t i = threadIdx.x; i < nn; i += blockDim.x) s += (h[i] + F[i]) * D[i];
    red[threadIdx.x] = s;
    __syncthreads();
    for (int o = blockDim.x / 2; o > 0; o >>= 1) {
        if ((int)threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x == 0) *out = red[0] + enuc;
}

// err = T - T^T
__global__ void antisym_kernel(int n, const double* __restrict__ T, double* __restrict__ E)
{
    const size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= (size_t)n * n) return;
    const int r = (int)(i / n), c = (int)(i % n);
    E[i] = T[i] - T[(size_t)c * n + r];
}

// DIIS: B_ij = e_i . e_j for the vectors in the ring (slot ids in order),
// then solve [B -1; -1 0] [c; l] = [0; -1] by Gaussian elimination with
// partial pivoting (one thread; the subspace has at most 8 vectors).
constexpr int DIIS_MAX = 8;
__global__ void diis_solve_kernel(int m, const double* __restrict__ Bfull, const int* __restrict__ slots,
                                  double* __restrict__ coef)
{
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    double A[DIIS_MAX + 1][DIIS_MAX + 2];
    for (int i = 0; i < m; ++i) {
        for (int j = 0; j < m; ++j) A[i][j] = Bfull[slots[i] * DIIS_MAX + slots[j]];
        A[i][m] = -1.0;
        A[i][m + 1] = 0.0;
    }
    for (int j = 0; j < m; ++j) A[m][j] = -1.0;
    A[m][m] = 0.0;
    A[m][m + 1] = -1.0;
    const int N = m + 1;
    for (int c = 0; c < N; ++c) {
        int piv = c;
        for (int r = c + 1; r < N; ++r)
            if (fabs(A[r][c]) > fabs(A[piv][c])) piv = r;
        if (piv != c)
            for (int k = 0; k <= N; ++k) { const double t = A[c][k]; A[c][k] = A[piv][k]; A[piv][k] = t; }
        const double d = A[c][c];
        if (fabs(d) < 1e-300) {  // singular subspace: fall back to the newest vector
            for (int i = 0; i < m; ++i) coef[i] = (i == m - 1) ? 1.0 : 0.0;
            return;
        }
        for (int r = c + 1; r < N; ++r) {
            const double f = A[r][c] / d;
            for (int k = c; k <= N; ++k) A[r][k] -= f * A[c][k];
        }
    }
    double x[DIIS_MAX + 1];
    for (int r = N - 1; r >= 0; --r) {
        double s = A[r][N];
        for (int k = r + 1; k < N; ++k) s -= A[r][k] * x[k];
        x[r] = s / A[r][r];
    }
    for (int i = 0; i < m; ++i) coef[i] = x[i];
}

struct FPtrs {
    const double* p[DIIS_MAX];
};

__global__ void diis_combine_kernel(size_t nn, int m, FPtrs F, const double* __restrict__ coef, double* __restrict__ out)
{
    const size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= nn) return;
    double s = 0.0;
    for (int k = 0; k < m; ++k) s += coef[k] * F.p[k][i];
    out[i] = s;
}

__global__ void real_to_complex_kernel(size_t n, const double* __restrict__ x, cuDoubleComplex* __restrict__ z)
{
    const size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) z[i] = make_cuDoubleComplex(x[i], 0.0);
}

// F = h + 2J - K + sum_d E_d M_d (complex Hermitian; J real)
__global__ void fock_complex_kernel(size_t nn, const double* __restrict__ h, const double* __restrict__ J,
                                    const cuDoubleComplex* __restrict__ K, const double* __restrict__ M, double ex,
                                    double ey, double ez, cuDoubleComplex* __restrict__ F)
{
    const size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= nn) return;
    const double v = h[i] + 2.0 * J[i] + ex * M[i] + ey * M[nn + i] + ez * M[2 * nn + i];
    F[i] = make_cuDoubleComplex(v - cuCreal(K[i]), -cuCimag(K[i]));
}

// Observables of a complex density P (AO): dipole_d = -2 Re Tr[M_d P] + nuc_d,
// Tr(PS), E = Re Tr[(h + F0) P] + Enuc with F0 = h + 2J - K.
__global__ void rt_obs_kernel(int n, const cuDoubleComplex* __restrict__ P, const double* __restrict__ M,
                              const double* __restrict__ S, const double* __restrict__ h, const double* __restrict__ J,
                              const cuDoubleComplex* __restrict__ K, double* __restrict__ out)
{
    __shared__ double red[5][256];
    double acc[5] = {0, 0, 0, 0, 0};
    const size_t nn = (size_t)n * n;
    for (size_t i = threadIdx.x; i < nn; i += blockDim.x) {
        const int r = (int)(i / n), c = (int)(i % n);
        const cuDoubleComplex pji = P[(size_t)c * n + r];
        const double pr = cuCreal(pji), pim = cuCimag(pji);
        for (int d = 0; d < 3; ++d) acc[d] += M[d * nn + i] * pr;
        acc[3] += S[i] * pr;
        const double fr = 2.0 * h[i] + 2.0 * J[i] - cuCreal(K[i]);
        const double fi = -cuCimag(K[i]);
        acc[4] += fr * pr - fi * pim;
    }
    for (int k = 0; k < 5; ++k) red[k][threadIdx.x] = acc[k];
    __syncthreads();
    for (int o = blockDim.x / 2; o > 0; o >>= 1) {
        if ((int)threadIdx.x < o)
            for (int k = 0; k < 5; ++k) red[k][threadIdx.x] += red[k][threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x == 0)
        for (int k = 0; k < 5; ++k) out[k] = red[k][0];
}

__global__ void identity_kernel(int n, cuDoubleComplex* __restrict__ I)
{
    const size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= (size_t)n * n) return;
    I[i] = make_cuDoubleComplex((i / n) == (i % n) ? 1.0 : 0.0, 0.0);
}

// max over columns of sum_r |A_rc| (1-norm), one block
__global__ void norm1_kernel(int n, const cuDoubleComplex* __restrict__ A, double* __restrict__ out)
{
    __shared__ double red[256];
    double m = 0.0;
    for (int c = threadIdx.x; c < n; c += blockDim.x) {
        double s = 0.0;
        for (int r = 0; r < n; ++r) s += cuCabs(A[(size_t)r * n + c]);
        m = fmax(m, s);
    }
    red[threadIdx.x] = m;
    __syncthreads();
    for (int o = blockDim.x / 2; o > 0; o >>= 1) {
        if ((int)threadIdx.x < o) red[threadIdx.x] = fmax(red[threadIdx.x], red[threadIdx.x + o]);
        __syncthreads();
    }
    if (threadIdx.x == 0) *out = red[0];
}

__global__ void zaxpby_kernel(size_t n, double a, const cuDoubleComplex* __restrict__ x, double b,
                              const cuDoubleComplex* __restrict__ y, cuDoubleComplex* __restrict__ z)
{
    const size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) z[i] = make_cuDoubleComplex(a * cuCreal(x[i]) + b * cuCreal(y[i]), a * cuCimag(x[i]) + b * cuCimag(y[i]));
}

static int nblk(size_t n) { return (int)((n + 255) / 256); }

// ------------------------------------------------------------------ set-up
int ensure_dense(cq_basis* b, cudaStream_t s)
{
    if (b->dense_ready) return CQ_OK;
    const int n = b->nbf;
    const size_t nn = (size_t)n * n;
    if (!b->blas) {
        cublasHandle_t h;
        CQ_BLAS(cublasCreate(&h));
        b->blas = h;
    }
    if (!b->solver) {
        cusolverDnHandle_t h;
        CQ_SOLVER(cusolverDnCreate(&h));
        b->solver = h;
    }
    cublasHandle_t blas = (cublasHandle_t)b->blas;
    cusolverDnHandle_t sol = (cusolverDnHandle_t)b->solver;
    CQ_BLAS(cublasSetStream(blas, s));
    CQ_SOLVER(cusolverDnSetStream(sol, s));
    int rc;
    double *T = nullptr, *V = nullptr, *Vec = nullptr, *Y = nullptr;
    if ((rc = scratch(b, &b->d_S, nn)) || (rc = scratch(b, &b->d_H, nn)) || (rc = scratch(b, &b->d_M, 3 * nn)) ||
        (rc = scratch(b, &T, nn)) || (rc = scratch(b, &V, nn)) || (rc = scratch(b, &Vec, nn)) ||
        (rc = scratch(b, &Y, nn)) || (rc = scratch(b, &b->d_w, n)) || (rc = scratch(b, &b->d_info, 1)))
        return rc;
    rc = cq_one_electron(b, b->d_S, T, V, b->d_M, nullptr, s);
    if (rc) return rc;
    add_kernel<<<nblk(nn), 256, 0, s>>>(nn, 1.0, T, 1.0, V, b->d_H);
    rc = cq_nuclear_repulsion(b, &b->enuc);
    if (rc) return rc;
    // eigenpairs of S
    CQ_CUDA(cudaMemcpyAsync(Vec, b->d_S, nn * sizeof(double), cudaMemcpyDeviceToDevice, s));
    int lw = 0;
    CQ_SOLVER(cusolverDnDsyevd_bufferSize(sol, CUSOLVER_EIG_MODE_VECTOR, CUBLAS_FILL_MODE_LOWER, n, Vec, n, b->d_w, &lw));
    lw = lw < 1 ? 1 : lw;
    // the same workspace serves the Fock eigenproblems (size <= n)
    if ((rc = scratch(b, &b->d_work, (size_t)lw))) return rc;
    b->lwork = lw;
    CQ_SOLVER(cusolverDnDsyevd(sol, CUSOLVER_EIG_MODE_VECTOR, CUBLAS_FILL_MODE_LOWER, n, Vec, n, b->d_w, b->d_work,
                               b->lwork, b->d_info));
    std::vector<double> w(n);
    int info = 0;
    CQ_CUDA(cudaMemcpyAsync(w.data(), b->d_w, n * sizeof(double), cudaMemcpyDeviceToHost, s));
    CQ_CUDA(cudaMemcpyAsync(&info, b->d_info, sizeof(int), cudaMemcpyDeviceToHost, s));
    CQ_CUDA(cudaStreamSynchronize(s));
    if (info != 0) { set_error("overlap eigensolver failed"); return CQ_ERR_NUMERIC; }
    int k0 = 0;
    while (k0 < n && w[k0] < 1e-8) ++k0;
    if (k0 == n) { set_error("overlap matrix has no eigenvalue above 1e-8"); return CQ_ERR_NUMERIC; }
    b->ndropped = k0;
    b->northo = n - k0;
    const int m = b->northo;
    if ((rc = scratch(b, &b->d_X, (size_t)n * m)) || (rc = scratch(b, &b->d_Xinv, (size_t)m * n))) return rc;
    ortho_y_kernel<<<nblk((size_t)n * m), 256, 0, s>>>(n, m, k0, Vec, b->d_w, k0 == 0 ? Y : b->d_X);
    if (k0 == 0)   // Loewdin: X = Y V^T, rows of Vec are the eigenvectors
        CQ_BLAS(dgemm_rm(blas, false, false, n, n, n, 1.0, Y, n, Vec, n, 0.0, b->d_X, n));
    // Xinv = X^T S  (so that X^T S X = 1 and P' = Xinv P Xinv^T)
    CQ_BLAS(dgemm_rm(blas, true, false, m, n, n, 1.0, b->d_X, m, b->d_S, n, 0.0, b->d_Xinv, n));
    CQ_CUDA(cudaGetLastError());
    b->dense_ready = 1;
    return CQ_OK;
}

}  // namespace cq

using namespace cq;

// ------------------------------------------------------------------ SCF
extern "C" int cq_scf(cq_basis* b, int nocc, const cq_scf_opts* opts, const double* D_in, double* D_out,
                      double* F_out, cq_scf_stats* stats, void* stream)
{
    if (!b || !D_out) { set_error("cq_scf: NULL basis or output"); return CQ_ERR_INVALID_ARG; }
    cq_scf_opts o{1e-10, 1e-8, 128, 8, CQ_PREC_FP64, 1e-5, 1e-14, 0, 8, 1e-5, 0, 0, 0.0};
    if (opts) o = *opts;
    const int n = b->nbf;
    if (b->nmol > 1) { set_error("cq_scf: batched basis; use cq_scf_batch"); return CQ_ERR_UNSUPPORTED; }
    if (nocc <= 0 || nocc > n) { set_error("cq_scf: nocc out of range"); return CQ_ERR_INVALID_ARG; }
    if (o.max_iter <= 0 || o.diis_size < 1 || o.diis_size > DIIS_MAX) {
        set_error("cq_scf: max_iter must be > 0 and diis_size in 1..8");
        return CQ_ERR_INVALID_ARG;
    }
    cudaStream_t s = (cudaStream_t)stream;
    int rc = ensure_dense(b, s);
    if (rc) return rc;
    const int m = b->northo;
    if (nocc > m) { set_error("cq_scf: more occupied orbitals than independent functions"); return CQ_ERR_INVALID_ARG; }
    cublasHandle_t blas = (cublasHandle_t)b->blas;
    cusolverDnHandle_t sol = (cusolverDnHandle_t)b->solver;
    CQ_BLAS(cublasSetStream(blas, s));
    CQ_SOLVER(cusolverDnSetStream(sol, s));
    const size_t nn = (size_t)n * n, mm = (size_t)m * m;
    // scratch (per call; the SCF is not on the per-iteration hot path of allocation)
    std::vector<void*> bufs;
    auto get = [&](double** p, size_t cnt) -> int {
        int r = dalloc(p, cnt);
        if (!r) bufs.push_back(*p);
        return r;
    };
    double *D, *Dold, *dD, *J, *K, *G, *F, *T1, *T2, *Err, *Ep, *Fd, *Fp, *C, *Bm, *coef, *scal;
    double *Fs[DIIS_MAX], *Es[DIIS_MAX];
    int* slots = nullptr;
    auto cleanup = [&]() {
        for (void* p : bufs) cudaFree(p);
        if (slots) cudaFree(slots);
    };
#define GET(p, c)                       \
    if ((rc = get(&(p), (c)))) {        \
        cleanup();                      \
        return rc;                      \
    }
    GET(D, nn) GET(Dold, nn) GET(dD, nn) GET(J, nn) GET(K, nn) GET(G, nn) GET(F, nn) GET(T1, nn) GET(T2, nn)
    GET(Err, nn) GET(Ep, mm) GET(Fd, nn) GET(Fp, mm) GET(C, (size_t)n * nocc) GET(Bm, DIIS_MAX * DIIS_MAX)
    GET(coef, DIIS_MAX) GET(scal, 4)
    for (int k = 0; k < o.diis_size; ++k) { GET(Fs[k], nn) GET(Es[k], mm) }
#undef GET
    if (cudaMalloc(&slots, DIIS_MAX * sizeof(int)) != cudaSuccess) { cleanup(); set_error("cq_scf: OOM"); return CQ_ERR_OOM; }

    auto density_from = [&](const double* Fm) -> int {
        // Fp = X^T F X ; eigh ; C = X V_occ ; D = C C^T
        CQ_BLAS(dgemm_rm(blas, true, false, m, n, n, 1.0, b->d_X, m, Fm, n, 0.0, T1, n));
        CQ_BLAS(dgemm_rm(blas, false, false, m, m, n, 1.0, T1, n, b->d_X, m, 0.0, Fp, m));
        CQ_SOLVER(cusolverDnDsyevd(sol, CUSOLVER_EIG_MODE_VECTOR, CUBLAS_FILL_MODE_LOWER, m, Fp, m, b->d_w, b->d_work,
                                   b->lwork, b->d_info));
        // rows of Fp are eigenvectors (ascending): C = X (Fp[0:nocc,:])^T
        CQ_BLAS(dgemm_rm(blas, false, true, n, nocc, m, 1.0, b->d_X, m, Fp, m, 0.0, C, nocc));
        CQ_BLAS(dgemm_rm(blas, false, true, n, n, nocc, 1.0, C, nocc, C, nocc, 0.0, D, n));
        return CQ_OK;
    };
    CQ_CUDA(cudaMemsetAsync(G, 0, nn * sizeof(double), s));
    CQ_CUDA(cudaMemsetAsync(Dold, 0, nn * sizeof(double), s));
    if (D_in) {
        CQ_CUDA(cudaMemcpyAsync(D, D_in, nn * sizeof(double), cudaMemcpyDeviceToDevice, s));
    } else if ((rc = density_from(b->d_H))) {
        cleanup();
        return rc;
    }
    cq_scf_stats st;
    memset(&st, 0, sizeof st);
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    cudaEventRecord(e0, s);
    double Eold = 0.0, E = 0.0, rms = 0.0;
    int nvec = 0, head = 0, since_full = 0;
    bool final_fp64 = (o.prec == CQ_PREC_FP64);
    bool converged = false;
    int it = 0;
    for (it = 1; it <= o.max_iter; ++it) {
        const bool incremental = o.incremental && since_full > 0 && since_full < o.full_every;
        cq_fock_opts fo{o.schwarz_tol, o.mixed_tol, final_fp64 ? CQ_PREC_FP64 : CQ_PREC_MIXED, 1, 1, o.fp64_tol};
        cq_fock_stats fst;
        const double* Dbuild = D;
        if (incremental) {
            add_kernel<<<nblk(nn), 256, 0, s>>>(nn, 1.0, D, -1.0, Dold, dD);
            Dbuild = dD;
        }
        rc = cq_fock_build(b, CQ_DENS_REAL_SYM, Dbuild, J, K, &fo, &fst, s);
        if (rc) { cleanup(); return rc; }
        st.quartets_fp64 += fst.quartets_fp64;
        st.quartets_fp32 += fst.quartets_fp32;
        st.quartets_df += fst.quartets_df;
        since_full = incremental ? since_full + 1 : 1;
        fock_real_kernel<<<nblk(nn), 256, 0, s>>>(nn, incremental ? 1 : 0, b->d_H, J, K, G, F);
        rhf_energy_kernel<<<1, 256, 0, s>>>(nn, b->d_H, F, D, b->enuc, scal);
        // DIIS error X^T (F D S - S D F) X
        CQ_BLAS(dgemm_rm(blas, false, false, n, n, n, 1.0, F, n, D, n, 0.0, T1, n));
        CQ_BLAS(dgemm_rm(blas, false, false, n, n, n, 1.0, T1, n, b->d_S, n, 0.0, T2, n));
        antisym_kernel<<<nblk(nn), 256, 0, s>>>(n, T2, Err);
        CQ_BLAS(dgemm_rm(blas, true, false, m, n, n, 1.0, b->d_X, m, Err, n, 0.0, T1, n));
        CQ_BLAS(dgemm_rm(blas, false, false, m, m, n, 1.0, T1, n, b->d_X, m, 0.0, Ep, m));
        dot_kernel<<<1, 256, 0, s>>>(mm, Ep, nullptr, 0.0, 1.0 / (double)mm, 1, scal + 1);
        double hv[2];
        CQ_CUDA(cudaMemcpyAsync(hv, scal, 2 * sizeof(double), cudaMemcpyDeviceToHost, s));
        CQ_CUDA(cudaStreamSynchronize(s));
        E = hv[0];
        rms = hv[1];
        if (!std::isfinite(E) || !std::isfinite(rms)) {
            cleanup();
            set_error("cq_scf: non-finite energy or error norm");
            return CQ_ERR_NUMERIC;
        }
        const double dE = std::fabs(E - Eold);
        Eold = E;
        if (it > 1 && dE < o.e_tol && rms < o.d_tol && final_fp64 && !incremental) {
            converged = true;
            break;
        }
        if (!final_fp64 && rms < o.switch_tol) {   // final iterations in full FP64
            final_fp64 = true;
            since_full = 0;
        }
        if (it > 1 && dE < o.e_tol && rms < o.d_tol && incremental) since_full = 0;   // confirm with a full build
        // DIIS push
        const int slot = head;
        head = (head + 1) % o.diis_size;
        nvec = nvec < o.diis_size ? nvec + 1 : nvec;
        CQ_CUDA(cudaMemcpyAsync(Fs[slot], F, nn * sizeof(double), cudaMemcpyDeviceToDevice, s));
        CQ_CUDA(cudaMemcpyAsync(Es[slot], Ep, mm * sizeof(double), cudaMemcpyDeviceToDevice, s));
        int order[DIIS_MAX];
        for (int k = 0; k < nvec; ++k) order[k] = (head - nvec + k + o.diis_size) % o.diis_size;
        for (int k = 0; k < nvec; ++k)
            dot_kernel<<<1, 256, 0, s>>>(mm, Es[slot], Es[order[k]], 0.0, 1.0, 0, Bm + slot * DIIS_MAX + order[k]);
        for (int k = 0; k < nvec; ++k)
            dot_kernel<<<1, 256, 0, s>>>(mm, Es[order[k]], Es[slot], 0.0, 1.0, 0, Bm + order[k] * DIIS_MAX + slot);
        const double* Fuse = F;
        if (nvec >= 2) {
            CQ_CUDA(cudaMemcpyAsync(slots, order, nvec * sizeof(int), cudaMemcpyHostToDevice, s));
            diis_solve_kernel<<<1, 32, 0, s>>>(nvec, Bm, slots, coef);
            FPtrs fp;
            for (int k = 0; k < nvec; ++k) fp.p[k] = Fs[order[k]];
            diis_combine_kernel<<<nblk(nn), 256, 0, s>>>(nn, nvec, fp, coef, Fd);
            Fuse = Fd;
        }
        CQ_CUDA(cudaMemcpyAsync(Dold, D, nn * sizeof(double), cudaMemcpyDeviceToDevice, s));
        if ((rc = density_from(Fuse))) { cleanup(); return rc; }
        CQ_CUDA(cudaGetLastError());
    }
    cudaEventRecord(e1, s);
    CQ_CUDA(cudaMemcpyAsync(D_out, D, nn * sizeof(double), cudaMemcpyDeviceToDevice, s));
    if (F_out) CQ_CUDA(cudaMemcpyAsync(F_out, F, nn * sizeof(double), cudaMemcpyDeviceToDevice, s));
    CQ_CUDA(cudaStreamSynchronize(s));
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cleanup();
    st.energy = E;
    st.iterations = converged ? it : o.max_iter;
    st.converged = converged ? 1 : 0;
    st.last_rms = rms;
    st.ms = ms;
    if (stats) *stats = st;
    if (!converged) {
        set_error("cq_scf: not converged within max_iter");
        return CQ_ERR_NOT_CONVERGED;
    }
    return CQ_OK;
}

// ------------------------------------------------------------------ RT-TDHF
namespace cq {

struct RTBufs {
    int n = 0, m = 0;
    cuDoubleComplex *Xc, *Xic, *Ppc, *Ppp, *Pao, *Fao, *Fp, *Fp2, *U, *W1, *W2, *Id;
    double *J, *obs, *nrm;
    cuDoubleComplex* K;
};

static int rt_bufs(cq_basis* b, RTBufs& r, cudaStream_t s)
{
    // allocated once per basis and kept in dense_bufs (freed with the basis)
    static_assert(sizeof(cuDoubleComplex) == 16, "complex layout");
    const int n = b->nbf, m = b->northo;
    const size_t nm = (size_t)n * m, mm = (size_t)m * m, nn = (size_t)n * n;
    int rc;
    if ((rc = scratch(b, &r.Xc, nm)) || (rc = scratch(b, &r.Xic, nm)) || (rc = scratch(b, &r.Ppc, mm)) ||
        (rc = scratch(b, &r.Ppp, mm)) || (rc = scratch(b, &r.Pao, nn)) || (rc = scratch(b, &r.Fao, nn)) ||
        (rc = scratch(b, &r.Fp, mm)) || (rc = scratch(b, &r.Fp2, mm)) || (rc = scratch(b, &r.U, mm)) ||
        (rc = scratch(b, &r.W1, (nn > mm ? nn : mm))) || (rc = scratch(b, &r.W2, (nn > mm ? nn : mm))) ||
        (rc = scratch(b, &r.Id, mm)) || (rc = scratch(b, &r.J, nn)) || (rc = scratch(b, &r.K, nn)) ||
        (rc = scratch(b, &r.obs, 8)) || (rc = scratch(b, &r.nrm, 2)))
        return rc;
    real_to_complex_kernel<<<nblk(nm), 256, 0, s>>>(nm, b->d_X, r.Xc);
    real_to_complex_kernel<<<nblk(nm), 256, 0, s>>>(nm, b->d_Xinv, r.Xic);
    identity_kernel<<<nblk(mm), 256, 0, s>>>(m, r.Id);
    r.n = n;
    r.m = m;
    CQ_CUDA(cudaGetLastError());
    return CQ_OK;
}

static RTBufs* rt_state(cq_basis* b, cudaStream_t s, int* rc)
{
    // one RT buffer set per basis, created on first use, freed with the basis
    if (b->rt) return (RTBufs*)b->rt;
    RTBufs* r = new RTBufs();
    *rc = rt_bufs(b, *r, s);
    if (*rc) { delete r; return nullptr; }
    b->rt = r;
    return r;
}

void dense_free(cq_basis* b)
{
    for (void* p : b->dense_bufs) cudaFree(p);
    b->dense_bufs.clear();
    if (b->blas) cublasDestroy((cublasHandle_t)b->blas);
    if (b->solver) cusolverDnDestroy((cusolverDnHandle_t)b->solver);
    b->blas = b->solver = nullptr;
    delete (RTBufs*)b->rt;
    b->rt = nullptr;
}

// P'(m x m) = Xinv P Xinv^T ; P (n x n)
static int to_ortho(cq_basis* b, RTBufs& r, const cuDoubleComplex* P, cuDoubleComplex* Pp)
{
    cublasHandle_t h = (cublasHandle_t)b->blas;
    const cuDoubleComplex one = make_cuDoubleComplex(1, 0), zero = make_cuDoubleComplex(0, 0);
    CQ_BLAS(zgemm_rm(h, 'N', 'N', r.m, r.n, r.n, one, r.Xic, r.n, P, r.n, zero, r.W1, r.n));
    CQ_BLAS(zgemm_rm(h, 'N', 'T', r.m, r.m, r.n, one, r.W1, r.n, r.Xic, r.n, zero, Pp, r.m));
    return CQ_OK;
}

// P (n x n) = X P' X^T
static int to_ao(cq_basis* b, RTBufs& r, const cuDoubleComplex* Pp, cuDoubleComplex* P)
{
    cublasHandle_t h = (cublasHandle_t)b->blas;
    const cuDoubleComplex one = make_cuDoubleComplex(1, 0), zero = make_cuDoubleComplex(0, 0);
    CQ_BLAS(zgemm_rm(h, 'N', 'N', r.n, r.m, r.m, one, r.Xc, r.m, Pp, r.m, zero, r.W1, r.m));
    CQ_BLAS(zgemm_rm(h, 'N', 'T', r.n, r.n, r.m, one, r.W1, r.m, r.Xc, r.m, zero, P, r.n));
    return CQ_OK;
}

// F'(t) of an orthonormal-basis density; with obs != NULL also the
// observables of that density (dipole x3, Tr PS, field-free energy).
static int fock_ortho(cq_basis* b, RTBufs& r, const cq_rt_opts& o, const cuDoubleComplex* Pp, double t,
                      cuDoubleComplex* Fp, double* obs, cudaStream_t s)
{
    int rc = to_ao(b, r, Pp, r.Pao);
    if (rc) return rc;
    cq_fock_opts fo{o.schwarz_tol, o.mixed_tol, o.prec, 1, 1, o.fp64_tol};
    rc = cq_fock_build(b, CQ_DENS_COMPLEX_HERM, r.Pao, r.J, r.K, &fo, nullptr, s);
    if (rc) return rc;
    const bool on = t >= o.t_on && t < o.t_off;
    const size_t nn = (size_t)r.n * r.n;
    fock_complex_kernel<<<nblk(nn), 256, 0, s>>>(nn, b->d_H, r.J, r.K, b->d_M, on ? o.field[0] : 0.0,
                                                 on ? o.field[1] : 0.0, on ? o.field[2] : 0.0, r.Fao);
    if (obs) rt_obs_kernel<<<1, 256, 0, s>>>(r.n, r.Pao, b->d_M, b->d_S, b->d_H, r.J, r.K, obs);
    cublasHandle_t h = (cublasHandle_t)b->blas;
    const cuDoubleComplex one = make_cuDoubleComplex(1, 0), zero = make_cuDoubleComplex(0, 0);
    CQ_BLAS(zgemm_rm(h, 'T', 'N', r.m, r.n, r.n, one, r.Xc, r.m, r.Fao, r.n, zero, r.W1, r.n));
    CQ_BLAS(zgemm_rm(h, 'N', 'N', r.m, r.m, r.n, one, r.W1, r.n, r.Xc, r.m, zero, Fp, r.m));
    CQ_CUDA(cudaGetLastError());
    return CQ_OK;
}

// U = exp(-i a F') by a Taylor series of degree 18 on A / 2^s (||A/2^s||_1
// <= 1/2) in Horner form, followed by s squarings (GEMMs only).
static int expm_i(cq_basis* b, RTBufs& r, const cuDoubleComplex* Fp, double a, cuDoubleComplex* U, cudaStream_t s)
{
    const int m = r.m;
    const size_t mm = (size_t)m * m;
    norm1_kernel<<<1, 256, 0, s>>>(m, Fp, r.nrm);
    double nrm = 0.0;
    CQ_CUDA(cudaMemcpyAsync(&nrm, r.nrm, sizeof(double), cudaMemcpyDeviceToHost, s));
    CQ_CUDA(cudaStreamSynchronize(s));
    nrm *= std::fabs(a);
    int sq = 0;
    while (nrm > 0.5 && sq < 60) { nrm *= 0.5; ++sq; }
    const double sc = a / std::ldexp(1.0, sq);
    cublasHandle_t h = (cublasHandle_t)b->blas;
    const int deg = 18;
    // T = I + (B/deg), B = -i sc F'
    cuDoubleComplex* T = r.W1;
    cuDoubleComplex* T2 = r.W2;
    CQ_CUDA(cudaMemcpyAsync(T, r.Id, mm * sizeof(cuDoubleComplex), cudaMemcpyDeviceToDevice, s));
    for (int k = deg; k >= 1; --k) {
        // T2 = I + (B/k) T
        CQ_CUDA(cudaMemcpyAsync(T2, r.Id, mm * sizeof(cuDoubleComplex), cudaMemcpyDeviceToDevice, s));
        const cuDoubleComplex alpha = make_cuDoubleComplex(0.0, -sc / k);
        CQ_BLAS(zgemm_rm(h, 'N', 'N', m, m, m, alpha, Fp, m, T, m, make_cuDoubleComplex(1, 0), T2, m));
        cuDoubleComplex* tmp = T; T = T2; T2 = tmp;
    }
    for (int k = 0; k < sq; ++k) {
        CQ_BLAS(zgemm_rm(h, 'N', 'N', m, m, m, make_cuDoubleComplex(1, 0), T, m, T, m, make_cuDoubleComplex(0, 0), T2, m));
        cuDoubleComplex* tmp = T; T = T2; T2 = tmp;
    }
    CQ_CUDA(cudaMemcpyAsync(U, T, mm * sizeof(cuDoubleComplex), cudaMemcpyDeviceToDevice, s));
    return CQ_OK;
}

// Pout = U P U^H
static int conjugate(cq_basis* b, RTBufs& r, const cuDoubleComplex* U, const cuDoubleComplex* P, cuDoubleComplex* Pout)
{
    cublasHandle_t h = (cublasHandle_t)b->blas;
    const cuDoubleComplex one = make_cuDoubleComplex(1, 0), zero = make_cuDoubleComplex(0, 0);
    CQ_BLAS(zgemm_rm(h, 'N', 'N', r.m, r.m, r.m, one, U, r.m, P, r.m, zero, r.W2, r.m));
    CQ_BLAS(zgemm_rm(h, 'N', 'C', r.m, r.m, r.m, one, r.W2, r.m, U, r.m, zero, Pout, r.m));
    return CQ_OK;
}

}  // namespace cq

extern "C" int cq_rt_step(cq_basis* b, const cq_rt_opts* opts, int step, void* P_prev, void* P_cur, cq_rt_obs* obs,
                          void* stream)
{
    if (!b || !opts || !P_cur || (!P_prev && step > 0)) {
        set_error("cq_rt_step: NULL argument");
        return CQ_ERR_INVALID_ARG;
    }
    const cq_rt_opts o = *opts;
    if (b->nmol > 1) { set_error("cq_rt_step: batched basis not supported"); return CQ_ERR_UNSUPPORTED; }
    if (!(o.dt > 0.0) || step < 0) { set_error("cq_rt_step: dt must be > 0 and step >= 0"); return CQ_ERR_INVALID_ARG; }
    cudaStream_t s = (cudaStream_t)stream;
    int rc = ensure_dense(b, s);
    if (rc) return rc;
    CQ_BLAS(cublasSetStream((cublasHandle_t)b->blas, s));
    RTBufs* r = rt_state(b, s, &rc);
    if (!r) return rc;
    const double t = step * o.dt;
    const bool em2 = step == 0 || !P_prev || (o.restart_every > 0 && step % o.restart_every == 0);
    cuDoubleComplex* Pc = (cuDoubleComplex*)P_cur;
    cuDoubleComplex* Pv = (cuDoubleComplex*)P_prev;
    if ((rc = to_ortho(b, *r, Pc, r->Ppc))) return rc;
    if ((rc = fock_ortho(b, *r, o, r->Ppc, t, r->Fp, obs ? r->obs : nullptr, s))) return rc;
    const size_t mm = (size_t)r->m * r->m, nn = (size_t)r->n * r->n;
    if (em2) {
        // P_FE = U_FE P_k U_FE^H, U_FE = exp(-i dt F_k); F_m = (F_k + F(P_FE, t+dt))/2
        if ((rc = expm_i(b, *r, r->Fp, o.dt, r->U, s))) return rc;
        if ((rc = conjugate(b, *r, r->U, r->Ppc, r->Ppp))) return rc;
        if ((rc = fock_ortho(b, *r, o, r->Ppp, t + o.dt, r->Fp2, nullptr, s))) return rc;
        zaxpby_kernel<<<nblk(mm), 256, 0, s>>>(mm, 0.5, r->Fp, 0.5, r->Fp2, r->Fp);
        if ((rc = expm_i(b, *r, r->Fp, o.dt, r->U, s))) return rc;
        if ((rc = conjugate(b, *r, r->U, r->Ppc, r->Ppp))) return rc;
    } else {
        // MMUT: P_{k+1} = U P_{k-1} U^H, U = exp(-2 i dt F_k)
        if ((rc = expm_i(b, *r, r->Fp, 2.0 * o.dt, r->U, s))) return rc;
        if ((rc = to_ortho(b, *r, Pv, r->Fp2))) return rc;
        if ((rc = conjugate(b, *r, r->U, r->Fp2, r->Ppp))) return rc;
    }
    // P_prev <- P_cur ; P_cur <- P_{k+1} (AO)
    if (P_prev) CQ_CUDA(cudaMemcpyAsync(P_prev, P_cur, nn * sizeof(cuDoubleComplex), cudaMemcpyDeviceToDevice, s));
    if ((rc = to_ao(b, *r, r->Ppp, Pc))) return rc;
    CQ_CUDA(cudaGetLastError());
    if (obs) {
        double h[5];
        CQ_CUDA(cudaMemcpyAsync(h, r->obs, sizeof h, cudaMemcpyDeviceToHost, s));
        CQ_CUDA(cudaStreamSynchronize(s));
        double nuc[3] = {0, 0, 0};
        for (int A = 0; A < b->natom; ++A)
            for (int d = 0; d < 3; ++d) nuc[d] += b->Z[A] * b->xyz[3 * A + d];
        for (int d = 0; d < 3; ++d) obs->dipole[d] = -2.0 * h[d] + nuc[d];
        obs->trPS = h[3];
        obs->energy = h[4] + b->enuc;
        obs->em2 = em2 ? 1 : 0;
    }
    return CQ_OK;
}

extern "C" int cq_dense_info(cq_basis* b, int* northo, int* ndropped, void* stream)
{
    if (!b) { set_error("cq_dense_info: NULL basis"); return CQ_ERR_INVALID_ARG; }
    int rc = ensure_dense(b, (cudaStream_t)stream);
    if (rc) return rc;
    if (northo) *northo = b->northo;
    if (ndropped) *ndropped = b->ndropped;
    return CQ_OK;
}

// ------------------------------------------------------------------ GHF SCF
// Two-component SCF in the Pauli representation (Eq. pauli_sep, Eq.
// 2c_fock): densities P^I (I = 0..3, complex n x n), F^0 = h + 2J[P^0] -
// K[P^0], F^k = -K[P^k]; the 2n x 2n Fock matrix sum_I sigma_I (x) F^I is
// diagonalised in the orthonormal basis diag(X, X), the nelec lowest spinors
// give P^{2C} = C C^+, split back into its Pauli components.  Energy
// E = sum_I Re Tr[(h^I + F^I) P^I] + E_nuc (h^k = 0).  DIIS on the
// orthogonal-basis commutator with real B_ij = Re <e_i|e_j>.
namespace cq {

__global__ void ghf_fock_kernel(size_t nn, const double* __restrict__ h, const double* __restrict__ J,
                                const cuDoubleComplex* __restrict__ K, cuDoubleComplex* __restrict__ F)
{
    const size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= nn) return;
    F[i] = make_cuDoubleComplex(h[i] + 2.0 * J[i] - K[i].x, -K[i].y);
    for (int k = 1; k < 4; ++k) F[k * nn + i] = make_cuDoubleComplex(-K[k * nn + i].x, -K[k * nn + i].y);
}

// out = F with h added to the scalar component (the energy's h^I + F^I)
__global__ void ghf_hf_kernel(size_t nn, const double* __restrict__ h, const cuDoubleComplex* __restrict__ F,
                              cuDoubleComplex* __restrict__ out)
{
    const size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= 4 * nn) return;
    cuDoubleComplex v = F[i];
    if (i < nn) v.x += h[i];
    out[i] = v;
}

// Y (2n x 2n) = sum_I sigma_I (x) X^I
__global__ void pauli_join_kernel(int n, const cuDoubleComplex* __restrict__ X, cuDoubleComplex* __restrict__ Y)
{
    const size_t nn = (size_t)n * n;
    const size_t t = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= nn) return;
    const int i = (int)(t / n), j = (int)(t % n);
    const cuDoubleComplex x0 = X[t], x1 = X[nn + t], x2 = X[2 * nn + t], x3 = X[3 * nn + t];
    const size_t N = 2 * (size_t)n;
    Y[i * N + j] = make_cuDoubleComplex(x0.x + x3.x, x0.y + x3.y);
    Y[(n + i) * N + n + j] = make_cuDoubleComplex(x0.x - x3.x, x0.y - x3.y);
    Y[i * N + n + j] = make_cuDoubleComplex(x1.x + x2.y, x1.y - x2.x);         // x1 - i x2
    Y[(n + i) * N + j] = make_cuDoubleComplex(x1.x - x2.y, x1.y + x2.x);       // x1 + i x2
}

// X^0 = (aa + bb)/2, X^1 = (ab + ba)/2, X^2 = i (ab - ba)/2, X^3 = (aa - bb)/2
__global__ void pauli_split_kernel(int n, const cuDoubleComplex* __restrict__ Y, cuDoubleComplex* __restrict__ X)
{
    const size_t nn = (size_t)n * n;
    const size_t t = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= nn) return;
    const int i = (int)(t / n), j = (int)(t % n);
    const size_t N = 2 * (size_t)n;
    const cuDoubleComplex aa = Y[i * N + j], bb = Y[(n + i) * N + n + j];
    const cuDoubleComplex ab = Y[i * N + n + j], ba = Y[(n + i) * N + j];
    X[t] = make_cuDoubleComplex(0.5 * (aa.x + bb.x), 0.5 * (aa.y + bb.y));
    X[nn + t] = make_cuDoubleComplex(0.5 * (ab.x + ba.x), 0.5 * (ab.y + ba.y));
    X[2 * nn + t] = make_cuDoubleComplex(-0.5 * (ab.y - ba.y), 0.5 * (ab.x - ba.x));
    X[3 * nn + t] = make_cuDoubleComplex(0.5 * (aa.x - bb.x), 0.5 * (aa.y - bb.y));
}

// X2 (2n x 2m) = diag(X, X), X real n x m
__global__ void block_diag_kernel(int n, int m, const double* __restrict__ X, cuDoubleComplex* __restrict__ X2)
{
    const size_t t = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= (size_t)4 * n * m) return;
    const int r = (int)(t / (2 * m)), c = (int)(t % (2 * m));
    const bool same = (r < n) == (c < m);
    X2[t] = make_cuDoubleComplex(same ? X[(size_t)(r % n) * m + (c % m)] : 0.0, 0.0);
}

// E = T - T^+
__global__ void antiherm_kernel(int N, const cuDoubleComplex* __restrict__ T, cuDoubleComplex* __restrict__ E)
{
    const size_t t = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= (size_t)N * N) return;
    const int i = (int)(t / N), j = (int)(t % N);
    const cuDoubleComplex a = T[t], b = T[(size_t)j * N + i];
    E[t] = make_cuDoubleComplex(a.x - b.x, a.y + b.y);
}

}  // namespace cq

extern "C" int cq_scf_ghf(cq_basis* b, int nelec, const cq_scf_opts* opts, const void* P_in, void* P_out,
                          void* F_out, cq_scf_stats* stats, void* stream)
{
    if (!b || !P_out) { set_error("cq_scf_ghf: NULL basis or output"); return CQ_ERR_INVALID_ARG; }
    cq_scf_opts o{1e-10, 1e-8, 128, 8, CQ_PREC_FP64, 1e-5, 1e-14, 0, 8, 1e-5, 0, 0, 0.0};
    if (opts) o = *opts;
    const int n = b->nbf;
    if (b->nmol > 1) { set_error("cq_scf_ghf: batched basis"); return CQ_ERR_UNSUPPORTED; }
    if (nelec <= 0 || nelec > 2 * n) { set_error("cq_scf_ghf: nelec out of range"); return CQ_ERR_INVALID_ARG; }
    if (o.max_iter <= 0 || o.diis_size < 1 || o.diis_size > DIIS_MAX) {
        set_error("cq_scf_ghf: max_iter must be > 0 and diis_size in 1..8");
        return CQ_ERR_INVALID_ARG;
    }
    if (o.prec != CQ_PREC_FP64 && o.prec != CQ_PREC_MIXED) {
        set_error("cq_scf_ghf: unknown precision mode");
        return CQ_ERR_INVALID_ARG;
    }
    cudaStream_t s = (cudaStream_t)stream;
    int rc = ensure_dense(b, s);
    if (rc) return rc;
    const int m = b->northo;
    if (nelec > 2 * m) { set_error("cq_scf_ghf: more electrons than spinors"); return CQ_ERR_INVALID_ARG; }
    cublasHandle_t blas = (cublasHandle_t)b->blas;
    cusolverDnHandle_t sol = (cusolverDnHandle_t)b->solver;
    CQ_BLAS(cublasSetStream(blas, s));
    CQ_SOLVER(cusolverDnSetStream(sol, s));
    const int N = 2 * n, M = 2 * m;
    const size_t nn = (size_t)n * n, NN = (size_t)N * N, MM = (size_t)M * M;
    using Z = cuDoubleComplex;
    std::vector<void*> bufs;
    auto get = [&](auto** p, size_t cnt) -> int {
        int r = dalloc(p, cnt);
        if (!r) bufs.push_back((void*)*p);
        return r;
    };
    Z *P, *P2, *F, *F2, *K, *X2, *S2, *T1, *T2, *Err, *Ep, *Fp, *C, *Fd, *HF, *work;
    Z *Fs[DIIS_MAX], *Es[DIIS_MAX];
    double *J, *w, *Bm, *coef, *scal;
    int *slots, *info;
    auto cleanup = [&]() {
        for (void* p : bufs) cudaFree(p);
    };
    int lwork = 0;
#define GETZ(p, c)                      \
    if ((rc = get(&(p), (c)))) {        \
        cleanup();                      \
        return rc;                      \
    }
    GETZ(P, 4 * nn) GETZ(P2, NN) GETZ(F, 4 * nn) GETZ(F2, NN) GETZ(K, 4 * nn) GETZ(X2, (size_t)N * M) GETZ(S2, NN)
    GETZ(T1, NN) GETZ(T2, NN) GETZ(Err, NN) GETZ(Ep, MM) GETZ(Fp, MM) GETZ(C, (size_t)N * nelec) GETZ(Fd, NN)
    GETZ(HF, 4 * nn) GETZ(J, nn) GETZ(w, M) GETZ(Bm, DIIS_MAX * DIIS_MAX) GETZ(coef, DIIS_MAX) GETZ(scal, 4)
    GETZ(slots, DIIS_MAX) GETZ(info, 1)
    for (int k = 0; k < o.diis_size; ++k) { GETZ(Fs[k], NN) GETZ(Es[k], MM) }
    if (cusolverDnZheevd_bufferSize(sol, CUSOLVER_EIG_MODE_VECTOR, CUBLAS_FILL_MODE_LOWER, M, Fp, M, w, &lwork) !=
        CUSOLVER_STATUS_SUCCESS) {
        cleanup();
        set_error("cusolverDnZheevd_bufferSize failed");
        return CQ_ERR_CUDA;
    }
    GETZ(work, (size_t)(lwork > 0 ? lwork : 1))
#undef GETZ
    const Z one = make_cuDoubleComplex(1.0, 0.0), zero = make_cuDoubleComplex(0.0, 0.0);
    block_diag_kernel<<<nblk((size_t)N * M), 256, 0, s>>>(n, m, b->d_X, X2);
    {   // S2 = diag(S, S) as a complex matrix: the Pauli join of (S, 0, 0, 0)
        CQ_CUDA(cudaMemsetAsync(HF, 0, 4 * nn * sizeof(Z), s));
        real_to_complex_kernel<<<nblk(nn), 256, 0, s>>>(nn, b->d_S, HF);
        pauli_join_kernel<<<nblk(nn), 256, 0, s>>>(n, HF, S2);
    }
    // P2 from a 2n x 2n Fock matrix: Fp = X2^+ F X2, eigh, C = X2 (rows 0..nelec-1 of Fp)^+, P2 = C C^+
    auto density_from = [&](const Z* Fm) -> int {
        CQ_BLAS(zgemm_rm(blas, 'C', 'N', M, N, N, one, X2, M, Fm, N, zero, T1, N));
        CQ_BLAS(zgemm_rm(blas, 'N', 'N', M, M, N, one, T1, N, X2, M, zero, Fp, M));
        CQ_SOLVER(cusolverDnZheevd(sol, CUSOLVER_EIG_MODE_VECTOR, CUBLAS_FILL_MODE_LOWER, M, Fp, M, w, work, lwork,
                                   info));
        CQ_BLAS(zgemm_rm(blas, 'N', 'C', N, nelec, M, one, X2, M, Fp, M, zero, C, nelec));
        CQ_BLAS(zgemm_rm(blas, 'N', 'C', N, N, nelec, one, C, nelec, C, nelec, zero, P2, N));
        pauli_split_kernel<<<nblk(nn), 256, 0, s>>>(n, P2, P);
        return CQ_OK;
    };
    if (P_in) {
        CQ_CUDA(cudaMemcpyAsync(P, P_in, 4 * nn * sizeof(Z), cudaMemcpyDeviceToDevice, s));
        pauli_join_kernel<<<nblk(nn), 256, 0, s>>>(n, P, P2);
    } else {   // core guess: diag(h, h)
        CQ_CUDA(cudaMemsetAsync(HF, 0, 4 * nn * sizeof(Z), s));
        real_to_complex_kernel<<<nblk(nn), 256, 0, s>>>(nn, b->d_H, HF);
        pauli_join_kernel<<<nblk(nn), 256, 0, s>>>(n, HF, F2);
        if ((rc = density_from(F2))) { cleanup(); return rc; }
    }
    cq_scf_stats st;
    memset(&st, 0, sizeof st);
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    cudaEventRecord(e0, s);
    double Eold = 0.0, E = 0.0, rms = 0.0;
    int nvec = 0, head = 0, it = 0;
    bool final_fp64 = (o.prec == CQ_PREC_FP64), converged = false;
    for (it = 1; it <= o.max_iter; ++it) {
        cq_fock_opts fo{o.schwarz_tol, o.mixed_tol, final_fp64 ? CQ_PREC_FP64 : CQ_PREC_MIXED, 1, 1, o.fp64_tol};
        cq_fock_stats fst;
        if ((rc = cq_fock_build(b, CQ_DENS_PAULI4, P, J, K, &fo, &fst, s))) { cleanup(); return rc; }
        st.quartets_fp64 += fst.quartets_fp64;
        st.quartets_fp32 += fst.quartets_fp32;
        st.quartets_df += fst.quartets_df;
        ghf_fock_kernel<<<nblk(nn), 256, 0, s>>>(nn, b->d_H, J, K, F);
        ghf_hf_kernel<<<nblk(4 * nn), 256, 0, s>>>(nn, b->d_H, F, HF);
        // Re sum (h^I + F^I)_ij conj(P^I_ij) = Re Tr[(h^I + F^I) P^I] for Hermitian P^I
        dot_kernel<<<1, 256, 0, s>>>(8 * nn, (const double*)HF, (const double*)P, b->enuc, 1.0, 0, scal);
        pauli_join_kernel<<<nblk(nn), 256, 0, s>>>(n, F, F2);
        // error X2^+ (F2 P2 S2 - S2 P2 F2) X2
        CQ_BLAS(zgemm_rm(blas, 'N', 'N', N, N, N, one, F2, N, P2, N, zero, T1, N));
        CQ_BLAS(zgemm_rm(blas, 'N', 'N', N, N, N, one, T1, N, S2, N, zero, T2, N));
        antiherm_kernel<<<nblk(NN), 256, 0, s>>>(N, T2, Err);
        CQ_BLAS(zgemm_rm(blas, 'C', 'N', M, N, N, one, X2, M, Err, N, zero, T1, N));
        CQ_BLAS(zgemm_rm(blas, 'N', 'N', M, M, N, one, T1, N, X2, M, zero, Ep, M));
        dot_kernel<<<1, 256, 0, s>>>(2 * MM, (const double*)Ep, nullptr, 0.0, 1.0 / (double)MM, 1, scal + 1);
        double hv[2];
        CQ_CUDA(cudaMemcpyAsync(hv, scal, 2 * sizeof(double), cudaMemcpyDeviceToHost, s));
        CQ_CUDA(cudaStreamSynchronize(s));
        E = hv[0];
        rms = hv[1];
        if (!std::isfinite(E) || !std::isfinite(rms)) {
            cleanup();
            set_error("cq_scf_ghf: non-finite energy or error norm");
            return CQ_ERR_NUMERIC;
        }
        const double dE = std::fabs(E - Eold);
        Eold = E;
        if (it > 1 && dE < o.e_tol && rms < o.d_tol && final_fp64) {
            converged = true;
            break;
        }
        if (!final_fp64 && rms < o.switch_tol) final_fp64 = true;
        const int slot = head;
        head = (head + 1) % o.diis_size;
        nvec = nvec < o.diis_size ? nvec + 1 : nvec;
        CQ_CUDA(cudaMemcpyAsync(Fs[slot], F2, NN * sizeof(Z), cudaMemcpyDeviceToDevice, s));
        CQ_CUDA(cudaMemcpyAsync(Es[slot], Ep, MM * sizeof(Z), cudaMemcpyDeviceToDevice, s));
        int order[DIIS_MAX];
        for (int k = 0; k < nvec; ++k) order[k] = (head - nvec + k + o.diis_size) % o.diis_size;
        for (int k = 0; k < nvec; ++k) {
            dot_kernel<<<1, 256, 0, s>>>(2 * MM, (const double*)Es[slot], (const double*)Es[order[k]], 0.0, 1.0, 0,
                                         Bm + slot * DIIS_MAX + order[k]);
            dot_kernel<<<1, 256, 0, s>>>(2 * MM, (const double*)Es[order[k]], (const double*)Es[slot], 0.0, 1.0, 0,
                                         Bm + order[k] * DIIS_MAX + slot);
        }
        const Z* Fuse = F2;
        if (nvec >= 2) {
            CQ_CUDA(cudaMemcpyAsync(slots, order, nvec * sizeof(int), cudaMemcpyHostToDevice, s));
            diis_solve_kernel<<<1, 32, 0, s>>>(nvec, Bm, slots, coef);
            FPtrs fp;
            for (int k = 0; k < nvec; ++k) fp.p[k] = (const double*)Fs[order[k]];
            // real coefficients: combine the interleaved (re, im) arrays
            diis_combine_kernel<<<nblk(2 * NN), 256, 0, s>>>(2 * NN, nvec, fp, coef, (double*)Fd);
            Fuse = Fd;
        }
        if ((rc = density_from(Fuse))) { cleanup(); return rc; }
        CQ_CUDA(cudaGetLastError());
    }
    cudaEventRecord(e1, s);
    CQ_CUDA(cudaMemcpyAsync(P_out, P, 4 * nn * sizeof(Z), cudaMemcpyDeviceToDevice, s));
    if (F_out) CQ_CUDA(cudaMemcpyAsync(F_out, F, 4 * nn * sizeof(Z), cudaMemcpyDeviceToDevice, s));
    CQ_CUDA(cudaStreamSynchronize(s));
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cleanup();
    st.energy = E;
    st.iterations = converged ? it : o.max_iter;
    st.converged = converged ? 1 : 0;
    st.last_rms = rms;
    st.ms = ms;
    if (stats) *stats = st;
    if (!converged) {
        set_error("cq_scf_ghf: not converged within max_iter");
        return CQ_ERR_NOT_CONVERGED;
    }
    return CQ_OK;
}
