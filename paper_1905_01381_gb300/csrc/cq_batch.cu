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

// per molecule (one block each): E = sum (H + F) D + Enuc; rms of E'
__global__ void batch_energy_rms_kernel(int ld, const double* __restrict__ H, const double* __restrict__ F,
                                        const double* __restrict__ D, const double* __restrict__ Ep,
                                        const double* __restrict__ enuc, const int* __restrict__ mol_n,
                                        double* __restrict__ E, double* __restrict__ rms)
{
    __shared__ double r0[256], r1[256];
    const int m = blockIdx.x;
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

// convergence flags and DIIS bookkeeping per molecule (one thread each)
__global__ void batch_conv_kernel(int nmol, const double* __restrict__ E, const double* __restrict__ Eold,
                                  const double* __restrict__ rms, double e_tol, double d_tol, int check,
                                  int* __restrict__ conv, int* __restrict__ iters, int it,
                                  unsigned int* __restrict__ nopen)
{
    const int m = blockIdx.x * blockDim.x + threadIdx.x;
    if (m >= nmol) return;
    if (conv[m]) return;
    if (check && fabs(E[m] - Eold[m]) < e_tol && rms[m] < d_tol) {
        conv[m] = 1;
        iters[m] = it;
        return;
    }
    atomicAdd(nopen, 1u);
}

// B[m][i][j] = e_i . e_j for slot pairs (grid: molecules x pairs)
__global__ void batch_dot_kernel(int ld, const double* const* __restrict__ Es, const int* __restrict__ pi,
                                 const int* __restrict__ pj, double* __restrict__ Bm)
{
    __shared__ double red[256];
    const int m = blockIdx.x, p = blockIdx.y;
    const size_t slot = (size_t)ld * ld, o = (size_t)m * slot;
    const double* a = Es[pi[p]] + o;
    const double* b = Es[pj[p]] + o;
    double s = 0.0;
    for (size_t i = threadIdx.x; i < slot; i += blockDim.x) s += a[i] * b[i];
    red[threadIdx.x] = s;
    __syncthreads();
    for (int k = blockDim.x / 2; k > 0; k >>= 1) {
        if ((int)threadIdx.x < k) red[threadIdx.x] += red[threadIdx.x + k];
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        Bm[(size_t)m * BDIIS * BDIIS + pi[p] * BDIIS + pj[p]] = red[0];
        Bm[(size_t)m * BDIIS * BDIIS + pj[p] * BDIIS + pi[p]] = red[0];
    }
}

// per molecule: solve the DIIS system over the slots in `order` (nvec)
__global__ void batch_diis_solve_kernel(int nmol, int nvec, const int* __restrict__ order,
                                        const double* __restrict__ Bm, double* __restrict__ coef)
{
    const int mol = blockIdx.x * blockDim.x + threadIdx.x;
    if (mol >= nmol) return;
    double A[BDIIS + 1][BDIIS + 2];
    const double* B = Bm + (size_t)mol * BDIIS * BDIIS;
    const int m = nvec, N = nvec + 1;
    for (int i = 0; i < m; ++i) {
        for (int j = 0; j < m; ++j) A[i][j] = B[order[i] * BDIIS + order[j]];
        A[i][m] = -1.0;
        A[i][m + 1] = 0.0;
    }
    for (int j = 0; j < m; ++j) A[m][j] = -1.0;
    A[m][m] = 0.0;
    A[m][m + 1] = -1.0;
    double* c = coef + (size_t)mol * BDIIS;
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

struct SlotPtrs {
    const double* p[BDIIS];
};

__global__ void batch_diis_combine_kernel(int nmol, int ld, int nvec, SlotPtrs F, const int* __restrict__ order,
                                          const double* __restrict__ coef, double* __restrict__ out)
{
    const size_t slot = (size_t)ld * ld;
    const size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= slot * nmol) return;
    const int m = (int)(i / slot);
    double s = 0.0;
    for (int k = 0; k < nvec; ++k) s += coef[(size_t)m * BDIIS + k] * F.p[order[k]][i];
    out[i] = s;
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
    cq_scf_opts o{1e-10, 1e-8, 128, 8, CQ_PREC_FP64, 1e-5, 1e-14, 0, 8, 1e-5};
    if (opts) o = *opts;
    if (o.diis_size < 1 || o.diis_size > BDIIS || o.max_iter <= 0) {
        set_error("cq_scf_batch: diis_size must be 1..8 and max_iter > 0");
        return CQ_ERR_INVALID_ARG;
    }
    const int nmol = b->nmol, ld = b->ld;
    for (int m = 0; m < nmol; ++m)
        if (nocc[m] <= 0 || nocc[m] > b->mol_n[m]) {
            set_error("cq_scf_batch: nocc out of range for molecule " + std::to_string(m));
            return CQ_ERR_INVALID_ARG;
        }
    cudaStream_t s = (cudaStream_t)stream;
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
    std::vector<void*> bufs;
    int rc = CQ_OK;
    auto get = [&](auto** p, size_t n) -> int {
        int r = dalloc(p, n);
        if (!r) bufs.push_back((void*)*p);
        return r;
    };
    auto cleanup = [&]() {
        for (void* p : bufs) cudaFree(p);
    };
    double *S, *T, *V, *H, *X, *shift, *w, *D, *Dn, *J, *K, *F, *T1, *T2, *Err, *Ep, *Fd, *Bm, *coef, *E, *Eold,
        *rms, *enuc;
    double *Fs[BDIIS], *Es[BDIIS];
    int *conv, *iters, *d_nocc, *d_order, *d_pi, *d_pj, *info;
    unsigned int* nopen;
    const double** d_Es;
#define GETB(p, n)                          \
    if ((rc = get(&(p), (n)))) {            \
        cleanup();                          \
        return rc;                          \
    }
    GETB(S, ms) GETB(T, ms) GETB(V, ms) GETB(H, ms) GETB(X, ms) GETB(shift, (size_t)nmol * ld) GETB(w, (size_t)nmol * ld)
    GETB(D, ms) GETB(Dn, ms) GETB(J, ms) GETB(K, ms) GETB(F, ms) GETB(T1, ms) GETB(T2, ms) GETB(Err, ms) GETB(Ep, ms)
    GETB(Fd, ms) GETB(Bm, (size_t)nmol * BDIIS * BDIIS) GETB(coef, (size_t)nmol * BDIIS) GETB(E, nmol) GETB(Eold, nmol)
    GETB(rms, nmol) GETB(enuc, nmol)
    for (int k = 0; k < o.diis_size; ++k) { GETB(Fs[k], ms) GETB(Es[k], ms) }
    GETB(conv, nmol) GETB(iters, nmol) GETB(d_nocc, nmol) GETB(d_order, BDIIS) GETB(d_pi, BDIIS) GETB(d_pj, BDIIS)
    GETB(info, nmol) GETB(nopen, 1) GETB(d_Es, BDIIS)
#undef GETB
    cusolverDnParams_t prm = nullptr;
    void* dwork = nullptr;
    std::vector<char> hwork;
    auto fail = [&](int r) {
        if (prm) cusolverDnDestroyParams(prm);
        if (dwork) cudaFree(dwork);
        cleanup();
        return r;
    };
    // ---- one-electron data, orthogonalisers
    if ((rc = cq_one_electron(b, S, T, V, nullptr, nullptr, s))) return fail(rc);
    slot_axpby_kernel<<<nb256(ms), 256, 0, s>>>(ms, 1.0, T, 1.0, V, H);
    {
        std::vector<double> en(nmol);
        if ((rc = cq_nuclear_repulsion_batch(b, en.data()))) return fail(rc);
        if (cudaMemcpyAsync(enuc, en.data(), nmol * sizeof(double), cudaMemcpyHostToDevice, s)) return fail(CQ_ERR_CUDA);
        if (cudaMemcpyAsync(d_nocc, nocc, nmol * sizeof(int), cudaMemcpyHostToDevice, s)) return fail(CQ_ERR_CUDA);
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
    auto density_from = [&](const double* Fm, double* Dout) -> int {
        CQ_BLAS_B(gemm_batch(blas, true, false, ld, nmol, 1.0, X, Fm, 0.0, T1));
        CQ_BLAS_B(gemm_batch(blas, false, false, ld, nmol, 1.0, T1, X, 0.0, T2));
        add_diag_kernel<<<nb256((size_t)nmol * ld), 256, 0, s>>>(nmol, ld, shift, T2);
        int r = eig(T2);
        if (r) return r;
        // rows of T2 are eigenvectors: C = X T2^T, occupied columns kept, D = C C^T
        CQ_BLAS_B(gemm_batch(blas, false, true, ld, nmol, 1.0, X, T2, 0.0, T1));
        occ_mask_kernel<<<nb256(ms), 256, 0, s>>>(nmol, ld, d_nocc, T1);
        CQ_BLAS_B(gemm_batch(blas, false, true, ld, nmol, 1.0, T1, T1, 0.0, Dout));
        return CQ_OK;
    };
    if (D_in) {
        if (cudaMemcpyAsync(D, D_in, ms * sizeof(double), cudaMemcpyDeviceToDevice, s)) return fail(CQ_ERR_CUDA);
    } else if ((rc = density_from(H, D))) {
        return fail(rc);
    }
    if (cudaMemsetAsync(conv, 0, nmol * sizeof(int), s) || cudaMemsetAsync(iters, 0, nmol * sizeof(int), s) ||
        cudaMemsetAsync(Eold, 0, nmol * sizeof(double), s))
        return fail(CQ_ERR_CUDA);
    {
        std::vector<const double*> ep(BDIIS, nullptr);
        for (int k = 0; k < o.diis_size; ++k) ep[k] = Es[k];
        if (cudaMemcpyAsync((void*)d_Es, ep.data(), BDIIS * sizeof(double*), cudaMemcpyHostToDevice, s))
            return fail(CQ_ERR_CUDA);
    }
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    cudaEventRecord(e0, s);
    cq_scf_stats st;
    memset(&st, 0, sizeof st);
    int nvec = 0, head = 0, it = 0, open = nmol;
    bool final_fp64 = (o.prec == CQ_PREC_FP64);
    for (it = 1; it <= o.max_iter && open > 0; ++it) {
        cq_fock_opts fo{o.schwarz_tol, o.mixed_tol, final_fp64 ? CQ_PREC_FP64 : CQ_PREC_MIXED, 1, 1};
        cq_fock_stats fst;
        if ((rc = cq_fock_build(b, CQ_DENS_REAL_SYM, D, J, K, &fo, &fst, s))) return fail(rc);
        st.quartets_fp64 += fst.quartets_fp64;
        st.quartets_fp32 += fst.quartets_fp32;
        batch_fock_kernel<<<nb256(ms), 256, 0, s>>>(ms, H, J, K, F);
        CQ_BLAS_B(gemm_batch(blas, false, false, ld, nmol, 1.0, F, D, 0.0, T1));
        CQ_BLAS_B(gemm_batch(blas, false, false, ld, nmol, 1.0, T1, S, 0.0, T2));
        batch_antisym_kernel<<<nb256(ms), 256, 0, s>>>(nmol, ld, T2, Err);
        CQ_BLAS_B(gemm_batch(blas, true, false, ld, nmol, 1.0, X, Err, 0.0, T1));
        CQ_BLAS_B(gemm_batch(blas, false, false, ld, nmol, 1.0, T1, X, 0.0, Ep));
        batch_energy_rms_kernel<<<nmol, 256, 0, s>>>(ld, H, F, D, Ep, enuc, b->d_mol_n, E, rms);
        if (cudaMemsetAsync(nopen, 0, sizeof(unsigned int), s)) return fail(CQ_ERR_CUDA);
        batch_conv_kernel<<<(nmol + 127) / 128, 128, 0, s>>>(nmol, E, Eold, rms, o.e_tol, o.d_tol,
                                                             (it > 1 && final_fp64) ? 1 : 0, conv, iters, it, nopen);
        unsigned int hopen = 0;
        double maxrms_probe = 0.0;
        if (cudaMemcpyAsync(&hopen, nopen, sizeof hopen, cudaMemcpyDeviceToHost, s)) return fail(CQ_ERR_CUDA);
        if (!final_fp64) {
            std::vector<double> hr(nmol);
            if (cudaMemcpyAsync(hr.data(), rms, nmol * sizeof(double), cudaMemcpyDeviceToHost, s))
                return fail(CQ_ERR_CUDA);
            if (cudaStreamSynchronize(s)) return fail(CQ_ERR_CUDA);
            for (double x : hr) maxrms_probe = std::fmax(maxrms_probe, x);
            if (maxrms_probe < o.switch_tol) final_fp64 = true;
        } else if (cudaStreamSynchronize(s)) {
            return fail(CQ_ERR_CUDA);
        }
        open = (int)hopen;
        if (open == 0) break;
        if (cudaMemcpyAsync(Eold, E, nmol * sizeof(double), cudaMemcpyDeviceToDevice, s)) return fail(CQ_ERR_CUDA);
        // a supplied starting density need not be idempotent: its Fock matrix
        // is diagonalised as it is and kept out of the DIIS subspace
        if (it == 1 && D_in) {
            if ((rc = density_from(F, Dn))) return fail(rc);
            freeze_update_kernel<<<nb256(ms), 256, 0, s>>>(nmol, ld, conv, Dn, D);
            continue;
        }
        // DIIS
        const int slot = head;
        head = (head + 1) % o.diis_size;
        nvec = nvec < o.diis_size ? nvec + 1 : nvec;
        if (cudaMemcpyAsync(Fs[slot], F, ms * sizeof(double), cudaMemcpyDeviceToDevice, s) ||
            cudaMemcpyAsync(Es[slot], Ep, ms * sizeof(double), cudaMemcpyDeviceToDevice, s))
            return fail(CQ_ERR_CUDA);
        int order[BDIIS], pi[BDIIS], pj[BDIIS];
        for (int k = 0; k < nvec; ++k) {
            order[k] = (head - nvec + k + o.diis_size) % o.diis_size;
            pi[k] = slot;
            pj[k] = order[k];
        }
        if (cudaMemcpyAsync(d_order, order, nvec * sizeof(int), cudaMemcpyHostToDevice, s) ||
            cudaMemcpyAsync(d_pi, pi, nvec * sizeof(int), cudaMemcpyHostToDevice, s) ||
            cudaMemcpyAsync(d_pj, pj, nvec * sizeof(int), cudaMemcpyHostToDevice, s))
            return fail(CQ_ERR_CUDA);
        batch_dot_kernel<<<dim3(nmol, nvec), 256, 0, s>>>(ld, d_Es, d_pi, d_pj, Bm);
        const double* Fuse = F;
        if (nvec >= 2) {
            batch_diis_solve_kernel<<<(nmol + 127) / 128, 128, 0, s>>>(nmol, nvec, d_order, Bm, coef);
            SlotPtrs fp;
            for (int k = 0; k < BDIIS; ++k) fp.p[k] = k < o.diis_size ? Fs[k] : nullptr;
            batch_diis_combine_kernel<<<nb256(ms), 256, 0, s>>>(nmol, ld, nvec, fp, d_order, coef, Fd);
            Fuse = Fd;
        }
        if ((rc = density_from(Fuse, Dn))) return fail(rc);
        freeze_update_kernel<<<nb256(ms), 256, 0, s>>>(nmol, ld, conv, Dn, D);
        if (cudaGetLastError() != cudaSuccess) return fail(CQ_ERR_CUDA);
    }
    cudaEventRecord(e1, s);
    if (cudaMemcpyAsync(D_out, D, ms * sizeof(double), cudaMemcpyDeviceToDevice, s)) return fail(CQ_ERR_CUDA);
    std::vector<double> hE(nmol);
    std::vector<int> hit(nmol), hconv(nmol);
    if (cudaMemcpyAsync(hE.data(), E, nmol * sizeof(double), cudaMemcpyDeviceToHost, s) ||
        cudaMemcpyAsync(hit.data(), iters, nmol * sizeof(int), cudaMemcpyDeviceToHost, s) ||
        cudaMemcpyAsync(hconv.data(), conv, nmol * sizeof(int), cudaMemcpyDeviceToHost, s) ||
        cudaStreamSynchronize(s))
        return fail(CQ_ERR_CUDA);
    float msf = 0.f;
    cudaEventElapsedTime(&msf, e0, e1);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    int nconv = 0;
    double esum = 0.0;
    for (int m = 0; m < nmol; ++m) {
        if (E_out) E_out[m] = hE[m];
        if (iters_out) iters_out[m] = hconv[m] ? hit[m] : o.max_iter;
        nconv += hconv[m];
        esum += hE[m];
    }
    st.energy = esum;
    st.iterations = it;
    st.converged = nconv;
    st.ms = msf;
    if (stats) *stats = st;
    fail(CQ_OK);
    if (nconv < nmol) {
        set_error("cq_scf_batch: " + std::to_string(nmol - nconv) + " molecule(s) not converged");
        return CQ_ERR_NOT_CONVERGED;
    }
    return CQ_OK;
}
