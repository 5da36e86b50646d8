// Learned initial density: a small MLP over atom-pair descriptors predicts
// the density blocks P_AB of the even-tempered s,p,d basis (H: 3s1p, 6
// functions; C/N/O: 4s3p2d, 25 functions), trained on converged SCF
// densities.  Hand-written kernels: FP32 tiled GEMM (forward and backward),
// bias + SiLU, masked MSE, Adam; descriptors, block gather and scatter.
// The guess is assembled per molecule, symmetrised, scaled to Tr(PS) = nocc
// and optionally McWeeny-purified (P <- 3PSP - 2PSPSP); the SCF then judges it, so only
// the iteration count can change, never the converged answer.
#include <cublas_v2.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <random>
#include <vector>

#include "cq_internal.h"

namespace cq {

constexpr int MLP_IN = 40, MLP_H = 256;
constexpr int MLP_NHEAD = 5;
// heads: 0 H on-site 6x6, 1 heavy on-site 25x25, 2 H-H 6x6, 3 H-heavy 6x25, 4 heavy-heavy 25x25
__host__ __device__ constexpr int head_rows(int h) { return (h == 1 || h == 4) ? 25 : 6; }
__host__ __device__ constexpr int head_cols(int h) { return (h == 0 || h == 2) ? 6 : 25; }
__host__ __device__ constexpr int head_off(int h)
{
    return h == 0 ? 0 : h == 1 ? 36 : h == 2 ? 661 : h == 3 ? 697 : h == 4 ? 847 : 1472;
}
constexpr int MLP_OUT = 1472;
constexpr size_t MLP_NPARAM = (size_t)MLP_H * MLP_IN + MLP_H + (size_t)MLP_H * MLP_H + MLP_H +
                              (size_t)MLP_OUT * MLP_H + MLP_OUT;

struct MLPView {
    float *W1, *b1, *W2, *b2, *W3, *b3;
};
static MLPView view(float* p)
{
    MLPView v;
    v.W1 = p; p += (size_t)MLP_H * MLP_IN;
    v.b1 = p; p += MLP_H;
    v.W2 = p; p += (size_t)MLP_H * MLP_H;
    v.b2 = p; p += MLP_H;
    v.W3 = p; p += (size_t)MLP_OUT * MLP_H;
    v.b3 = p;
    return v;
}

// ------------------------------------------------------------ descriptors
struct PairRec {
    int mol, first, second;   // atoms (first = the H atom of an H-heavy pair)
    int head;
    int f_first, f_second;    // first function of each atom within its molecule
};

__device__ __forceinline__ int zslot(int Z) { return Z == 1 ? 0 : Z == 6 ? 1 : Z == 7 ? 2 : 3; }

__global__ void descriptor_kernel(int npair, const PairRec* __restrict__ pr, const double* __restrict__ xyz,
                                  const double* __restrict__ Zc, const int* __restrict__ mol_atom_off,
                                  float* __restrict__ X)
{
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= npair) return;
    const PairRec r = pr[p];
    float* x = X + (size_t)p * MLP_IN;
    for (int k = 0; k < MLP_IN; ++k) x[k] = 0.f;
    const int A = r.first, B = r.second;
    x[zslot((int)Zc[A])] = 1.f;
    x[4 + zslot((int)Zc[B])] = 1.f;
    double d[3], R2 = 0.0;
    for (int k = 0; k < 3; ++k) { d[k] = xyz[3 * B + k] - xyz[3 * A + k]; R2 += d[k] * d[k]; }
    const double R = sqrt(R2);
    x[8] = A == B ? 1.f : 0.f;
    x[9] = (float)(R / 4.0);
    for (int k = 0; k < 16; ++k) {
        const double t = (R - 0.5 * k) / 0.5;
        x[10 + k] = (float)exp(-t * t);
    }
    if (A != B) {
        const double u[3] = {d[0] / R, d[1] / R, d[2] / R};
        x[26] = (float)u[0]; x[27] = (float)u[1]; x[28] = (float)u[2];
        x[29] = (float)(u[0] * u[0]); x[30] = (float)(u[0] * u[1]); x[31] = (float)(u[0] * u[2]);
        x[32] = (float)(u[1] * u[1]); x[33] = (float)(u[1] * u[2]); x[34] = (float)(u[2] * u[2]);
    }
    // smooth coordination numbers of both atoms within their molecule
    double cA = 0.0, cB = 0.0;
    for (int C = mol_atom_off[r.mol]; C < mol_atom_off[r.mol + 1]; ++C) {
        double ra = 0.0, rb = 0.0;
        for (int k = 0; k < 3; ++k) {
            ra += (xyz[3 * C + k] - xyz[3 * A + k]) * (xyz[3 * C + k] - xyz[3 * A + k]);
            rb += (xyz[3 * C + k] - xyz[3 * B + k]) * (xyz[3 * C + k] - xyz[3 * B + k]);
        }
        if (C != A) cA += exp(-ra / 9.0);
        if (C != B) cB += exp(-rb / 9.0);
    }
    x[35] = (float)cA;
    x[36] = (float)cB;
}

// ------------------------------------------------------------ FP32 GEMM
// C (M x N) = op(A) op(B) (+ bias over columns), row-major, 64 x 64 tiles,
// 256 threads with 4 x 4 outputs each; op(A) is M x K, op(B) is K x N.
constexpr int GT = 64, GK = 16;
__global__ void __launch_bounds__(256) sgemm_kernel(int M, int N, int K, int ta, int tb, const float* __restrict__ A,
                                                    int lda, const float* __restrict__ B, int ldb,
                                                    float* __restrict__ C, int ldc, const float* __restrict__ bias,
                                                    float beta)
{
    __shared__ float As[GK][GT + 4];
    __shared__ float Bs[GK][GT + 4];
    const int tx = threadIdx.x % 16, ty = threadIdx.x / 16;
    const int row0 = blockIdx.y * GT, col0 = blockIdx.x * GT;
    float acc[4][4] = {};
    for (int k0 = 0; k0 < K; k0 += GK) {
        for (int e = threadIdx.x; e < GK * GT; e += 256) {
            const int kk = e / GT, mm = e % GT;
            const int gr = row0 + mm, gk = k0 + kk;
            float va = 0.f;
            if (gr < M && gk < K) va = ta ? A[(size_t)gk * lda + gr] : A[(size_t)gr * lda + gk];
            As[kk][mm] = va;
            const int gc = col0 + mm;
            float vb = 0.f;
            if (gc < N && gk < K) vb = tb ? B[(size_t)gc * ldb + gk] : B[(size_t)gk * ldb + gc];
            Bs[kk][mm] = vb;
        }
        __syncthreads();
#pragma unroll
        for (int kk = 0; kk < GK; ++kk) {
            float a[4], b[4];
#pragma unroll
            for (int i = 0; i < 4; ++i) { a[i] = As[kk][ty * 4 + i]; b[i] = Bs[kk][tx * 4 + i]; }
#pragma unroll
            for (int i = 0; i < 4; ++i)
#pragma unroll
                for (int j = 0; j < 4; ++j) acc[i][j] = fmaf(a[i], b[j], acc[i][j]);
        }
        __syncthreads();
    }
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const int r = row0 + ty * 4 + i, c = col0 + tx * 4 + j;
            if (r < M && c < N) {
                float v = acc[i][j] + (bias ? bias[c] : 0.f);
                if (beta != 0.f) v += beta * C[(size_t)r * ldc + c];
                C[(size_t)r * ldc + c] = v;
            }
        }
}

static void sgemm(cudaStream_t s, int M, int N, int K, bool ta, bool tb, const float* A, int lda, const float* B,
                  int ldb, float* C, int ldc, const float* bias = nullptr, float beta = 0.f)
{
    dim3 grid((N + GT - 1) / GT, (M + GT - 1) / GT);
    sgemm_kernel<<<grid, 256, 0, s>>>(M, N, K, ta, tb, A, lda, B, ldb, C, ldc, bias, beta);
}

__device__ __forceinline__ float sigm(float z) { return 1.f / (1.f + __expf(-z)); }

__global__ void silu_kernel(size_t n, const float* __restrict__ z, float* __restrict__ h)
{
    const size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) h[i] = z[i] * sigm(z[i]);
}

__global__ void silu_back_kernel(size_t n, const float* __restrict__ z, float* __restrict__ g)
{
    const size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const float s = sigm(z[i]);
    g[i] *= s * (1.f + z[i] * (1.f - s));
}

// masked MSE over each sample's head slice: loss and dY = 2 (y - t) / count
__global__ void mse_kernel(int n, const float* __restrict__ Y, const float* __restrict__ T,
                           const int* __restrict__ head, float inv_count, float* __restrict__ dY,
                           double* __restrict__ loss)
{
    const size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= (size_t)n * MLP_OUT) return;
    const int r = (int)(i / MLP_OUT), c = (int)(i % MLP_OUT);
    const int h = head[r];
    const bool on = c >= head_off(h) && c < head_off(h + 1);
    const float d = on ? Y[i] - T[i] : 0.f;
    dY[i] = 2.f * d * inv_count;
    if (on && loss) atomicAdd(loss, (double)d * d * inv_count);
}

__global__ void colsum_kernel(int n, int cols, const float* __restrict__ G, float* __restrict__ out)
{
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= cols) return;
    float s = 0.f;
    for (int r = 0; r < n; ++r) s += G[(size_t)r * cols + c];
    out[c] = s;
}

__global__ void adam_kernel(size_t n, float* __restrict__ p, const float* __restrict__ g, float* __restrict__ m,
                            float* __restrict__ v, float lr, float b1, float b2, float c1, float c2, float eps)
{
    const size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    m[i] = b1 * m[i] + (1.f - b1) * g[i];
    v[i] = b2 * v[i] + (1.f - b2) * g[i] * g[i];
    p[i] -= lr * (m[i] / c1) / (sqrtf(v[i] / c2) + eps);
}

__global__ void gather_rows_kernel(int n, int cols, const int* __restrict__ idx, const float* __restrict__ src,
                                   float* __restrict__ dst)
{
    const size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= (size_t)n * cols) return;
    const int r = (int)(i / cols), c = (int)(i % cols);
    dst[i] = src[(size_t)idx[r] * cols + c];
}

__global__ void gather_int_kernel(int n, const int* __restrict__ idx, const int* __restrict__ src, int* __restrict__ dst)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) dst[i] = src[idx[i]];
}

// density blocks -> targets (rows first atom, columns second atom)
__global__ void block_gather_kernel(int npair, const PairRec* __restrict__ pr, int ld, const double* __restrict__ D,
                                    float* __restrict__ T)
{
    const int p = blockIdx.x;
    const PairRec r = pr[p];
    const int nr = head_rows(r.head), nc = head_cols(r.head), off = head_off(r.head);
    const double* Dm = D + (size_t)r.mol * ld * ld;
    for (int e = threadIdx.x; e < MLP_OUT; e += blockDim.x) {
        float v = 0.f;
        if (e >= off && e < off + nr * nc) {
            const int i = (e - off) / nc, j = (e - off) % nc;
            v = (float)Dm[(size_t)(r.f_first + i) * ld + r.f_second + j];
        }
        T[(size_t)p * MLP_OUT + e] = v;
    }
}

// predictions -> guess density blocks (and transposes); on-site blocks
// symmetrised
__global__ void block_scatter_kernel(int npair, const PairRec* __restrict__ pr, int ld, const float* __restrict__ Y,
                                     double* __restrict__ D, int onsite_only)
{
    const int p = blockIdx.x;
    const PairRec r = pr[p];
    if (onsite_only && r.first != r.second) return;
    const int nr = head_rows(r.head), nc = head_cols(r.head), off = head_off(r.head);
    double* Dm = D + (size_t)r.mol * ld * ld;
    for (int e = threadIdx.x; e < nr * nc; e += blockDim.x) {
        const int i = e / nc, j = e % nc;
        const float* y = Y + (size_t)p * MLP_OUT + off;
        if (r.first == r.second) {
            Dm[(size_t)(r.f_first + i) * ld + r.f_second + j] = 0.5 * ((double)y[i * nc + j] + (double)y[j * nc + i]);
        } else {
            Dm[(size_t)(r.f_first + i) * ld + r.f_second + j] = (double)y[e];
            Dm[(size_t)(r.f_second + j) * ld + r.f_first + i] = (double)y[e];
        }
    }
}

// per molecule (one block): t = Tr(P S)
__global__ void trace_ps_kernel(int ld, const double* __restrict__ P, const double* __restrict__ S,
                                double* __restrict__ t)
{
    __shared__ double red[256];
    const int m = blockIdx.x;
    const size_t o = (size_t)m * ld * ld;
    double a = 0.0;
    for (size_t i = threadIdx.x; i < (size_t)ld * ld; i += blockDim.x) a += P[o + i] * S[o + i];
    red[threadIdx.x] = a;
    __syncthreads();
    for (int k = blockDim.x / 2; k > 0; k >>= 1) {
        if ((int)threadIdx.x < k) red[threadIdx.x] += red[threadIdx.x + k];
        __syncthreads();
    }
    if (threadIdx.x == 0) t[m] = red[0];
}

__global__ void scale_slots_kernel(int nmol, int ld, const double* __restrict__ t, const int* __restrict__ nocc,
                                   double* __restrict__ P)
{
    const size_t slot = (size_t)ld * ld;
    const size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= slot * nmol) return;
    const int m = (int)(i / slot);
    const double tr = t[m];
    P[i] *= (tr > 1e-12) ? nocc[m] / tr : 0.0;
}

__global__ void axpby_d_kernel(size_t n, double a, const double* __restrict__ x, double b, const double* __restrict__ y,
                               double* __restrict__ z)
{
    const size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) z[i] = a * x[i] + b * y[i];
}

static int nb(size_t n) { return (int)((n + 255) / 256); }

static std::vector<PairRec> build_pairs(const cq_basis* b, int* bad)
{
    std::vector<PairRec> out;
    *bad = 0;
    // first function of each atom within its molecule; function count per atom
    std::vector<int> afirst(b->natom, -1), acount(b->natom, 0);
    for (int s = 0; s < b->nsh; ++s) {
        const int A = b->atom[s];
        if (afirst[A] < 0) afirst[A] = b->bfo[s];
        acount[A] += ncart(b->L[s]);
    }
    for (int m = 0; m < b->nmol; ++m) {
        const int f0 = b->mol_bfo[m];
        for (int A = b->mol_atom_off[m]; A < b->mol_atom_off[m + 1]; ++A) {
            const int nA = acount[A];
            if (!((b->Z[A] == 1 && nA == 6) || (b->Z[A] > 1 && nA == 25))) { *bad = 1; continue; }
            for (int B = b->mol_atom_off[m]; B <= A; ++B) {
                const int nB = acount[B];
                if (!((b->Z[B] == 1 && nB == 6) || (b->Z[B] > 1 && nB == 25))) continue;
                PairRec r;
                r.mol = m;
                int first = A, second = B;
                const bool hA = b->Z[A] == 1, hB = b->Z[B] == 1;
                if (A == B) r.head = hA ? 0 : 1;
                else if (hA && hB) r.head = 2;
                else if (!hA && !hB) r.head = 4;
                else { r.head = 3; if (!hA) std::swap(first, second); }
                r.first = first;
                r.second = second;
                r.f_first = afirst[first] - f0;
                r.f_second = afirst[second] - f0;
                out.push_back(r);
            }
        }
    }
    return out;
}

struct GuessCtx {
    std::vector<PairRec> pairs;
    PairRec* d_pairs = nullptr;
    float* d_X = nullptr;
    int* d_head = nullptr;
};

static int prepare(const cq_basis* b, GuessCtx& g, cudaStream_t s)
{
    int bad = 0;
    g.pairs = build_pairs(b, &bad);
    if (bad) {
        set_error("learned guess: every atom must carry the even-tempered s,p,d basis (H 3s1p, heavy 4s3p2d)");
        return CQ_ERR_UNSUPPORTED;
    }
    const int np = (int)g.pairs.size();
    int rc;
    if ((rc = dalloc(&g.d_pairs, np)) || (rc = dalloc(&g.d_X, (size_t)np * MLP_IN)) || (rc = dalloc(&g.d_head, np)))
        return rc;
    std::vector<int> heads(np);
    for (int p = 0; p < np; ++p) heads[p] = g.pairs[p].head;
    CQ_CUDA(cudaMemcpyAsync(g.d_pairs, g.pairs.data(), np * sizeof(PairRec), cudaMemcpyHostToDevice, s));
    CQ_CUDA(cudaMemcpyAsync(g.d_head, heads.data(), np * sizeof(int), cudaMemcpyHostToDevice, s));
    descriptor_kernel<<<nb(np), 256, 0, s>>>(np, g.d_pairs, b->d_axyz, b->d_Z, b->d_mol_atom_off, g.d_X);
    CQ_CUDA(cudaGetLastError());
    CQ_CUDA(cudaStreamSynchronize(s));
    return CQ_OK;
}

static void release(GuessCtx& g)
{
    if (g.d_pairs) cudaFree(g.d_pairs);
    if (g.d_X) cudaFree(g.d_X);
    if (g.d_head) cudaFree(g.d_head);
    g.d_pairs = nullptr; g.d_X = nullptr; g.d_head = nullptr;
}

// forward pass for n rows: z1, h1, z2, h2 saved (n x H each), Y (n x OUT)
static void forward(cudaStream_t s, const MLPView& w, int n, const float* X, float* z1, float* h1, float* z2,
                    float* h2, float* Y)
{
    sgemm(s, n, MLP_H, MLP_IN, false, true, X, MLP_IN, w.W1, MLP_IN, z1, MLP_H, w.b1);
    silu_kernel<<<nb((size_t)n * MLP_H), 256, 0, s>>>((size_t)n * MLP_H, z1, h1);
    sgemm(s, n, MLP_H, MLP_H, false, true, h1, MLP_H, w.W2, MLP_H, z2, MLP_H, w.b2);
    silu_kernel<<<nb((size_t)n * MLP_H), 256, 0, s>>>((size_t)n * MLP_H, z2, h2);
    sgemm(s, n, MLP_OUT, MLP_H, false, true, h2, MLP_H, w.W3, MLP_H, Y, MLP_OUT, w.b3);
}

// backward pass from dY; gradients into g (same layout as the parameters)
static void backward(cudaStream_t s, const MLPView& w, const MLPView& g, int n, const float* X, const float* z1,
                     const float* h1, const float* z2, const float* h2, float* dY, float* d2, float* d1)
{
    sgemm(s, MLP_OUT, MLP_H, n, true, false, dY, MLP_OUT, h2, MLP_H, g.W3, MLP_H);
    colsum_kernel<<<nb(MLP_OUT), 256, 0, s>>>(n, MLP_OUT, dY, g.b3);
    sgemm(s, n, MLP_H, MLP_OUT, false, false, dY, MLP_OUT, w.W3, MLP_H, d2, MLP_H);
    silu_back_kernel<<<nb((size_t)n * MLP_H), 256, 0, s>>>((size_t)n * MLP_H, z2, d2);
    sgemm(s, MLP_H, MLP_H, n, true, false, d2, MLP_H, h1, MLP_H, g.W2, MLP_H);
    colsum_kernel<<<nb(MLP_H), 256, 0, s>>>(n, MLP_H, d2, g.b2);
    sgemm(s, n, MLP_H, MLP_H, false, false, d2, MLP_H, w.W2, MLP_H, d1, MLP_H);
    silu_back_kernel<<<nb((size_t)n * MLP_H), 256, 0, s>>>((size_t)n * MLP_H, z1, d1);
    sgemm(s, MLP_H, MLP_IN, n, true, false, d1, MLP_H, X, MLP_IN, g.W1, MLP_IN);
    colsum_kernel<<<nb(MLP_H), 256, 0, s>>>(n, MLP_H, d1, g.b1);
}

struct Work {
    float *z1 = nullptr, *h1 = nullptr, *z2 = nullptr, *h2 = nullptr, *Y = nullptr, *d1 = nullptr, *d2 = nullptr;
    int alloc(size_t n)
    {
        int rc;
        if ((rc = dalloc(&z1, n * MLP_H)) || (rc = dalloc(&h1, n * MLP_H)) || (rc = dalloc(&z2, n * MLP_H)) ||
            (rc = dalloc(&h2, n * MLP_H)) || (rc = dalloc(&Y, n * MLP_OUT)) || (rc = dalloc(&d1, n * MLP_H)) ||
            (rc = dalloc(&d2, n * MLP_H)))
            return rc;
        return CQ_OK;
    }
    ~Work()
    {
        float* p[] = {z1, h1, z2, h2, Y, d1, d2};
        for (float* x : p)
            if (x) cudaFree(x);
    }
};

}  // namespace cq

using namespace cq;

extern "C" size_t cq_mlp_param_count(void) { return MLP_NPARAM; }

// Seeded initialisation (uniform, +-sqrt(6 / (fan_in + fan_out)), zero biases).
extern "C" int cq_mlp_init(float* params, unsigned long long seed, void* stream)
{
    if (!params) { set_error("cq_mlp_init: NULL"); return CQ_ERR_INVALID_ARG; }
    std::vector<float> h(MLP_NPARAM, 0.f);
    std::mt19937_64 g(seed);
    auto fill = [&](size_t off, int rows, int cols) {
        const float a = std::sqrt(6.f / (rows + cols));
        std::uniform_real_distribution<float> u(-a, a);
        for (size_t i = 0; i < (size_t)rows * cols; ++i) h[off + i] = u(g);
    };
    size_t o = 0;
    fill(o, MLP_H, MLP_IN); o += (size_t)MLP_H * MLP_IN + MLP_H;
    fill(o, MLP_H, MLP_H); o += (size_t)MLP_H * MLP_H + MLP_H;
    fill(o, MLP_OUT, MLP_H);
    CQ_CUDA(cudaMemcpyAsync(params, h.data(), MLP_NPARAM * sizeof(float), cudaMemcpyHostToDevice,
                            (cudaStream_t)stream));
    CQ_CUDA(cudaStreamSynchronize((cudaStream_t)stream));
    return CQ_OK;
}

// Training set from a batched basis and its converged densities (batched
// layout): descriptors X (npair x 40), targets T (npair x 1472), heads.
// Returns the pair count in *npair; X/T/head may be NULL to only count.
extern "C" int cq_guess_dataset(cq_basis* b, const double* D, float* X, float* T, int* head, int* npair, void* stream)
{
    if (!b || !npair) { set_error("cq_guess_dataset: NULL argument"); return CQ_ERR_INVALID_ARG; }
    cudaStream_t s = (cudaStream_t)stream;
    GuessCtx g;
    int rc = prepare(b, g, s);
    if (rc) { release(g); return rc; }
    const int np = (int)g.pairs.size();
    *npair = np;
    if (X) cudaMemcpyAsync(X, g.d_X, (size_t)np * MLP_IN * sizeof(float), cudaMemcpyDeviceToDevice, s);
    if (head) cudaMemcpyAsync(head, g.d_head, np * sizeof(int), cudaMemcpyDeviceToDevice, s);
    if (T && D && np > 0) block_gather_kernel<<<np, 256, 0, s>>>(np, g.d_pairs, b->ld, D, T);
    cudaError_t e = cudaStreamSynchronize(s);
    release(g);
    if (e != cudaSuccess) return cuda_fail(e, "cq_guess_dataset");
    return CQ_OK;
}

// Loss and gradient of the masked MSE for n samples (gradient check support).
extern "C" int cq_mlp_loss_grad(const float* params, int n, const float* X, const float* T, const int* head,
                                float* grad, double* loss, void* stream)
{
    if (!params || !X || !T || !head || n <= 0) { set_error("cq_mlp_loss_grad: bad argument"); return CQ_ERR_INVALID_ARG; }
    cudaStream_t s = (cudaStream_t)stream;
    Work w;
    int rc = w.alloc(n);
    if (rc) return rc;
    double* dl = nullptr;
    if ((rc = dalloc(&dl, 1))) return rc;
    std::vector<int> hh(n);
    CQ_CUDA(cudaMemcpy(hh.data(), head, n * sizeof(int), cudaMemcpyDeviceToHost));
    double cnt = 0.0;
    for (int h : hh) cnt += head_rows(h) * head_cols(h);
    const MLPView pv = view(const_cast<float*>(params));
    forward(s, pv, n, X, w.z1, w.h1, w.z2, w.h2, w.Y);
    cudaMemsetAsync(dl, 0, sizeof(double), s);
    mse_kernel<<<nb((size_t)n * MLP_OUT), 256, 0, s>>>(n, w.Y, T, head, (float)(1.0 / cnt), w.Y, dl);
    if (grad) backward(s, pv, view(grad), n, X, w.z1, w.h1, w.z2, w.h2, w.Y, w.d2, w.d1);
    double hl = 0.0;
    cudaMemcpyAsync(&hl, dl, sizeof hl, cudaMemcpyDeviceToHost, s);
    cudaError_t e = cudaStreamSynchronize(s);
    cudaFree(dl);
    if (e != cudaSuccess) return cuda_fail(e, "cq_mlp_loss_grad");
    if (loss) *loss = hl;
    return CQ_OK;
}

// Adam training over (X, T, head) for `epochs` passes with minibatches of
// `batch` rows shuffled by `seed`.  Returns the mean loss of the last epoch.
extern "C" int cq_mlp_train(float* params, int n, const float* X, const float* T, const int* head, int epochs,
                            int batch, float lr, unsigned long long seed, double* last_loss, void* stream)
{
    if (!params || !X || !T || !head || n <= 0 || epochs <= 0 || batch <= 0) {
        set_error("cq_mlp_train: bad argument");
        return CQ_ERR_INVALID_ARG;
    }
    cudaStream_t s = (cudaStream_t)stream;
    batch = std::min(batch, n);
    Work w;
    int rc = w.alloc(batch);
    if (rc) return rc;
    float *g = nullptr, *m = nullptr, *v = nullptr, *Xb = nullptr, *Tb = nullptr;
    int *idx = nullptr, *hb = nullptr;
    double* dl = nullptr;
    std::vector<void*> bufs;
    auto cleanup = [&]() {
        for (void* p : bufs) cudaFree(p);
    };
#define GETM(p, c)                       \
    if ((rc = dalloc(&(p), (c)))) {      \
        cleanup();                       \
        return rc;                       \
    }                                    \
    bufs.push_back((void*)(p));
    GETM(g, MLP_NPARAM) GETM(m, MLP_NPARAM) GETM(v, MLP_NPARAM) GETM(Xb, (size_t)batch * MLP_IN)
    GETM(Tb, (size_t)batch * MLP_OUT) GETM(idx, n) GETM(hb, batch) GETM(dl, 1)
#undef GETM
    cudaMemsetAsync(m, 0, MLP_NPARAM * sizeof(float), s);
    cudaMemsetAsync(v, 0, MLP_NPARAM * sizeof(float), s);
    std::vector<int> hh(n), perm(n);
    CQ_CUDA(cudaMemcpy(hh.data(), head, n * sizeof(int), cudaMemcpyDeviceToHost));
    for (int i = 0; i < n; ++i) perm[i] = i;
    std::mt19937_64 rng(seed);
    const MLPView pv = view(params), gv = view(g);
    int step = 0;
    double epoch_loss = 0.0;
    for (int ep = 0; ep < epochs; ++ep) {
        std::shuffle(perm.begin(), perm.end(), rng);
        CQ_CUDA(cudaMemcpyAsync(idx, perm.data(), n * sizeof(int), cudaMemcpyHostToDevice, s));
        cudaMemsetAsync(dl, 0, sizeof(double), s);
        int nbat = 0;
        for (int b0 = 0; b0 + batch <= n || (b0 < n && nbat == 0); b0 += batch) {
            const int nb_rows = std::min(batch, n - b0);
            double cnt = 0.0;
            for (int r = 0; r < nb_rows; ++r) cnt += head_rows(hh[perm[b0 + r]]) * head_cols(hh[perm[b0 + r]]);
            gather_rows_kernel<<<nb((size_t)nb_rows * MLP_IN), 256, 0, s>>>(nb_rows, MLP_IN, idx + b0, X, Xb);
            gather_rows_kernel<<<nb((size_t)nb_rows * MLP_OUT), 256, 0, s>>>(nb_rows, MLP_OUT, idx + b0, T, Tb);
            gather_int_kernel<<<nb(nb_rows), 256, 0, s>>>(nb_rows, idx + b0, head, hb);
            forward(s, pv, nb_rows, Xb, w.z1, w.h1, w.z2, w.h2, w.Y);
            mse_kernel<<<nb((size_t)nb_rows * MLP_OUT), 256, 0, s>>>(nb_rows, w.Y, Tb, hb, (float)(1.0 / cnt), w.Y, dl);
            backward(s, pv, gv, nb_rows, Xb, w.z1, w.h1, w.z2, w.h2, w.Y, w.d2, w.d1);
            ++step;
            const float b1 = 0.9f, b2 = 0.999f;
            adam_kernel<<<nb(MLP_NPARAM), 256, 0, s>>>(MLP_NPARAM, params, g, m, v, lr, b1, b2,
                                                      1.f - std::pow(b1, (float)step), 1.f - std::pow(b2, (float)step),
                                                      1e-8f);
            ++nbat;
        }
        double hl = 0.0;
        CQ_CUDA(cudaMemcpyAsync(&hl, dl, sizeof hl, cudaMemcpyDeviceToHost, s));
        CQ_CUDA(cudaStreamSynchronize(s));
        epoch_loss = hl / std::max(1, nbat);
    }
    CQ_CUDA(cudaGetLastError());
    if (last_loss) *last_loss = epoch_loss;
    cleanup();
    return CQ_OK;
}

// Learned guess for every molecule of a batched basis: predicted blocks
// assembled into D (batched layout; flags bit 0: on-site blocks only, a
// superposition of learned atomic densities), scaled to Tr(DS) = nocc[m],
// then `npurify` McWeeny steps D <- 3DSD - 2DSDSD.
extern "C" int cq_guess_density(cq_basis* b, const float* params, const int* nocc, int npurify, int flags,
                                double* D, void* stream)
{
    if (!b || !params || !nocc || !D) { set_error("cq_guess_density: NULL argument"); return CQ_ERR_INVALID_ARG; }
    cudaStream_t s = (cudaStream_t)stream;
    GuessCtx g;
    int rc = prepare(b, g, s);
    if (rc) { release(g); return rc; }
    const int np = (int)g.pairs.size();
    const int nmol = b->nmol, ld = b->ld;
    const size_t ms = (size_t)b->mstride;
    Work w;
    if ((rc = w.alloc(np))) { release(g); return rc; }
    double *S = nullptr, *t = nullptr, *A = nullptr, *Bt = nullptr, *C = nullptr;
    int* dno = nullptr;
    std::vector<void*> bufs;
    auto cleanup = [&]() {
        for (void* p : bufs) cudaFree(p);
        release(g);
    };
#define GETG(p, c)                       \
    if ((rc = dalloc(&(p), (c)))) {      \
        cleanup();                       \
        return rc;                       \
    }                                    \
    bufs.push_back((void*)(p));
    GETG(S, ms) GETG(t, nmol) GETG(A, ms) GETG(Bt, ms) GETG(C, ms) GETG(dno, nmol)
#undef GETG
    CQ_CUDA(cudaMemcpyAsync(dno, nocc, nmol * sizeof(int), cudaMemcpyHostToDevice, s));
    forward(s, view(const_cast<float*>(params)), np, g.d_X, w.z1, w.h1, w.z2, w.h2, w.Y);
    CQ_CUDA(cudaMemsetAsync(D, 0, ms * sizeof(double), s));
    block_scatter_kernel<<<np, 256, 0, s>>>(np, g.d_pairs, ld, w.Y, D, flags & 1);
    if ((rc = cq_one_electron(b, S, nullptr, nullptr, nullptr, nullptr, s))) { cleanup(); return rc; }
    trace_ps_kernel<<<nmol, 256, 0, s>>>(ld, D, S, t);
    scale_slots_kernel<<<nb(ms), 256, 0, s>>>(nmol, ld, t, dno, D);
    if (!b->blas) {
        cublasHandle_t h;
        if (cublasCreate(&h) != CUBLAS_STATUS_SUCCESS) { cleanup(); set_error("cublasCreate failed"); return CQ_ERR_CUDA; }
        b->blas = h;
    }
    cublasHandle_t h = (cublasHandle_t)b->blas;
    cublasSetStream(h, s);
    const long long st = (long long)ld * ld;
    const double one = 1.0, zero = 0.0;
    for (int k = 0; k < npurify; ++k) {
        // A = D S ; Bt = A D (= DSD) ; C = A Bt (= DSDSD) ; D = 3 Bt - 2 C  (row-major via transposed calls)
        cublasDgemmStridedBatched(h, CUBLAS_OP_N, CUBLAS_OP_N, ld, ld, ld, &one, S, ld, st, D, ld, st, &zero, A, ld, st, nmol);
        cublasDgemmStridedBatched(h, CUBLAS_OP_N, CUBLAS_OP_N, ld, ld, ld, &one, D, ld, st, A, ld, st, &zero, Bt, ld, st, nmol);
        cublasDgemmStridedBatched(h, CUBLAS_OP_N, CUBLAS_OP_N, ld, ld, ld, &one, Bt, ld, st, A, ld, st, &zero, C, ld, st, nmol);
        axpby_d_kernel<<<nb(ms), 256, 0, s>>>(ms, 3.0, Bt, -2.0, C, D);
    }
    cudaError_t e = cudaStreamSynchronize(s);
    cleanup();
    if (e != cudaSuccess) return cuda_fail(e, "cq_guess_density");
    return CQ_OK;
}
