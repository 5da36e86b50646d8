// One-electron integrals over contracted Cartesian Gaussians (Obara-Saika):
// overlap, kinetic energy, nuclear attraction and dipole-moment matrices,
// one thread per ordered shell pair.  They give the core Hamiltonian
// h = T + V of Eq. 2c_fock and the electric-dipole operator of the
// real-time perturbation (Sec. "Real-Time Electronic Dynamics").
//
//   1-D overlap:   S_{i+1,j} = X_PA S_ij + (i S_{i-1,j} + j S_{i,j-1}) / (2p)
//                  S_{i,j+1} = X_PB S_ij + (i S_{i-1,j} + j S_{i,j-1}) / (2p)
//                  S_00 = sqrt(pi/p) exp(-mu X_AB^2)
//   kinetic:       <i|d2/dx2|j> = j(j-1) S_{i,j-2} - 2b(2j+1) S_ij + 4b^2 S_{i,j+2}
//   dipole:        <i| x - C |j> = S_{i,j+1} + (B - C) S_ij
//   nuclear:       [a+1_i|b]^(m) = PA_i [a|b]^(m) - PC_i [a|b]^(m+1)
//                      + a_i/(2p) ([a-1_i|b]^(m) - [a-1_i|b]^(m+1)), built for b = 0,
//                  then (a|b+1_i) = (a+1_i|b) + AB_i (a|b);
//                  [0|0]^(m) = (2 pi / p) exp(-mu AB^2) F_m(p PC^2).
#include "cq_internal.h"

namespace cq {

__device__ __forceinline__ void boys_rt(int L, double T, double* F, const double* __restrict__ tab)
{
    switch (L) {
        case 0: boys<0>(T, F, tab); break;
        case 1: boys<1>(T, F, tab); break;
        case 2: boys<2>(T, F, tab); break;
        case 3: boys<3>(T, F, tab); break;
        default: boys<4>(T, F, tab); break;
    }
}

// index of a Cartesian exponent triple with total <= 4 in a 5x5x5 cube
__device__ __forceinline__ int cidx(int x, int y, int z) { return (x * 5 + y) * 5 + z; }

// One thread per (molecule, shell, shell) of the batched layout; each
// molecule sees only its own nuclei.
__global__ void one_electron_kernel(int nmol, int ld, int lds, const int* __restrict__ mol_nsh,
                                    const int* __restrict__ mol_sho, const int* __restrict__ mol_bfo,
                                    const int* __restrict__ mol_atom_off, const int* __restrict__ L,
                                    const int* __restrict__ np, const int* __restrict__ poff,
                                    const int* __restrict__ bfo, const double* __restrict__ ctr,
                                    const double* __restrict__ ex, const double* __restrict__ coef,
                                    const double* __restrict__ scale, const double* __restrict__ axyz,
                                    const double* __restrict__ Zc, const double* __restrict__ boys_tab, double ox,
                                    double oy, double oz, double* S, double* Tm, double* V, double* M)
{
    const size_t sslot = (size_t)lds * lds;
    const size_t p = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= sslot * nmol) return;
    const int mol = (int)(p / sslot);
    const int la_loc = (int)((p / lds) % lds), lb_loc = (int)(p % lds);
    if (la_loc >= mol_nsh[mol] || lb_loc >= mol_nsh[mol]) return;
    const int sa = mol_sho[mol] + la_loc, sb = mol_sho[mol] + lb_loc;
    const int a0 = mol_atom_off[mol], a1 = mol_atom_off[mol + 1];
    const size_t mbase = (size_t)mol * ld * ld, mstride = (size_t)nmol * ld * ld;
    const int f0 = mol_bfo[mol];
    const int la = L[sa], lb = L[sb];
    const int na = ncart(la), nb = ncart(lb);
    int ca[6][3], cb[6][3];
    {
        int c = 0;
        for (int x = la; x >= 0; --x)
            for (int y = la - x; y >= 0; --y, ++c) { ca[c][0] = x; ca[c][1] = y; ca[c][2] = la - x - y; }
        c = 0;
        for (int x = lb; x >= 0; --x)
            for (int y = lb - x; y >= 0; --y, ++c) { cb[c][0] = x; cb[c][1] = y; cb[c][2] = lb - x - y; }
    }
    const double* A = ctr + 3 * sa;
    const double* B = ctr + 3 * sb;
    const double O[3] = {ox, oy, oz};
    double s_acc[36], t_acc[36], v_acc[36], m_acc[3][36];
    for (int i = 0; i < na * nb; ++i) {
        s_acc[i] = t_acc[i] = v_acc[i] = 0.0;
        m_acc[0][i] = m_acc[1][i] = m_acc[2][i] = 0.0;
    }
    const double pi = 3.14159265358979323846;
    for (int i = 0; i < np[sa]; ++i)
        for (int j = 0; j < np[sb]; ++j) {
            const double a = ex[poff[sa] + i], b = ex[poff[sb] + j];
            const double pz = a + b, mu = a * b / pz, o2p = 0.5 / pz;
            const double cc = coef[poff[sa] + i] * coef[poff[sb] + j];
            double P[3], AB2 = 0.0;
            for (int x = 0; x < 3; ++x) {
                P[x] = (a * A[x] + b * B[x]) / pz;
                AB2 += (A[x] - B[x]) * (A[x] - B[x]);
            }
            // 1-D overlaps S[x][i][j], i <= la, j <= lb + 2
            double S1[3][3][5];
            for (int x = 0; x < 3; ++x) {
                const double XPA = P[x] - A[x], XPB = P[x] - B[x];
                const double XAB = A[x] - B[x];
                S1[x][0][0] = sqrt(pi / pz) * exp(-mu * XAB * XAB);
                for (int ii = 0; ii <= la; ++ii)
                    for (int jj = 0; jj <= lb + 2; ++jj) {
                        if (ii == 0 && jj == 0) continue;
                        double v;
                        if (jj == 0) {
                            v = XPA * S1[x][ii - 1][0];
                            if (ii > 1) v += o2p * (ii - 1) * S1[x][ii - 2][0];
                        } else {
                            v = XPB * S1[x][ii][jj - 1];
                            if (ii > 0) v += o2p * ii * S1[x][ii - 1][jj - 1];
                            if (jj > 1) v += o2p * (jj - 1) * S1[x][ii][jj - 2];
                        }
                        S1[x][ii][jj] = v;
                    }
            }
            // nuclear attraction: [e|0]^(m) for |e| <= la+lb, then HRR to (a|b)
            const int lt = la + lb;
            double Vt[125];  // (e|0) for each e, m = 0 after the recursion
            for (int k = 0; k < 125; ++k) Vt[k] = 0.0;
            for (int C = a0; C < a1; ++C) {
                double PC[3], PC2 = 0.0;
                for (int x = 0; x < 3; ++x) { PC[x] = P[x] - axyz[3 * C + x]; PC2 += PC[x] * PC[x]; }
                double F[5];
                boys_rt(lt, pz * PC2, F, boys_tab);
                const double pre = -Zc[C] * 2.0 * pi / pz * exp(-mu * AB2);
                // W[m][e]: build by increasing |e|
                double W[5][125];
                for (int m = 0; m <= lt; ++m) W[m][cidx(0, 0, 0)] = pre * F[m];
                for (int l = 1; l <= lt; ++l)
                    for (int x = l; x >= 0; --x)
                        for (int y = l - x; y >= 0; --y) {
                            const int z = l - x - y;
                            const int e[3] = {x, y, z};
                            int d = 0;
                            if (e[1] > e[d]) d = 1;
                            if (e[2] > e[d]) d = 2;
                            int e1[3] = {x, y, z};
                            e1[d] -= 1;
                            int e2[3] = {e1[0], e1[1], e1[2]};
                            e2[d] -= 1;
                            for (int m = 0; m <= lt - l; ++m) {
                                double v = (P[d] - A[d]) * W[m][cidx(e1[0], e1[1], e1[2])] -
                                           PC[d] * W[m + 1][cidx(e1[0], e1[1], e1[2])];
                                if (e1[d] > 0)
                                    v += e1[d] * o2p * (W[m][cidx(e2[0], e2[1], e2[2])] -
                                                        W[m + 1][cidx(e2[0], e2[1], e2[2])]);
                                W[m][cidx(x, y, z)] = v;
                            }
                        }
                for (int l = 0; l <= lt; ++l)
                    for (int x = l; x >= 0; --x)
                        for (int y = l - x; y >= 0; --y) Vt[cidx(x, y, l - x - y)] += W[0][cidx(x, y, l - x - y)];
            }
            for (int u = 0; u < na; ++u)
                for (int w = 0; w < nb; ++w) {
                    const int* ia = ca[u];
                    const int* ib = cb[w];
                    const double sx = S1[0][ia[0]][ib[0]], sy = S1[1][ia[1]][ib[1]], sz = S1[2][ia[2]][ib[2]];
                    double dd[3];
                    for (int x = 0; x < 3; ++x) {
                        const int jj = ib[x];
                        double v = -2.0 * b * (2 * jj + 1) * S1[x][ia[x]][jj] + 4.0 * b * b * S1[x][ia[x]][jj + 2];
                        if (jj >= 2) v += jj * (jj - 1) * S1[x][ia[x]][jj - 2];
                        dd[x] = v;
                    }
                    s_acc[u * nb + w] += cc * sx * sy * sz;
                    t_acc[u * nb + w] += cc * -0.5 * (dd[0] * sy * sz + sx * dd[1] * sz + sx * sy * dd[2]);
                    const double s3[3] = {sx, sy, sz};
                    for (int x = 0; x < 3; ++x) {
                        const double mx = S1[x][ia[x]][ib[x] + 1] + (B[x] - O[x]) * S1[x][ia[x]][ib[x]];
                        m_acc[x][u * nb + w] += cc * mx * s3[(x + 1) % 3] * s3[(x + 2) % 3];
                    }
                    // HRR (a|b) from (e|0): expand b's powers onto a with binomial shifts
                    // (x_B)^k = (x_A + AB)^k, exact for the axis-separable monomials
                    double v = 0.0;
                    for (int kx = 0; kx <= ib[0]; ++kx)
                        for (int ky = 0; ky <= ib[1]; ++ky)
                            for (int kz = 0; kz <= ib[2]; ++kz) {
                                const int bin[3][3] = {{1, 0, 0}, {1, 1, 0}, {1, 2, 1}};
                                double c = bin[ib[0]][kx] * bin[ib[1]][ky] * bin[ib[2]][kz];
                                c *= pow(A[0] - B[0], ib[0] - kx) * pow(A[1] - B[1], ib[1] - ky) *
                                     pow(A[2] - B[2], ib[2] - kz);
                                v += c * Vt[cidx(ia[0] + kx, ia[1] + ky, ia[2] + kz)];
                            }
                    v_acc[u * nb + w] += cc * v;
                }
        }
    for (int u = 0; u < na; ++u)
        for (int w = 0; w < nb; ++w) {
            const int r = bfo[sa] + u, c = bfo[sb] + w;
            const double f = scale[r] * scale[c];
            const size_t o = mbase + (size_t)(r - f0) * ld + (c - f0);
            if (S) S[o] = f * s_acc[u * nb + w];
            if (Tm) Tm[o] = f * t_acc[u * nb + w];
            if (V) V[o] = f * v_acc[u * nb + w];
            if (M)
                for (int x = 0; x < 3; ++x) M[(size_t)x * mstride + o] = f * m_acc[x][u * nb + w];
        }
}

}  // namespace cq

using namespace cq;

extern "C" int cq_one_electron(cq_basis* b, double* S, double* T, double* V, double* M, const double* origin,
                               void* stream)
{
    if (!b) { set_error("cq_one_electron: NULL basis"); return CQ_ERR_INVALID_ARG; }
    const double o[3] = {origin ? origin[0] : 0.0, origin ? origin[1] : 0.0, origin ? origin[2] : 0.0};
    cudaStream_t s = (cudaStream_t)stream;
    // padding elements of the batched layout are zero
    const size_t ms = (size_t)b->mstride;
    if (b->nmol > 1) {
        if (S) CQ_CUDA(cudaMemsetAsync(S, 0, ms * sizeof(double), s));
        if (T) CQ_CUDA(cudaMemsetAsync(T, 0, ms * sizeof(double), s));
        if (V) CQ_CUDA(cudaMemsetAsync(V, 0, ms * sizeof(double), s));
        if (M) CQ_CUDA(cudaMemsetAsync(M, 0, 3 * ms * sizeof(double), s));
    }
    const size_t nt = (size_t)b->nmol * b->lds * b->lds;
    one_electron_kernel<<<(unsigned)((nt + 63) / 64), 64, 0, s>>>(
        b->nmol, b->ld, b->lds, b->d_mol_nsh, b->d_mol_sho, b->d_mol_bfo, b->d_mol_atom_off, b->d_L, b->d_nprim,
        b->d_poff, b->d_bfo, b->d_ctr, b->d_exps, b->d_coef, b->d_scale, b->d_axyz, b->d_Z, b->d_boys, o[0], o[1],
        o[2], S, T, V, M);
    CQ_CUDA(cudaGetLastError());
    return CQ_OK;
}
