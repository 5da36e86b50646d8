// Basis set-up: shell normalisation, primitive-pair preparation, the Boys
// table and the Schwarz factors (direct-SCF integral screening).
#include <algorithm>
#include <climits>
#include <cmath>
#include <cstring>
#include <numeric>

#include "cq_internal.h"
#include "cq_jk.cuh"

namespace cq {

const int PC_L[NPC][2] = {{0, 0}, {1, 0}, {1, 1}, {2, 0}, {2, 1}, {2, 2}};

// kernel variant per class before tuning: in FP64 the warp-cooperative
// kernel for the classes with the largest recurrences, (dp|dp) (dd|pp)
// (dd|dp) (dd|dd); in FP32 the axis-permutation lane groups for every class
// of total angular momentum 6 or more; in double-float the axis-permutation
// kernel up to total angular momentum 5, the cooperative kernel on the
// screened list above, lane groups for the light classes
const int DEFAULT_VARIANT[NQC][3] = {{0, 0, 0}, {0, 0, 0}, {0, 0, 0}, {0, 0, 0}, {0, 0, 0}, {0, 0, 2}, {0, 0, 0},
                                     {0, 0, 0}, {0, 0, 2}, {0, 0, 2}, {0, 0, 0}, {0, 0, 2}, {0, 0, 2}, {0, 0, 2},
                                     {1, 2, 3}, {0, 0, 2}, {0, 0, 2}, {1, 2, 3}, {0, 2, 3}, {1, 2, 3}, {1, 2, 3}};

static thread_local std::string g_err;

void set_error(const std::string& msg) { g_err = msg; }

int cuda_fail(cudaError_t e, const char* what)
{
    g_err = std::string(what) + ": " + cudaGetErrorString(e);
    return e == cudaErrorMemoryAllocation ? CQ_ERR_OOM : CQ_ERR_CUDA;
}

// ---------------------------------------------------------------- kernels

// Boys table: row k holds F_m(T_k), T_k = k/16, m = 0..15 (FP64) and
// m = 0..12 (FP32), plus e^{-T_k}.  F_15 from the power series
//   F_m(T) = e^{-T} sum_i (2T)^i / ((2m+1)(2m+3)...(2m+2i+1)),
// lower orders by downward recursion.
__global__ void boys_table_kernel(double* tab, float* tabf)
{
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= BOYS_NT) return;
    const double T = k * 0.0625;
    const int mtop = 15;
    double term = 1.0 / (2 * mtop + 1), sum = term;
    for (int i = 1; i < 1000; ++i) {
        term *= 2.0 * T / (2 * mtop + 2 * i + 1);
        sum += term;
        if (term < 1e-19 * sum) break;
    }
    const double e = exp(-T);
    double F[16];
    F[mtop] = e * sum;
    for (int m = mtop - 1; m >= 0; --m) F[m] = (2.0 * T * F[m + 1] + e) / (2 * m + 1);
    for (int m = 0; m < 16; ++m) tab[k * BOYS_D_COLS + m] = F[m];
    tab[k * BOYS_D_COLS + BOYS_D_EXP] = e;
    tab[k * BOYS_D_COLS + BOYS_D_EXP + 1] = 0.0;
    for (int m = 0; m < BOYS_F_EXP; ++m) tabf[k * BOYS_F_COLS + m] = (float)F[m];
    tabf[k * BOYS_F_COLS + BOYS_F_EXP] = (float)e;
    df* tabx = reinterpret_cast<df*>(tabf + boys_x_offset());
    for (int m = 0; m < 16; ++m) tabx[k * BOYS_X_COLS + m] = df(F[m]);
    tabx[k * BOYS_X_COLS + BOYS_X_EXP] = df(e);
}

__device__ double dfact_odd(int n)  // (n)!! for odd n >= -1
{
    double r = 1.0;
    for (int k = n; k > 1; k -= 2) r *= k;
    return r;
}

// Contraction coefficients c_k N_L(alpha_k) / sqrt(S), N_L = (2a/pi)^{3/4}(4a)^{L/2},
// S the self-overlap of the x^L component (closed form of a same-centre
// Gaussian product: prod_x (2l-1)!!/(2p)^l * (pi/p)^{3/2}).
__global__ void normalize_kernel(int nsh, const int* L, const int* np, const int* poff,
                                 const double* ex, const double* co, double* out)
{
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= nsh) return;
    const int l = L[s], n = np[s], o = poff[s];
    const double pi = 3.14159265358979323846;
    for (int k = 0; k < n; ++k) {
        const double a = ex[o + k];
        out[o + k] = co[o + k] * pow(2.0 * a / pi, 0.75) * pow(4.0 * a, 0.5 * l);
    }
    double S = 0.0;
    for (int i = 0; i < n; ++i)
        for (int j = 0; j < n; ++j) {
            const double p = ex[o + i] + ex[o + j];
            S += out[o + i] * out[o + j] * dfact_odd(2 * l - 1) / pow(2.0 * p, (double)l) *
                 pow(pi / p, 1.5);
        }
    const double f = 1.0 / sqrt(S);
    for (int k = 0; k < n; ++k) out[o + k] *= f;
}

// Per-function factor of a Cartesian component relative to the x^L one:
// sqrt((2L-1)!! / ((2lx-1)!!(2ly-1)!!(2lz-1)!!)).
__global__ void scale_kernel(int nsh, const int* L, const int* bfo, double* scale)
{
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= nsh) return;
    const int l = L[s];
    int c = 0;
    for (int lx = l; lx >= 0; --lx)
        for (int ly = l - lx; ly >= 0; --ly, ++c) {
            const int lz = l - lx - ly;
            scale[bfo[s] + c] =
                sqrt(dfact_odd(2 * l - 1) / (dfact_odd(2 * lx - 1) * dfact_odd(2 * ly - 1) * dfact_odd(2 * lz - 1)));
        }
}

// Primitive-pair data, one thread per shell pair.
__global__ void pair_prep_kernel(int npair, const PairHdr* pairs, const double* ctr, const int* np,
                                 const int* poff, const double* ex, const double* coef, PrimPair* out,
                                 PrimPairF* outf, PrimPairX* outx)
{
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= npair) return;
    const PairHdr h = pairs[p];
    const double* A = ctr + 3 * h.a;
    const double* B = ctr + 3 * h.b;
    const double AB2 = h.AB[0] * h.AB[0] + h.AB[1] * h.AB[1] + h.AB[2] * h.AB[2];
    const double kfac = 1.4142135623730951 * pow(3.14159265358979323846, 1.25);  // sqrt(2) pi^{5/4}
    int q = h.poff;
    for (int i = 0; i < np[h.a]; ++i)
        for (int j = 0; j < np[h.b]; ++j, ++q) {
            const double a = ex[poff[h.a] + i], b = ex[poff[h.b] + j];
            const double z = a + b;
            PrimPair o;
            o.zeta = z;
            o.oo2z = 0.5 / z;
            for (int x = 0; x < 3; ++x) {
                o.P[x] = (a * A[x] + b * B[x]) / z;
                o.PA[x] = o.P[x] - A[x];
            }
            o.K = coef[poff[h.a] + i] * coef[poff[h.b] + j] * exp(-a * b / z * AB2) * kfac / z;
            o.pad[0] = o.pad[1] = o.pad[2] = 0.0;
            out[q] = o;
            PrimPairF f;
            f.zeta = (float)o.zeta; f.oo2z = (float)o.oo2z; f.K = (float)o.K;
            for (int x = 0; x < 3; ++x) { f.P[x] = (float)o.P[x]; f.PA[x] = (float)o.PA[x]; }
            f.pad[0] = f.pad[1] = f.pad[2] = 0.f;
            outf[q] = f;
            PrimPairX x;
            x.zeta = df(o.zeta); x.oo2z = df(o.oo2z); x.K = df(o.K);
            for (int c = 0; c < 3; ++c) { x.P[c] = df(o.P[c]); x.PA[c] = df(o.PA[c]); x.pad[c] = df(0.0); }
            outx[q] = x;
        }
}

}  // namespace cq

using namespace cq;

extern "C" const char* cq_last_error(void) { return cq::g_err.c_str(); }

static void free_basis(cq_basis* b)
{
    if (!b) return;
    dense_free(b);
    void* ptrs[] = {b->d_pass_qoff, b->d_boys, b->d_boysf, b->d_pairs, b->d_prims, b->d_primsf, b->d_primsx, b->d_tasks,
                    b->d_Qf, b->d_Qd, b->d_scale, b->d_ctr, b->d_L, b->d_nprim, b->d_poff,
                    b->d_bfo, b->d_exps, b->d_coef, b->d_axyz, b->d_Z, b->d_Dp, b->d_Jp,
                    b->d_Kp, b->d_Dmax, b->d_cnt, b->d_coop_tasks, b->d_qlist, b->d_qcount,
                    b->d_task_off, b->d_qoff, b->d_tcount, b->d_toff, b->d_mol_n, b->d_mol_bfo,
                    b->d_mol_nsh, b->d_mol_sho, b->d_mol_atom_off};
    for (void* p : ptrs)
        if (p) cudaFree(p);
    if (b->ev0) cudaEventDestroy(b->ev0);
    if (b->ev1) cudaEventDestroy(b->ev1);
    for (int q = 0; q < NQC; ++q)
        for (int p = 0; p < 3; ++p)
            for (int e = 0; e < 2; ++e)
                if (b->pev[q][p][e]) cudaEventDestroy(b->pev[q][p][e]);
    for (int q = 0; q < NQC; ++q)
        for (int p = 0; p < 3; ++p)
            for (cudaEvent_t ev : b->pev_pass[q][p]) cudaEventDestroy(ev);
    for (int k = 0; k < cq_basis::NSIDE; ++k) {
        if (b->side[k]) cudaStreamDestroy(b->side[k]);
        if (b->join_ev[k]) cudaEventDestroy(b->join_ev[k]);
    }
    if (b->fork_ev) cudaEventDestroy(b->fork_ev);
    if (b->batch_stream) cudaStreamDestroy(b->batch_stream);
    if (b->batch_ev) cudaEventDestroy(b->batch_ev);
    delete b;
}

template <typename T>
static int upload(T** d, const std::vector<T>& h)
{
    int rc = dalloc(d, h.size());
    if (rc) return rc;
    if (!h.empty()) CQ_CUDA(cudaMemcpy(*d, h.data(), h.size() * sizeof(T), cudaMemcpyHostToDevice));
    return CQ_OK;
}

static int create_impl(int natom, const double* xyz, const int* Z, const int* atom_mol, int nshell,
                       const int* shell_atom, const int* shell_L, const int* shell_nprim, const double* exps,
                       const double* coefs, cq_basis* b)
{
    CQ_CUDA(cudaGetDevice(&b->device));
    b->atom_mol.assign(natom, 0);
    if (atom_mol) b->atom_mol.assign(atom_mol, atom_mol + natom);
    for (int q = 0; q < NQC; ++q) {
        for (int p = 0; p < 3; ++p) b->variant[q][p] = DEFAULT_VARIANT[q][p];
    }
    b->natom = natom;
    b->nsh = nshell;
    b->xyz.assign(xyz, xyz + 3 * natom);
    b->Z.assign(Z, Z + natom);
    b->L.assign(shell_L, shell_L + nshell);
    b->nprim.assign(shell_nprim, shell_nprim + nshell);
    b->atom.assign(shell_atom, shell_atom + nshell);
    b->poff.resize(nshell);
    b->bfo.resize(nshell + 1);
    int np = 0, nbf = 0;
    for (int s = 0; s < nshell; ++s) {
        b->poff[s] = np;
        b->bfo[s] = nbf;
        np += b->nprim[s];
        nbf += ncart(b->L[s]);
    }
    b->bfo[nshell] = nbf;
    b->nbf = nbf;
    b->exps.assign(exps, exps + np);
    b->coefs.assign(coefs, coefs + np);

    // ---- molecules: atoms, shells and functions of each are contiguous
    {
        b->mol_atom_off.assign(1, 0);
        for (int a = 1; a < natom; ++a)
            if (b->atom_mol[a] != b->atom_mol[a - 1]) b->mol_atom_off.push_back(a);
        b->mol_atom_off.push_back(natom);
        b->nmol = (int)b->mol_atom_off.size() - 1;
        b->mol_sho.assign(b->nmol + 1, nshell);
        for (int s = nshell - 1; s >= 0; --s) b->mol_sho[b->atom_mol[b->atom[s]]] = s;
        for (int m = b->nmol - 1; m >= 0; --m)
            if (b->mol_sho[m] > b->mol_sho[m + 1]) b->mol_sho[m] = b->mol_sho[m + 1];
        b->mol_bfo.resize(b->nmol + 1);
        b->mol_n.resize(b->nmol);
        b->mol_nsh.resize(b->nmol);
        b->ld = b->lds = 1;
        for (int m = 0; m < b->nmol; ++m) {
            b->mol_bfo[m] = b->bfo[b->mol_sho[m]];
            b->mol_nsh[m] = b->mol_sho[m + 1] - b->mol_sho[m];
            b->mol_n[m] = b->bfo[b->mol_sho[m + 1]] - b->mol_bfo[m];
            b->ld = std::max(b->ld, b->mol_n[m]);
            b->lds = std::max(b->lds, b->mol_nsh[m]);
        }
        b->mol_bfo[b->nmol] = nbf;
        b->mstride = (long long)b->nmol * b->ld * b->ld;
    }

    // ---- shell pairs within each molecule, grouped by class, then molecule,
    // then sorted by primitive count
    std::vector<double> ctr(3 * nshell);
    for (int s = 0; s < nshell; ++s)
        for (int x = 0; x < 3; ++x) ctr[3 * s + x] = xyz[3 * b->atom[s] + x];
    const int nmol = b->nmol;
    std::vector<std::vector<PairHdr>> bycls(NPC * nmol);
    for (int m = 0; m < nmol; ++m)
        for (int a = b->mol_sho[m]; a < b->mol_sho[m + 1]; ++a)
            for (int c = b->mol_sho[m]; c <= a; ++c) {
                int s1 = a, s2 = c;
                if (b->L[s1] < b->L[s2]) std::swap(s1, s2);
                PairHdr h;
                h.a = s1; h.b = s2;
                h.bfa = b->bfo[s1] - b->mol_bfo[m]; h.bfb = b->bfo[s2] - b->mol_bfo[m];
                h.sa = s1 - b->mol_sho[m]; h.sb = s2 - b->mol_sho[m];
                h.mbase = (long long)m * b->ld * b->ld;
                h.smbase = (long long)m * b->lds * b->lds;
                h.nprim = b->nprim[s1] * b->nprim[s2];
                h.poff = 0;
                for (int x = 0; x < 3; ++x) h.AB[x] = ctr[3 * s1 + x] - ctr[3 * s2 + x];
                bycls[pc_of(b->L[s1], b->L[s2]) * nmol + m].push_back(h);
            }
    b->pairs.clear();
    b->molcls_off.assign(NPC * (nmol + 1), 0);
    for (int c = 0; c < NPC; ++c) {
        b->cls_off[c] = (int)b->pairs.size();
        for (int m = 0; m < nmol; ++m) {
            auto& v = bycls[c * nmol + m];
            std::stable_sort(v.begin(), v.end(), [](const PairHdr& x, const PairHdr& y) {
                if (x.nprim != y.nprim) return x.nprim > y.nprim;
                if (x.a != y.a) return x.a < y.a;
                return x.b < y.b;
            });
            b->molcls_off[c * (nmol + 1) + m] = (int)b->pairs.size();
            b->pairs.insert(b->pairs.end(), v.begin(), v.end());
        }
        b->molcls_off[c * (nmol + 1) + nmol] = (int)b->pairs.size();
    }
    b->cls_off[NPC] = (int)b->pairs.size();
    b->npair = (int)b->pairs.size();
    int q = 0;
    for (auto& h : b->pairs) { h.poff = q; q += h.nprim; }
    b->nprim_pairs = q;

    // ---- warp tasks per quartet class: (bra, ket candidates [j0, j1)) with
    // bra and kets of one molecule, costliest first.  The candidate range
    // per task shrinks for classes with few quartets so that every class
    // offers enough warps to fill the GPU (about 32 per SM).
    b->task_off.assign(NQC + 1, 0);
    b->qoff.assign(NQC + 1, 0);
    {   // candidate quartets over all classes decide the mode
        long long total = 0;
        for (int X = 0; X < NPC; ++X)
            for (int Y = 0; Y <= X; ++Y)
                for (int m = 0; m < nmol; ++m) {
                    const long long nbra = b->mol_range(X, m).second - b->mol_range(X, m).first;
                    const long long nket = b->mol_range(Y, m).second - b->mol_range(Y, m).first;
                    total += (X == Y) ? nbra * (nbra + 1) / 2 : nbra * nket;
                }
        b->passes = total > g_list_capacity;
        b->list_cap = b->passes ? g_list_capacity : total;
    }
    std::vector<int4> tasks;
    // prefix sums of primitive-pair counts over the pair array: the cost of
    // a task (bra i, kets [j0, j1)) is nprim_i * (pref[j1] - pref[j0])
    std::vector<long long> npref(b->pairs.size() + 1, 0);
    for (size_t j = 0; j < b->pairs.size(); ++j) npref[j + 1] = npref[j] + b->pairs[j].nprim;
    for (int X = 0, qc = 0; X < NPC; ++X)
        for (int Y = 0; Y <= X; ++Y, ++qc) {
            b->task_off[qc] = (int)tasks.size();
            long long cand = 0;
            for (int m = 0; m < nmol; ++m) {
                const long long nbra = b->mol_range(X, m).second - b->mol_range(X, m).first;
                const long long nket = b->mol_range(Y, m).second - b->mol_range(Y, m).first;
                cand += (X == Y) ? nbra * (nbra + 1) / 2 : nbra * nket;
            }
            b->qoff[qc + 1] = b->qoff[qc] + cand;
            int range = (int)std::min<long long>(JK_RANGE, std::max<long long>(4, cand / (152 * 32)));
            range = std::max(4, range & ~3);
            if (b->passes) range = INT_MAX;   // one task per bra pair
            std::vector<std::pair<double, int4>> tv;
            for (int m = 0; m < nmol; ++m) {
                const auto br = b->mol_range(X, m), kr = b->mol_range(Y, m);
                for (int i = br.first; i < br.second; ++i) {
                    const int jb = kr.first, je = (X == Y) ? i + 1 : kr.second;
                    for (int j0 = jb; j0 < je; j0 = (je - j0 > range) ? j0 + range : je) {
                        const int j1 = (je - j0 > range) ? j0 + range : je;
                        const double cost = (double)(npref[j1] - npref[j0]);
                        tv.push_back({cost * b->pairs[i].nprim, make_int4(i, j0, j1, 0)});
                    }
                }
            }
            std::stable_sort(tv.begin(), tv.end(),
                             [](const std::pair<double, int4>& x, const std::pair<double, int4>& y) {
                                 return x.first > y.first;
                             });
            for (auto& t : tv) tasks.push_back(t.second);
        }
    b->task_off[NQC] = (int)tasks.size();
    if (b->passes) {
        b->task_cand.assign(tasks.size() + 1, 0);
        for (size_t t = 0; t < tasks.size(); ++t) b->task_cand[t + 1] = b->task_cand[t] + (tasks[t].z - tasks[t].y);
    }

    // ---- device copies
    int rc;
    std::vector<double> axyz(xyz, xyz + 3 * natom), zc(Z, Z + natom);
    if ((rc = upload(&b->d_ctr, ctr))) return rc;
    if ((rc = upload(&b->d_L, b->L))) return rc;
    if ((rc = upload(&b->d_nprim, b->nprim))) return rc;
    if ((rc = upload(&b->d_poff, b->poff))) return rc;
    if ((rc = upload(&b->d_bfo, b->bfo))) return rc;
    if ((rc = upload(&b->d_exps, b->exps))) return rc;
    if ((rc = upload(&b->d_pairs, b->pairs))) return rc;
    if ((rc = upload(&b->d_tasks, tasks))) return rc;
    if ((rc = upload(&b->d_task_off, b->task_off))) return rc;
    if ((rc = upload(&b->d_qoff, b->qoff))) return rc;
    if ((rc = dalloc(&b->d_qlist, (size_t)b->list_cap))) return rc;
    if (b->passes) {
        std::vector<long long> pq = {0, b->list_cap};
        if ((rc = upload(&b->d_pass_qoff, pq))) return rc;
    }
    if ((rc = dalloc(&b->d_qcount, 3 * NQC))) return rc;
    if ((rc = dalloc(&b->d_tcount, 3 * tasks.size()))) return rc;
    if ((rc = dalloc(&b->d_toff, 3 * tasks.size()))) return rc;
    if ((rc = upload(&b->d_axyz, axyz))) return rc;
    if ((rc = upload(&b->d_mol_n, b->mol_n))) return rc;
    if ((rc = upload(&b->d_mol_bfo, b->mol_bfo))) return rc;
    if ((rc = upload(&b->d_mol_nsh, b->mol_nsh))) return rc;
    if ((rc = upload(&b->d_mol_sho, b->mol_sho))) return rc;
    if ((rc = upload(&b->d_mol_atom_off, b->mol_atom_off))) return rc;
    if ((rc = upload(&b->d_Z, zc))) return rc;
    if ((rc = dalloc(&b->d_coef, np))) return rc;
    if ((rc = dalloc(&b->d_scale, nbf))) return rc;
    if ((rc = dalloc(&b->d_prims, b->nprim_pairs))) return rc;
    if ((rc = dalloc(&b->d_primsf, b->nprim_pairs))) return rc;
    if ((rc = dalloc(&b->d_primsx, b->nprim_pairs))) return rc;
    if ((rc = dalloc(&b->d_boys, (size_t)BOYS_NT * BOYS_D_COLS))) return rc;
    if ((rc = dalloc(&b->d_boysf, boys_x_offset() + (size_t)2 * BOYS_NT * BOYS_X_COLS))) return rc;
    if ((rc = dalloc(&b->d_Qf, b->npair))) return rc;
    if ((rc = dalloc(&b->d_Qd, b->npair))) return rc;
    if ((rc = dalloc(&b->d_cnt, CNT_WORDS))) return rc;
    {
        std::vector<double> coefs_raw(coefs, coefs + np);
        double* d_raw = nullptr;
        if ((rc = upload(&d_raw, coefs_raw))) return rc;
        normalize_kernel<<<(nshell + 127) / 128, 128>>>(nshell, b->d_L, b->d_nprim, b->d_poff, b->d_exps,
                                                      d_raw, b->d_coef);
        cudaError_t e = cudaDeviceSynchronize();
        cudaFree(d_raw);
        CQ_CUDA(e);
    }
    scale_kernel<<<(nshell + 127) / 128, 128>>>(nshell, b->d_L, b->d_bfo, b->d_scale);
    boys_table_kernel<<<(BOYS_NT + 127) / 128, 128>>>(b->d_boys, b->d_boysf);
    pair_prep_kernel<<<(b->npair + 127) / 128, 128>>>(b->npair, b->d_pairs, b->d_ctr, b->d_nprim,
                                                      b->d_poff, b->d_exps, b->d_coef, b->d_prims,
                                                      b->d_primsf, b->d_primsx);
    CQ_CUDA(cudaGetLastError());
    CQ_CUDA(cudaEventCreate(&b->ev0));
    CQ_CUDA(cudaEventCreate(&b->ev1));
    CQ_CUDA(cudaEventCreateWithFlags(&b->fork_ev, cudaEventDisableTiming));
    for (int k = 0; k < cq_basis::NSIDE; ++k) {
        CQ_CUDA(cudaStreamCreateWithFlags(&b->side[k], cudaStreamNonBlocking));
        CQ_CUDA(cudaEventCreateWithFlags(&b->join_ev[k], cudaEventDisableTiming));
    }
    rc = cq_schwarz(b, nullptr, nullptr);
    if (rc) return rc;
    rc = ensure_coop_tasks(b);
    if (rc) return rc;
    CQ_CUDA(cudaDeviceSynchronize());
    return CQ_OK;
}

namespace cq {
// (bra, ket, [p0, p1)) for every candidate quartet of the classes that use
// the cooperative kernel, split into chunks of at most COOP_CHUNK primitive
// quartets; costliest first within a class.
int ensure_coop_tasks(cq_basis* b)
{
    if (!b->coop_dirty) return CQ_OK;
    std::vector<int4> tasks;
    b->coop_off.assign(NQC + 1, 0);
    // Large bases: the cooperative kernel reads the screened quartet lists
    // (one warp per quartet, all its primitives) instead of a task per
    // candidate quartet and primitive chunk, whose table would grow with
    // the candidate count.
    long long cand = 0;
    for (int X = 0, qc = 0; X < NPC; ++X)
        for (int Y = 0; Y <= X; ++Y, ++qc) {
            if (b->variant[qc][0] != VARIANT_COOP && b->variant[qc][1] != VARIANT_COOP) continue;
            for (int m = 0; m < b->nmol; ++m) {
                const long long nbra = b->mol_range(X, m).second - b->mol_range(X, m).first;
                const long long nket = b->mol_range(Y, m).second - b->mol_range(Y, m).first;
                cand += (X == Y) ? nbra * (nbra + 1) / 2 : nbra * nket;
            }
        }
    b->coop_list = b->passes || cand > COOP_TASK_CANDIDATES;
    if (b->coop_list) {
        if (b->d_coop_tasks) cudaFree(b->d_coop_tasks);
        b->d_coop_tasks = nullptr;
        b->coop_dirty = false;
        return CQ_OK;
    }
    for (int X = 0, qc = 0; X < NPC; ++X)
        for (int Y = 0; Y <= X; ++Y, ++qc) {
            b->coop_off[qc] = (int)tasks.size();
            if (b->variant[qc][0] != VARIANT_COOP && b->variant[qc][1] != VARIANT_COOP) continue;
            std::vector<std::pair<int, int4>> tv;
            for (int m = 0; m < b->nmol; ++m)
            for (int i = b->mol_range(X, m).first; i < b->mol_range(X, m).second; ++i) {
                const int jb = b->mol_range(Y, m).first, je = (X == Y) ? i + 1 : b->mol_range(Y, m).second;
                for (int j = jb; j < je; ++j) {
                    const int np = b->pairs[i].nprim * b->pairs[j].nprim;
                    for (int p0 = 0; p0 < np; p0 += COOP_CHUNK) {
                        const int p1 = std::min(np, p0 + COOP_CHUNK);
                        tv.push_back({p1 - p0, make_int4(i, j, p0, p1)});
                    }
                }
            }
            std::stable_sort(tv.begin(), tv.end(), [](const std::pair<int, int4>& x, const std::pair<int, int4>& y) {
                return x.first > y.first;
            });
            for (auto& t : tv) tasks.push_back(t.second);
        }
    b->coop_off[NQC] = (int)tasks.size();
    if (b->d_coop_tasks) cudaFree(b->d_coop_tasks);
    b->d_coop_tasks = nullptr;
    int rc = dalloc(&b->d_coop_tasks, tasks.size());
    if (rc) return rc;
    if (!tasks.empty())
        CQ_CUDA(cudaMemcpy(b->d_coop_tasks, tasks.data(), tasks.size() * sizeof(int4), cudaMemcpyHostToDevice));
    b->coop_dirty = false;
    return CQ_OK;
}
}  // namespace cq

static int create_checked(int natom, const double* xyz, const int* Z, const int* atom_mol, int nshell,
                          const int* shell_atom, const int* shell_L, const int* shell_nprim, const double* exps,
                          const double* coefs, cq_basis** out);

extern "C" int cq_basis_create(int natom, const double* xyz, const int* Z, int nshell,
                               const int* shell_atom, const int* shell_L, const int* shell_nprim,
                               const double* exps, const double* coefs, cq_basis** out)
{
    return create_checked(natom, xyz, Z, nullptr, nshell, shell_atom, shell_L, shell_nprim, exps, coefs, out);
}

extern "C" int cq_basis_create_batch(int natom, const double* xyz, const int* Z, const int* atom_mol, int nshell,
                                     const int* shell_atom, const int* shell_L, const int* shell_nprim,
                                     const double* exps, const double* coefs, cq_basis** out)
{
    if (!atom_mol) { set_error("cq_basis_create_batch: atom_mol is NULL"); return CQ_ERR_INVALID_ARG; }
    for (int a = 0; a < natom; ++a) {
        if (atom_mol[a] < 0 || (a > 0 && atom_mol[a] != atom_mol[a - 1] && atom_mol[a] != atom_mol[a - 1] + 1) ||
            (a == 0 && atom_mol[0] != 0)) {
            set_error("cq_basis_create_batch: atom_mol must be 0,..,0,1,..,1,... (consecutive molecule ids)");
            return CQ_ERR_INVALID_ARG;
        }
    }
    for (int s = 1; s < nshell; ++s)
        if (shell_atom && shell_atom[s] >= 0 && shell_atom[s] < natom && shell_atom[s - 1] >= 0 &&
            shell_atom[s - 1] < natom && atom_mol[shell_atom[s]] < atom_mol[shell_atom[s - 1]]) {
            set_error("cq_basis_create_batch: shells must be ordered by molecule");
            return CQ_ERR_INVALID_ARG;
        }
    return create_checked(natom, xyz, Z, atom_mol, nshell, shell_atom, shell_L, shell_nprim, exps, coefs, out);
}

static int create_checked(int natom, const double* xyz, const int* Z, const int* atom_mol, int nshell,
                          const int* shell_atom, const int* shell_L, const int* shell_nprim, const double* exps,
                          const double* coefs, cq_basis** out)
{
    if (!out) { set_error("cq_basis_create: out is NULL"); return CQ_ERR_INVALID_ARG; }
    *out = nullptr;
    if (natom <= 0 || nshell <= 0 || !xyz || !Z || !shell_atom || !shell_L || !shell_nprim || !exps ||
        !coefs) {
        set_error("cq_basis_create: empty basis or NULL argument");
        return CQ_ERR_INVALID_ARG;
    }
    int np = 0;
    for (int s = 0; s < nshell; ++s) {
        if (shell_L[s] < 0 || shell_L[s] > LMAX) {
            set_error("cq_basis_create: shell angular momentum outside 0..2");
            return CQ_ERR_INVALID_ARG;
        }
        if (shell_nprim[s] < 1 || shell_nprim[s] > MAX_PRIM) {
            set_error("cq_basis_create: primitive count outside 1..16");
            return CQ_ERR_INVALID_ARG;
        }
        if (shell_atom[s] < 0 || shell_atom[s] >= natom) {
            set_error("cq_basis_create: shell_atom out of range");
            return CQ_ERR_INVALID_ARG;
        }
        np += shell_nprim[s];
    }
    for (int k = 0; k < np; ++k)
        if (!(exps[k] > 0.0) || !std::isfinite(exps[k]) || !std::isfinite(coefs[k])) {
            set_error("cq_basis_create: exponents must be positive and finite");
            return CQ_ERR_INVALID_ARG;
        }
    for (int k = 0; k < 3 * natom; ++k)
        if (!std::isfinite(xyz[k])) {
            set_error("cq_basis_create: non-finite coordinate");
            return CQ_ERR_INVALID_ARG;
        }
    cq_basis* b = new cq_basis();
    int rc = create_impl(natom, xyz, Z, atom_mol, nshell, shell_atom, shell_L, shell_nprim, exps, coefs, b);
    if (rc) { free_basis(b); return rc; }
    *out = b;
    return CQ_OK;
}

extern "C" void cq_basis_destroy(cq_basis* b)
{
    if (b) cudaDeviceSynchronize();
    free_basis(b);
}

extern "C" int cq_basis_layout(const cq_basis* b, int* nmol, int* ld, int* mol_n)
{
    if (!b) { set_error("cq_basis_layout: NULL basis"); return CQ_ERR_INVALID_ARG; }
    if (nmol) *nmol = b->nmol;
    if (ld) *ld = b->ld;
    if (mol_n)
        for (int m = 0; m < b->nmol; ++m) mol_n[m] = b->mol_n[m];
    return CQ_OK;
}

extern "C" int cq_basis_info(const cq_basis* b, int* nbf, int* nshell, int* npair)
{
    if (!b) { set_error("cq_basis_info: NULL basis"); return CQ_ERR_INVALID_ARG; }
    if (nbf) *nbf = b->nbf;
    if (nshell) *nshell = b->nsh;
    if (npair) *npair = b->npair;
    return CQ_OK;
}

// Boys values F_0..F_mmax at n arguments with the same device functions the
// integral kernels use (FP64, or FP32 with FP64 below the first table
// interval); results widened to FP64, row-major n x (mmax + 1).
template <typename R>
__global__ void boys_eval_kernel(int mmax, int n, const double* __restrict__ T, const double* __restrict__ tabd,
                                 const float* __restrict__ tabf, double* __restrict__ F)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const R t = (R)T[i];
    R f[LTOT_MAX + 1];
    switch (mmax) {
        case 0: boys_q<0>(t, f, tabd, tabf); break;
        case 1: boys_q<1>(t, f, tabd, tabf); break;
        case 2: boys_q<2>(t, f, tabd, tabf); break;
        case 3: boys_q<3>(t, f, tabd, tabf); break;
        case 4: boys_q<4>(t, f, tabd, tabf); break;
        case 5: boys_q<5>(t, f, tabd, tabf); break;
        case 6: boys_q<6>(t, f, tabd, tabf); break;
        case 7: boys_q<7>(t, f, tabd, tabf); break;
        default: boys_q<8>(t, f, tabd, tabf); break;
    }
    for (int m = 0; m <= mmax; ++m) F[(size_t)i * (mmax + 1) + m] = (double)f[m];
}

extern "C" int cq_boys(const cq_basis* b, int fp32, int mmax, int n, const double* T, double* F, void* stream)
{
    if (!b || (n > 0 && (!T || !F)) || mmax < 0 || mmax > LTOT_MAX || n < 0 || fp32 < 0 || fp32 > 2) {
        set_error("cq_boys: bad argument");
        return CQ_ERR_INVALID_ARG;
    }
    if (n == 0) return CQ_OK;
    cudaStream_t s = (cudaStream_t)stream;
    const int blocks = (n + 127) / 128;
    if (fp32 == 2) boys_eval_kernel<df><<<blocks, 128, 0, s>>>(mmax, n, T, b->d_boys, b->d_boysf, F);
    else if (fp32) boys_eval_kernel<float><<<blocks, 128, 0, s>>>(mmax, n, T, b->d_boys, b->d_boysf, F);
    else boys_eval_kernel<double><<<blocks, 128, 0, s>>>(mmax, n, T, b->d_boys, b->d_boysf, F);
    CQ_CUDA(cudaGetLastError());
    return CQ_OK;
}

__global__ void schwarz_square_kernel(int npair, const PairHdr* pairs, const double* Qd, int nsh, double* Q)
{
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= npair) return;
    const PairHdr h = pairs[p];
    Q[(size_t)h.a * nsh + h.b] = Qd[p];
    Q[(size_t)h.b * nsh + h.a] = Qd[p];
}

extern "C" int cq_schwarz(cq_basis* b, double* Q, void* stream)
{
    if (!b) { set_error("cq_schwarz: NULL basis"); return CQ_ERR_INVALID_ARG; }
    cudaStream_t s = (cudaStream_t)stream;
    JKArgs a;
    memset(&a, 0, sizeof a);
    a.pairs = b->d_pairs; a.prims = b->d_prims; a.primsf = b->d_primsf;
    a.boys_d = b->d_boys; a.boys_f = b->d_boysf;
    for (int c = 0; c < NPC; ++c) {
        const int beg = b->cls_off[c], end = b->cls_off[c + 1];
        if (end > beg) SCHWARZ_LAUNCH[c](a, beg, end, b->d_Qf, b->d_Qd, s);
    }
    CQ_CUDA(cudaGetLastError());
    if (Q && b->nmol > 1) {
        set_error("cq_schwarz: the nshell x nshell table is only available for a single-molecule basis");
        return CQ_ERR_UNSUPPORTED;
    }
    if (Q) {
        schwarz_square_kernel<<<(b->npair + 127) / 128, 128, 0, s>>>(b->npair, b->d_pairs, b->d_Qd, b->nsh, Q);
        CQ_CUDA(cudaGetLastError());
    }
    return CQ_OK;
}

extern "C" int cq_nuclear_repulsion_batch(const cq_basis* b, double* E)
{
    if (!b || !E) { set_error("cq_nuclear_repulsion: NULL argument"); return CQ_ERR_INVALID_ARG; }
    for (int m = 0; m < b->nmol; ++m) {
        double e = 0.0;
        for (int i = b->mol_atom_off[m]; i < b->mol_atom_off[m + 1]; ++i)
            for (int j = b->mol_atom_off[m]; j < i; ++j) {
                const double dx = b->xyz[3 * i] - b->xyz[3 * j], dy = b->xyz[3 * i + 1] - b->xyz[3 * j + 1],
                             dz = b->xyz[3 * i + 2] - b->xyz[3 * j + 2];
                e += (double)b->Z[i] * b->Z[j] / std::sqrt(dx * dx + dy * dy + dz * dz);
            }
        E[m] = e;
    }
    return CQ_OK;
}

extern "C" int cq_nuclear_repulsion(const cq_basis* b, double* E)
{
    if (!b || !E) { set_error("cq_nuclear_repulsion: NULL argument"); return CQ_ERR_INVALID_ARG; }
    std::vector<double> e(b->nmol);
    int rc = cq_nuclear_repulsion_batch(b, e.data());
    if (rc) return rc;
    double t = 0.0;
    for (double x : e) t += x;
    *E = t;
    return CQ_OK;
}
