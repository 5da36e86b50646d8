/*
 * Oracle -- test infrastructure only.  Plain, slow FP64 CPU reference for
 * the integrals and the Coulomb/exchange contraction of the Hartree-Fock
 * Fock matrix (Sec. "Reference Wave Functions", Eq. 2c_fock).  Only the
 * tests, __graft_entry__.smoke() and bench.py's cpu_baseline leg may load
 * it; the product path never does.
 *
 * Algorithms (deliberately different from the GPU path):
 *   - Boys function: power series for T < 30, erf + upward recursion above.
 *   - All integrals by McMurchie-Davidson Hermite expansion (Hermite
 *     coefficients E^{ij}_t by their three-term recurrence, Hermite Coulomb
 *     integrals R^n_{tuv} by their recursion from Boys values).
 *   - Basis functions: Cartesian, lexicographic component order
 *     (x..; xx,xy,xz,yy,yz,zz); primitive norm (2a/pi)^{3/4}(4a)^{L/2},
 *     then every Cartesian component of the contracted function is scaled
 *     to unit self-overlap.
 *   - J/K: every permutationally unique function quartet is visited once and
 *     each of its distinct index permutations is applied explicitly; no
 *     screening and no degeneracy factors.
 *
 * Definitions used throughout (real integrals, general real density D):
 *   J_{mn} = sum_{ls} (mn|ls) D_{ls},   K_{mn} = sum_{ls} (ml|sn) D_{ls}.
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define LMAX 2
#define LTOT (4 * LMAX)
#define NR (LTOT + 1)

typedef struct {
    int nsh, nbf;
    const double *ctr;   /* 3*nsh */
    const int *L, *np, *poff;
    const double *ex, *co;
    int *bfo;            /* basis function offset per shell */
    double *pn;          /* primitive-normalised coefficients */
    double *f;           /* per-function renormalisation to S_mm = 1 */
} Basis;

static const int NCART[3] = {1, 3, 6};
static const int CART[3][6][3] = {
    {{0, 0, 0}},
    {{1, 0, 0}, {0, 1, 0}, {0, 0, 1}},
    {{2, 0, 0}, {1, 1, 0}, {1, 0, 1}, {0, 2, 0}, {0, 1, 1}, {0, 0, 2}}};

/* ---------------- Boys function ---------------- */
void or_boys(int mmax, double T, double *F)
{
    if (T < 30.0) {
        double e = exp(-T);
        for (int m = 0; m <= mmax; ++m) {
            double term = 1.0 / (2 * m + 1), sum = term;
            for (int i = 1; i < 2000; ++i) {
                term *= 2.0 * T / (2 * m + 2 * i + 1);
                sum += term;
                if (term < 1e-18 * sum) break;
            }
            F[m] = e * sum;
        }
    } else {
        double e = exp(-T);
        F[0] = 0.5 * sqrt(M_PI / T) * erf(sqrt(T));
        for (int m = 0; m < mmax; ++m)
            F[m + 1] = ((2 * m + 1) * F[m] - e) / (2.0 * T);
    }
}

/* ---------------- Hermite expansion coefficients ---------------- */
/* E[i][j][t] for 0<=i<=la, 0<=j<=lb, 0<=t<=i+j; one Cartesian direction. */
static void hermite_E(int la, int lb, double a, double b, double Ax, double Bx,
                      double E[LMAX + 2][LMAX + 2][2 * LMAX + 4])
{
    double p = a + b, mu = a * b / p, X = Ax - Bx;
    double XPA = -b / p * X, XPB = a / p * X, o2p = 0.5 / p;
    memset(E, 0, sizeof(double) * (LMAX + 2) * (LMAX + 2) * (2 * LMAX + 4));
    E[0][0][0] = exp(-mu * X * X);
    for (int i = 0; i <= la; ++i)
        for (int j = 0; j <= lb; ++j) {
            if (i == 0 && j == 0) continue;
            for (int t = 0; t <= i + j; ++t) {
                double v;
                if (i > 0) {
                    v = XPA * E[i - 1][j][t];
                    if (t > 0) v += o2p * E[i - 1][j][t - 1];
                    if (t + 1 <= i - 1 + j) v += (t + 1) * E[i - 1][j][t + 1];
                } else {
                    v = XPB * E[i][j - 1][t];
                    if (t > 0) v += o2p * E[i][j - 1][t - 1];
                    if (t + 1 <= i + j - 1) v += (t + 1) * E[i][j - 1][t + 1];
                }
                E[i][j][t] = v;
            }
        }
}

/* Hermite Coulomb integrals R_{tuv} = R^0_{tuv}(p, PC) for t+u+v <= L. */
static void hermite_R(int L, double p, double X, double Y, double Z,
                      double R[NR][NR][NR])
{
    static __thread double Rn[NR + 1][NR][NR][NR];
    double F[NR + 1];
    or_boys(L, p * (X * X + Y * Y + Z * Z), F);
    double m2p = 1.0;
    for (int n = 0; n <= L; ++n) {
        Rn[n][0][0][0] = m2p * F[n];
        m2p *= -2.0 * p;
    }
    for (int n = L - 1; n >= 0; --n)
        for (int s = 1; s <= L - n; ++s)
            for (int t = 0; t <= s; ++t)
                for (int u = 0; u <= s - t; ++u) {
                    int v = s - t - u;
                    double r;
                    if (t > 0) {
                        r = X * Rn[n + 1][t - 1][u][v];
                        if (t > 1) r += (t - 1) * Rn[n + 1][t - 2][u][v];
                    } else if (u > 0) {
                        r = Y * Rn[n + 1][t][u - 1][v];
                        if (u > 1) r += (u - 1) * Rn[n + 1][t][u - 2][v];
                    } else {
                        r = Z * Rn[n + 1][t][u][v - 1];
                        if (v > 1) r += (v - 1) * Rn[n + 1][t][u][v - 2];
                    }
                    Rn[n][t][u][v] = r;
                }
    for (int t = 0; t <= L; ++t)
        for (int u = 0; u <= L - t; ++u)
            for (int v = 0; v <= L - t - u; ++v) R[t][u][v] = Rn[0][t][u][v];
}

/* ---------------- basis set-up and normalisation ---------------- */
typedef double Eab[3][LMAX + 2][LMAX + 2][2 * LMAX + 4];

static void overlap_block(const Basis *B, int a, int b, double *out);

static void basis_init(Basis *B, int nsh, const double *ctr, const int *L,
                       const int *np, const int *poff, const double *ex,
                       const double *co)
{
    B->nsh = nsh; B->ctr = ctr; B->L = L; B->np = np; B->poff = poff;
    B->ex = ex; B->co = co;
    B->bfo = (int *)malloc(sizeof(int) * (nsh + 1));
    int o = 0, npt = 0;
    for (int s = 0; s < nsh; ++s) {
        B->bfo[s] = o;
        o += NCART[L[s]];
        if (poff[s] + np[s] > npt) npt = poff[s] + np[s];
    }
    B->bfo[nsh] = o;
    B->nbf = o;
    B->pn = (double *)malloc(sizeof(double) * (npt > 0 ? npt : 1));
    for (int s = 0; s < nsh; ++s)
        for (int k = 0; k < np[s]; ++k) {
            double a = ex[poff[s] + k];
            B->pn[poff[s] + k] = co[poff[s] + k] * pow(2.0 * a / M_PI, 0.75) *
                                 pow(4.0 * a, 0.5 * L[s]);
        }
    B->f = (double *)malloc(sizeof(double) * o);
    for (int i = 0; i < o; ++i) B->f[i] = 1.0;
    double blk[36];
    for (int s = 0; s < nsh; ++s) {
        overlap_block(B, s, s, blk);
        int n = NCART[L[s]];
        for (int i = 0; i < n; ++i) B->f[B->bfo[s] + i] = 1.0 / sqrt(blk[i * n + i]);
    }
}

static void basis_free(Basis *B)
{
    free(B->bfo); free(B->pn); free(B->f);
}

/* Hermite coefficients of one primitive pair in x, y, z. */
static void pair_E(const Basis *B, int a, int b, double ea, double eb, Eab E)
{
    for (int x = 0; x < 3; ++x)
        hermite_E(B->L[a], B->L[b], ea, eb, B->ctr[3 * a + x], B->ctr[3 * b + x], E[x]);
}

/* ---------------- one-electron integrals ---------------- */
/* Overlap block (un-renormalised, i.e. before the per-function factor f). */
static void overlap_block(const Basis *B, int a, int b, double *out)
{
    int la = B->L[a], lb = B->L[b], na = NCART[la], nb = NCART[lb];
    memset(out, 0, sizeof(double) * na * nb);
    Eab E;
    for (int i = 0; i < B->np[a]; ++i)
        for (int j = 0; j < B->np[b]; ++j) {
            double ea = B->ex[B->poff[a] + i], eb = B->ex[B->poff[b] + j];
            double p = ea + eb, c = B->pn[B->poff[a] + i] * B->pn[B->poff[b] + j];
            pair_E(B, a, b, ea, eb, E);
            double s3 = pow(M_PI / p, 1.5);
            for (int m = 0; m < na; ++m)
                for (int n = 0; n < nb; ++n) {
                    const int *u = CART[la][m], *v = CART[lb][n];
                    out[m * nb + n] += c * s3 * E[0][u[0]][v[0]][0] *
                                       E[1][u[1]][v[1]][0] * E[2][u[2]][v[2]][0];
                }
        }
}

/* 1-D overlap of x_A^i x_B^j Gaussians (no sqrt(pi/p) factor) for j up to lb+2,
 * used by the kinetic-energy integral. */
static double ov1d(int i, int j, double a, double b, double A, double Bx)
{
    double E[LMAX + 2][LMAX + 4][2 * LMAX + 6];
    double p = a + b, mu = a * b / p, X = A - Bx;
    double XPA = -b / p * X, XPB = a / p * X, o2p = 0.5 / p;
    memset(E, 0, sizeof E);
    E[0][0][0] = exp(-mu * X * X);
    for (int ii = 0; ii <= i; ++ii)
        for (int jj = 0; jj <= j; ++jj) {
            if (ii == 0 && jj == 0) continue;
            for (int t = 0; t <= ii + jj; ++t) {
                double v;
                if (ii > 0) {
                    v = XPA * E[ii - 1][jj][t];
                    if (t > 0) v += o2p * E[ii - 1][jj][t - 1];
                    if (t + 1 <= ii - 1 + jj) v += (t + 1) * E[ii - 1][jj][t + 1];
                } else {
                    v = XPB * E[ii][jj - 1][t];
                    if (t > 0) v += o2p * E[ii][jj - 1][t - 1];
                    if (t + 1 <= ii + jj - 1) v += (t + 1) * E[ii][jj - 1][t + 1];
                }
                E[ii][jj][t] = v;
            }
        }
    return E[i][j][0] * sqrt(M_PI / p);
}

/* kind: 0 overlap, 1 kinetic, 2 nuclear attraction, 3..5 dipole x,y,z
 * (moment about origin O; no electron charge sign). */
static void one_block(const Basis *B, int kind, int a, int b, int natom,
                      const double *axyz, const double *Zc, const double *O,
                      double *out)
{
    int la = B->L[a], lb = B->L[b], na = NCART[la], nb = NCART[lb];
    memset(out, 0, sizeof(double) * na * nb);
    const double *A = B->ctr + 3 * a, *Bc = B->ctr + 3 * b;
    for (int i = 0; i < B->np[a]; ++i)
        for (int j = 0; j < B->np[b]; ++j) {
            double ea = B->ex[B->poff[a] + i], eb = B->ex[B->poff[b] + j];
            double p = ea + eb, c = B->pn[B->poff[a] + i] * B->pn[B->poff[b] + j];
            double P[3];
            for (int x = 0; x < 3; ++x) P[x] = (ea * A[x] + eb * Bc[x]) / p;
            Eab E;
            pair_E(B, a, b, ea, eb, E);
            for (int m = 0; m < na; ++m)
                for (int n = 0; n < nb; ++n) {
                    const int *u = CART[la][m], *v = CART[lb][n];
                    double val = 0.0;
                    if (kind == 0) {
                        val = pow(M_PI / p, 1.5) * E[0][u[0]][v[0]][0] *
                              E[1][u[1]][v[1]][0] * E[2][u[2]][v[2]][0];
                    } else if (kind == 1) {
                        double S[3], D[3];
                        for (int x = 0; x < 3; ++x) {
                            int ii = u[x], jj = v[x];
                            S[x] = ov1d(ii, jj, ea, eb, A[x], Bc[x]);
                            double d = -2.0 * eb * (2 * jj + 1) * S[x] +
                                       4.0 * eb * eb * ov1d(ii, jj + 2, ea, eb, A[x], Bc[x]);
                            if (jj >= 2) d += jj * (jj - 1) * ov1d(ii, jj - 2, ea, eb, A[x], Bc[x]);
                            D[x] = d;
                        }
                        val = -0.5 * (D[0] * S[1] * S[2] + S[0] * D[1] * S[2] +
                                      S[0] * S[1] * D[2]);
                    } else if (kind == 2) {
                        int lt = u[0] + v[0] + u[1] + v[1] + u[2] + v[2];
                        double R[NR][NR][NR];
                        for (int C = 0; C < natom; ++C) {
                            hermite_R(lt, p, P[0] - axyz[3 * C], P[1] - axyz[3 * C + 1],
                                      P[2] - axyz[3 * C + 2], R);
                            double s = 0.0;
                            for (int t = 0; t <= u[0] + v[0]; ++t)
                                for (int uu = 0; uu <= u[1] + v[1]; ++uu)
                                    for (int w = 0; w <= u[2] + v[2]; ++w)
                                        s += E[0][u[0]][v[0]][t] * E[1][u[1]][v[1]][uu] *
                                             E[2][u[2]][v[2]][w] * R[t][uu][w];
                            val -= Zc[C] * 2.0 * M_PI / p * s;
                        }
                    } else {
                        int d = kind - 3;
                        double f3 = pow(M_PI / p, 1.5);
                        double m1 = E[d][u[d]][v[d]][1] + (P[d] - O[d]) * E[d][u[d]][v[d]][0];
                        double o1 = E[(d + 1) % 3][u[(d + 1) % 3]][v[(d + 1) % 3]][0];
                        double o2 = E[(d + 2) % 3][u[(d + 2) % 3]][v[(d + 2) % 3]][0];
                        val = f3 * m1 * o1 * o2;
                    }
                    out[m * nb + n] += c * val;
                }
        }
}

/* ---------------- two-electron integrals ---------------- */
/* Contracted shell quartet (ab|cd), un-renormalised, layout [m][n][l][s]. */
static void eri_block(const Basis *B, int a, int b, int c, int d, double *out)
{
    int la = B->L[a], lb = B->L[b], lc = B->L[c], ld = B->L[d];
    int na = NCART[la], nb = NCART[lb], nc = NCART[lc], nd = NCART[ld];
    int Lt = la + lb + lc + ld;
    memset(out, 0, sizeof(double) * na * nb * nc * nd);
    const double *A = B->ctr + 3 * a, *Bc = B->ctr + 3 * b;
    const double *C = B->ctr + 3 * c, *D = B->ctr + 3 * d;
    double R[NR][NR][NR];
    Eab Eb, Ek;
    double G[NR][NR][NR];
    for (int i = 0; i < B->np[a]; ++i)
        for (int j = 0; j < B->np[b]; ++j) {
            double ea = B->ex[B->poff[a] + i], eb = B->ex[B->poff[b] + j];
            double p = ea + eb;
            double cab = B->pn[B->poff[a] + i] * B->pn[B->poff[b] + j];
            double P[3];
            for (int x = 0; x < 3; ++x) P[x] = (ea * A[x] + eb * Bc[x]) / p;
            pair_E(B, a, b, ea, eb, Eb);
            for (int k = 0; k < B->np[c]; ++k)
                for (int l = 0; l < B->np[d]; ++l) {
                    double ec = B->ex[B->poff[c] + k], ed = B->ex[B->poff[d] + l];
                    double q = ec + ed;
                    double ccd = B->pn[B->poff[c] + k] * B->pn[B->poff[d] + l];
                    double Q[3];
                    for (int x = 0; x < 3; ++x) Q[x] = (ec * C[x] + ed * D[x]) / q;
                    pair_E(B, c, d, ec, ed, Ek);
                    double alpha = p * q / (p + q);
                    hermite_R(Lt, alpha, P[0] - Q[0], P[1] - Q[1], P[2] - Q[2], R);
                    double pref = 2.0 * pow(M_PI, 2.5) / (p * q * sqrt(p + q)) * cab * ccd;
                    for (int ml = 0; ml < nc; ++ml)
                        for (int ms = 0; ms < nd; ++ms) {
                            const int *u = CART[lc][ml], *v = CART[ld][ms];
                            /* G_{tuv} = sum_{tau,nu,phi} (-1)^{tau+nu+phi} E^{cd} R_{t+tau,...} */
                            for (int t = 0; t <= la + lb; ++t)
                                for (int uu = 0; uu <= la + lb - t; ++uu)
                                    for (int w = 0; w <= la + lb - t - uu; ++w) {
                                        double s = 0.0;
                                        for (int t2 = 0; t2 <= u[0] + v[0]; ++t2)
                                            for (int u2 = 0; u2 <= u[1] + v[1]; ++u2)
                                                for (int w2 = 0; w2 <= u[2] + v[2]; ++w2) {
                                                    double sg = ((t2 + u2 + w2) & 1) ? -1.0 : 1.0;
                                                    s += sg * Ek[0][u[0]][v[0]][t2] *
                                                         Ek[1][u[1]][v[1]][u2] *
                                                         Ek[2][u[2]][v[2]][w2] *
                                                         R[t + t2][uu + u2][w + w2];
                                                }
                                        G[t][uu][w] = s;
                                    }
                            for (int mm = 0; mm < na; ++mm)
                                for (int mn = 0; mn < nb; ++mn) {
                                    const int *x = CART[la][mm], *y = CART[lb][mn];
                                    double s = 0.0;
                                    for (int t = 0; t <= x[0] + y[0]; ++t)
                                        for (int uu = 0; uu <= x[1] + y[1]; ++uu)
                                            for (int w = 0; w <= x[2] + y[2]; ++w)
                                                s += Eb[0][x[0]][y[0]][t] * Eb[1][x[1]][y[1]][uu] *
                                                     Eb[2][x[2]][y[2]][w] * G[t][uu][w];
                                    out[((mm * nb + mn) * nc + ml) * nd + ms] += pref * s;
                                }
                        }
                }
        }
}

/* ---------------- exported API ---------------- */
int or_nbf(int nsh, const int *L)
{
    int n = 0;
    for (int s = 0; s < nsh; ++s) n += NCART[L[s]];
    return n;
}

/* One-electron matrix (nbf x nbf, row-major, normalised functions). */
void or_one_electron(int kind, int nsh, const double *ctr, const int *L,
                     const int *np, const int *poff, const double *ex,
                     const double *co, int natom, const double *axyz,
                     const double *Zc, const double *O, double *M)
{
    Basis B;
    basis_init(&B, nsh, ctr, L, np, poff, ex, co);
    int n = B.nbf;
    double blk[36];
    for (int a = 0; a < nsh; ++a)
        for (int b = 0; b < nsh; ++b) {
            one_block(&B, kind, a, b, natom, axyz, Zc, O, blk);
            int na = NCART[L[a]], nb = NCART[L[b]];
            for (int m = 0; m < na; ++m)
                for (int k = 0; k < nb; ++k) {
                    int i = B.bfo[a] + m, j = B.bfo[b] + k;
                    M[i * n + j] = blk[m * nb + k] * B.f[i] * B.f[j];
                }
        }
    basis_free(&B);
}

/* Normalised contracted shell quartet block [m][n][l][s]. */
void or_eri_shell(int nsh, const double *ctr, const int *L, const int *np,
                  const int *poff, const double *ex, const double *co, int a,
                  int b, int c, int d, double *out)
{
    Basis B;
    basis_init(&B, nsh, ctr, L, np, poff, ex, co);
    eri_block(&B, a, b, c, d, out);
    int na = NCART[L[a]], nb = NCART[L[b]], nc = NCART[L[c]], nd = NCART[L[d]];
    for (int m = 0; m < na; ++m)
        for (int k = 0; k < nb; ++k)
            for (int l = 0; l < nc; ++l)
                for (int s = 0; s < nd; ++s)
                    out[((m * nb + k) * nc + l) * nd + s] *=
                        B.f[B.bfo[a] + m] * B.f[B.bfo[b] + k] * B.f[B.bfo[c] + l] *
                        B.f[B.bfo[d] + s];
    basis_free(&B);
}

/* Full ERI tensor (nbf^4) over all ordered shell quartets; tiny bases only. */
void or_eri_full(int nsh, const double *ctr, const int *L, const int *np,
                 const int *poff, const double *ex, const double *co, double *T)
{
    Basis B;
    basis_init(&B, nsh, ctr, L, np, poff, ex, co);
    long n = B.nbf;
    double *blk = (double *)malloc(sizeof(double) * 1296);
    for (int a = 0; a < nsh; ++a)
        for (int b = 0; b < nsh; ++b)
            for (int c = 0; c < nsh; ++c)
                for (int d = 0; d < nsh; ++d) {
                    eri_block(&B, a, b, c, d, blk);
                    int na = NCART[L[a]], nb = NCART[L[b]], nc = NCART[L[c]], nd = NCART[L[d]];
                    for (int m = 0; m < na; ++m)
                        for (int k = 0; k < nb; ++k)
                            for (int l = 0; l < nc; ++l)
                                for (int s = 0; s < nd; ++s) {
                                    long i = B.bfo[a] + m, j = B.bfo[b] + k;
                                    long kk = B.bfo[c] + l, ll = B.bfo[d] + s;
                                    T[((i * n + j) * n + kk) * n + ll] =
                                        blk[((m * nb + k) * nc + l) * nd + s] * B.f[i] *
                                        B.f[j] * B.f[kk] * B.f[ll];
                                }
                }
    free(blk);
    basis_free(&B);
}

/* Schwarz table Q_ab = sqrt(max_{m in a, n in b} |(mn|mn)|), nsh x nsh. */
void or_schwarz(int nsh, const double *ctr, const int *L, const int *np,
                const int *poff, const double *ex, const double *co, double *Q)
{
    Basis B;
    basis_init(&B, nsh, ctr, L, np, poff, ex, co);
    double blk[1296];
    for (int a = 0; a < nsh; ++a)
        for (int b = 0; b < nsh; ++b) {
            eri_block(&B, a, b, a, b, blk);
            int na = NCART[L[a]], nb = NCART[L[b]];
            double mx = 0.0;
            for (int m = 0; m < na; ++m)
                for (int k = 0; k < nb; ++k) {
                    double v = blk[((m * nb + k) * na + m) * nb + k] * B.f[B.bfo[a] + m] *
                               B.f[B.bfo[b] + k] * B.f[B.bfo[a] + m] * B.f[B.bfo[b] + k];
                    if (fabs(v) > mx) mx = fabs(v);
                }
            Q[a * nsh + b] = sqrt(mx);
        }
    basis_free(&B);
}

static inline void apply_tuple(int n, int nd, const double *D, double *J,
                               double *K, int i, int j, int k, int l, double v)
{
    /* (ij|kl): J_ij += v D_kl ; K_il += v D_jk  (per density) */
    for (int q = 0; q < nd; ++q) {
        const double *Dq = D + (long)q * n * n;
        J[(long)q * n * n + (long)i * n + j] += v * Dq[(long)k * n + l];
        K[(long)q * n * n + (long)i * n + l] += v * Dq[(long)j * n + k];
    }
}

/* J and K for nd general real densities (each nbf x nbf row-major).
 * Visits every permutationally unique function quartet once. */
static long jk_impl(int nsh, const double *ctr, const int *L, const int *np,
           const int *poff, const double *ex, const double *co, int nd,
           const double *D, double *J, double *K, int nthreads, int stride, int offset,
           const unsigned char *sel)
{
    Basis B;
    basis_init(&B, nsh, ctr, L, np, poff, ex, co);
    long n = B.nbf, nn = n * n * nd;
    memset(J, 0, sizeof(double) * nn);
    memset(K, 0, sizeof(double) * nn);
    int npair = nsh * (nsh + 1) / 2;
    long nq = 0;
    int *pa = (int *)malloc(sizeof(int) * npair), *pb = (int *)malloc(sizeof(int) * npair);
    for (int a = 0, p = 0; a < nsh; ++a)
        for (int b = 0; b <= a; ++b, ++p) { pa[p] = a; pb[p] = b; }
    /* work items (bra pair, first ket, end of kets): one per bra pair for a
     * full build; a sample splits its bra pairs' kets into blocks of 64 so
     * that a few bra pairs still spread over all threads */
    const int kblk = (sel || stride > 1) ? 64 : npair;
    long nitem = 0;
    for (int p1 = npair - 1; p1 >= 0; --p1)
        if (sel ? sel[p1] : p1 % stride == offset) nitem += (p1 + kblk) / kblk;
    int *it1 = (int *)malloc(sizeof(int) * (nitem > 0 ? nitem : 1));
    int *it2 = (int *)malloc(sizeof(int) * (nitem > 0 ? nitem : 1));
    nitem = 0;
    for (int p1 = npair - 1; p1 >= 0; --p1)
        if (sel ? sel[p1] : p1 % stride == offset) {
            nq += p1 + 1;
            for (int q = 0; q <= p1; q += kblk) { it1[nitem] = p1; it2[nitem] = q; ++nitem; }
        }
#ifdef _OPENMP
    if (nthreads > 0) omp_set_num_threads(nthreads);
#endif
#pragma omp parallel
    {
        double *Jt = (double *)calloc(nn, sizeof(double));
        double *Kt = (double *)calloc(nn, sizeof(double));
        double *blk = (double *)malloc(sizeof(double) * 1296);
#pragma omp for schedule(dynamic, 1)
        for (long w = 0; w < nitem; ++w) {
            const int p1 = it1[w], q0 = it2[w];
            const int q1 = q0 + kblk - 1 < p1 ? q0 + kblk - 1 : p1;
            int a = pa[p1], b = pb[p1];
            for (int p2 = q0; p2 <= q1; ++p2) {
                int c = pa[p2], d = pb[p2];
                eri_block(&B, a, b, c, d, blk);
                int na = NCART[L[a]], nb = NCART[L[b]], nc = NCART[L[c]], ndd = NCART[L[d]];
                for (int m = 0; m < na; ++m)
                    for (int k2 = 0; k2 < nb; ++k2)
                        for (int l2 = 0; l2 < nc; ++l2)
                            for (int s = 0; s < ndd; ++s) {
                                int i = B.bfo[a] + m, j = B.bfo[b] + k2;
                                int k = B.bfo[c] + l2, l = B.bfo[d] + s;
                                if (a == b && j > i) continue;
                                if (c == d && l > k) continue;
                                if (p1 == p2 && (i < k || (i == k && j < l))) continue;
                                double v = blk[((m * nb + k2) * nc + l2) * ndd + s] *
                                           B.f[i] * B.f[j] * B.f[k] * B.f[l];
                                int tp[8][4] = {{i, j, k, l}, {j, i, k, l}, {i, j, l, k},
                                                {j, i, l, k}, {k, l, i, j}, {l, k, i, j},
                                                {k, l, j, i}, {l, k, j, i}};
                                for (int t = 0; t < 8; ++t) {
                                    int dup = 0;
                                    for (int t2 = 0; t2 < t && !dup; ++t2)
                                        dup = tp[t][0] == tp[t2][0] && tp[t][1] == tp[t2][1] &&
                                              tp[t][2] == tp[t2][2] && tp[t][3] == tp[t2][3];
                                    if (!dup)
                                        apply_tuple(n, nd, D, Jt, Kt, tp[t][0], tp[t][1],
                                                    tp[t][2], tp[t][3], v);
                                }
                            }
            }
        }
#pragma omp critical
        {
            for (long x = 0; x < nn; ++x) { J[x] += Jt[x]; K[x] += Kt[x]; }
        }
        free(Jt); free(Kt); free(blk);
    }
    free(pa); free(pb); free(it1); free(it2);
    basis_free(&B);
    return nq;
}

void or_jk(int nsh, const double *ctr, const int *L, const int *np,
           const int *poff, const double *ex, const double *co, int nd,
           const double *D, double *J, double *K, int nthreads)
{
    jk_impl(nsh, ctr, L, np, poff, ex, co, nd, D, J, K, nthreads, 1, 0, NULL);
}

/* The same loop restricted to bra shell pairs p with p % stride == offset
 * (a deterministic sample of the unique shell quartets, used only to time
 * the oracle on large cases).  Returns the number of shell quartets visited. */
long or_jk_sample(int nsh, const double *ctr, const int *L, const int *np,
                  const int *poff, const double *ex, const double *co, int nd,
                  const double *D, double *J, double *K, int nthreads, int stride, int offset)
{
    return jk_impl(nsh, ctr, L, np, poff, ex, co, nd, D, J, K, nthreads, stride, offset, NULL);
}

/* The same over an explicit set of bra shell pairs (sel[p] != 0, p the
 * pair index a(a+1)/2 + b, a >= b); timing support only. */
long or_jk_pairs(int nsh, const double *ctr, const int *L, const int *np,
                 const int *poff, const double *ex, const double *co, int nd,
                 const double *D, double *J, double *K, int nthreads, const unsigned char *sel)
{
    return jk_impl(nsh, ctr, L, np, poff, ex, co, nd, D, J, K, nthreads, 1, 0, sel);
}

/* Selected elements straight from the definition, for sampling large cases:
 * for each requested (mu, nu): J_{mu nu} = sum_{ls} (mu nu|ls) D_ls and
 * K_{mu nu} = sum_{ls} (mu l|s nu) D_ls, over every (l, s), nd densities.
 * Output layout Jo[q*ne + e], Ko[q*ne + e]. */
void or_jk_elements(int nsh, const double *ctr, const int *L, const int *np,
                    const int *poff, const double *ex, const double *co, int nd,
                    const double *D, int ne, const int *mu, const int *nu,
                    double *Jo, double *Ko, int nthreads)
{
    Basis B;
    basis_init(&B, nsh, ctr, L, np, poff, ex, co);
    long n = B.nbf;
    int *shell_of = (int *)malloc(sizeof(int) * n);
    for (int s = 0; s < nsh; ++s)
        for (int i = B.bfo[s]; i < B.bfo[s + 1]; ++i) shell_of[i] = s;
#ifdef _OPENMP
    if (nthreads > 0) omp_set_num_threads(nthreads);
#endif
#pragma omp parallel for schedule(dynamic, 1)
    for (int e = 0; e < ne; ++e) {
        double blk[1296];
        int i = mu[e], j = nu[e];
        int a = shell_of[i], b = shell_of[j];
        int ia = i - B.bfo[a], jb = j - B.bfo[b];
        int na = NCART[L[a]], nb = NCART[L[b]];
        double *jq = (double *)calloc(nd, sizeof(double));
        double *kq = (double *)calloc(nd, sizeof(double));
        for (int c = 0; c < nsh; ++c)
            for (int d = 0; d < nsh; ++d) {
                int nc = NCART[L[c]], ndd = NCART[L[d]];
                /* J: (a b | c d) */
                eri_block(&B, a, b, c, d, blk);
                for (int l = 0; l < nc; ++l)
                    for (int s = 0; s < ndd; ++s) {
                        int k = B.bfo[c] + l, ll = B.bfo[d] + s;
                        double v = blk[((ia * nb + jb) * nc + l) * ndd + s] * B.f[i] *
                                   B.f[j] * B.f[k] * B.f[ll];
                        for (int q = 0; q < nd; ++q) jq[q] += v * D[(long)q * n * n + k * n + ll];
                    }
                /* K: (a c | d b) with lambda in c, sigma in d */
                eri_block(&B, a, c, d, b, blk);
                for (int l = 0; l < nc; ++l)
                    for (int s = 0; s < ndd; ++s) {
                        int k = B.bfo[c] + l, ll = B.bfo[d] + s;
                        double v = blk[((ia * nc + l) * ndd + s) * nb + jb] * B.f[i] *
                                   B.f[k] * B.f[ll] * B.f[j];
                        for (int q = 0; q < nd; ++q) kq[q] += v * D[(long)q * n * n + k * n + ll];
                    }
            }
        for (int q = 0; q < nd; ++q) { Jo[(long)q * ne + e] = jq[q]; Ko[(long)q * ne + e] = kq[q]; }
        free(jq); free(kq);
        (void)na;
    }
    free(shell_of);
    basis_free(&B);
}

/* Whole shell-pair blocks straight from the definition, for sampling large
 * cases: for each requested shell pair (a, b) and every (c, d),
 *   J_{mn} += sum_{ls} (mn|ls) D_ls   (m in a, n in b; l in c, s in d),
 *   K_{mn} += sum_{ls} (ml|sn) D_ls,
 * nd densities.  Output Jo/Ko[(q * np + p) * 36 + m * nb + n]. */
void or_jk_blocks(int nsh, const double *ctr, const int *L, const int *np,
                  const int *poff, const double *ex, const double *co, int nd,
                  const double *D, int npairs, const int *pa, const int *pb,
                  double *Jo, double *Ko, int nthreads)
{
    Basis B;
    basis_init(&B, nsh, ctr, L, np, poff, ex, co);
    long n = B.nbf;
    memset(Jo, 0, sizeof(double) * nd * npairs * 36);
    memset(Ko, 0, sizeof(double) * nd * npairs * 36);
#ifdef _OPENMP
    if (nthreads > 0) omp_set_num_threads(nthreads);
#endif
    for (int p = 0; p < npairs; ++p) {
        const int a = pa[p], b = pb[p];
        const int na = NCART[L[a]], nb = NCART[L[b]];
#pragma omp parallel
        {
            double blk[1296];
            double *jt = (double *)calloc(nd * 36, sizeof(double));
            double *kt = (double *)calloc(nd * 36, sizeof(double));
#pragma omp for schedule(dynamic, 1)
            for (int c = 0; c < nsh; ++c)
                for (int d = 0; d < nsh; ++d) {
                    const int nc = NCART[L[c]], ndd = NCART[L[d]];
                    eri_block(&B, a, b, c, d, blk);          /* (ab|cd) */
                    for (int m = 0; m < na; ++m)
                        for (int k2 = 0; k2 < nb; ++k2)
                            for (int l = 0; l < nc; ++l)
                                for (int s = 0; s < ndd; ++s) {
                                    const int i = B.bfo[a] + m, j = B.bfo[b] + k2;
                                    const int k = B.bfo[c] + l, ll = B.bfo[d] + s;
                                    const double v = blk[((m * nb + k2) * nc + l) * ndd + s] * B.f[i] *
                                                     B.f[j] * B.f[k] * B.f[ll];
                                    for (int q = 0; q < nd; ++q)
                                        jt[q * 36 + m * nb + k2] += v * D[(long)q * n * n + k * n + ll];
                                }
                    eri_block(&B, a, c, d, b, blk);          /* (ac|db) */
                    for (int m = 0; m < na; ++m)
                        for (int l = 0; l < nc; ++l)
                            for (int s = 0; s < ndd; ++s)
                                for (int k2 = 0; k2 < nb; ++k2) {
                                    const int i = B.bfo[a] + m, j = B.bfo[b] + k2;
                                    const int k = B.bfo[c] + l, ll = B.bfo[d] + s;
                                    const double v = blk[((m * nc + l) * ndd + s) * nb + k2] * B.f[i] *
                                                     B.f[k] * B.f[ll] * B.f[j];
                                    for (int q = 0; q < nd; ++q)
                                        kt[q * 36 + m * nb + k2] += v * D[(long)q * n * n + k * n + ll];
                                }
                }
#pragma omp critical
            {
                for (int q = 0; q < nd; ++q)
                    for (int e = 0; e < 36; ++e) {
                        Jo[((long)q * npairs + p) * 36 + e] += jt[q * 36 + e];
                        Ko[((long)q * npairs + p) * 36 + e] += kt[q * 36 + e];
                    }
            }
            free(jt); free(kt);
        }
    }
    basis_free(&B);
}

/* Per-function renormalisation factors (exposed for tests). */
void or_norm_factors(int nsh, const double *ctr, const int *L, const int *np,
                     const int *poff, const double *ex, const double *co, double *f)
{
    Basis B;
    basis_init(&B, nsh, ctr, L, np, poff, ex, co);
    for (int i = 0; i < B.nbf; ++i) f[i] = B.f[i];
    basis_free(&B);
}
