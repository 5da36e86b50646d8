/*
 * cq.h -- C ABI of the GB300 direct-SCF Fock-build library (libcq.so).
 *
 * What it computes (ChronusQ paper, Sec. "Reference Wave Functions",
 * Eq. 2c_fock, and Sec. "General Infrastructure for the Unified Treatment of
 * Electronic Spin", Eq. pauli_sep): Coulomb and exchange matrices over
 * contracted Cartesian Gaussian basis functions,
 *     J_{mn} = sum_{ls} (mn|ls) P_{ls},     K_{mn} = sum_{ls} (ml|sn) P_{ls},
 * evaluated directly (integrals recomputed on every call, "direct SCF"),
 * with Schwarz x density screening, for real symmetric, complex Hermitian
 * and two-component (Pauli scalar + 3 spin components) densities; and the
 * drivers built on it (RHF/GHF SCF, RT-TDHF steps).
 *
 * Conventions for every entry point:
 *   - Matrices are row-major nbf x nbf.  Complex matrices are interleaved
 *     (re, im) doubles (the layout of complex128).
 *   - Basis functions are Cartesian, lexicographic within a shell
 *     (s; x,y,z; xx,xy,xz,yy,yz,zz); every Cartesian component of every
 *     contracted function is normalised to unit self-overlap.
 *   - "device" pointers are CUDA device memory owned by the caller; "host"
 *     pointers are host memory owned by the caller.  The library never frees
 *     caller memory.  Scratch memory the library needs is allocated inside the
 *     basis handle (cq_basis_create / first use) and freed by cq_basis_destroy.
 *   - `stream` is a cudaStream_t (NULL = legacy default stream).  All work of
 *     a call is enqueued on that stream; calls that return host values
 *     synchronise it.
 *   - No entry point aborts or traps.  Every failure returns a negative
 *     cq_status and sets a thread-local message read by cq_last_error().
 *   - A basis handle holds the scratch of its builds and drivers: calls on
 *     one handle must not overlap (one host thread, or calls ordered by the
 *     caller); different handles are independent.  cq_fock_build_noalloc
 *     shares one scratch array across all handles of a device.
 */
#ifndef CQ_H
#define CQ_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    CQ_OK = 0,
    CQ_ERR_INVALID_ARG = -1,
    CQ_ERR_CUDA = -2,
    CQ_ERR_OOM = -3,
    CQ_ERR_NOT_CONVERGED = -4,
    CQ_ERR_NUMERIC = -5,
    CQ_ERR_TIMEOUT = -6,
    CQ_ERR_UNSUPPORTED = -7
} cq_status;

/* Density kinds for cq_fock_build (Eq. spin_generalization). */
typedef enum {
    CQ_DENS_REAL_SYM = 0,      /* P real symmetric (one spin block, RHF)     */
    CQ_DENS_COMPLEX_HERM = 1,  /* P complex Hermitian (RT-TDHF, one block)   */
    CQ_DENS_PAULI4 = 2,        /* P^0..P^3 complex Hermitian (GHF, 2C)       */
    CQ_DENS_REAL_GENERAL = 3   /* P real, any symmetry: the transition
                                  densities of the direct ph-RPA products,
                                  contracted as in Eq. 2c_fock with a
                                  non-Hermitian density (Sec. "Residue
                                  Methods")                                  */
} cq_dens_kind;

typedef enum { CQ_PREC_FP64 = 0, CQ_PREC_MIXED = 1 } cq_prec;

typedef struct cq_basis cq_basis;   /* opaque; owns device copies + scratch */

/* cq_basis_create: build a basis from host arrays (copied; caller keeps
 * ownership).  Contracted Cartesian Gaussian shells (paper Sec.
 * "Input Specification": CGTO expansions, segmented contraction).
 *   natom, xyz[3*natom] (bohr), Z[natom]            nuclei
 *   nshell, shell_atom[nshell], shell_L[nshell] (0..2),
 *   shell_nprim[nshell] (1..16)
 *   exps[sum nprim] (>0), coefs[sum nprim]          raw contraction
 *                                                   coefficients of
 *                                                   unnormalised primitives
 * Errors: CQ_ERR_INVALID_ARG (L>2, nprim out of range, exponent <= 0, NULL),
 * CQ_ERR_CUDA / CQ_ERR_OOM on device failures.  Runs on the current device
 * and synchronises it.  The Schwarz table (cq_schwarz) is computed here. */
int cq_basis_create(int natom, const double* xyz, const int* Z, int nshell,
                    const int* shell_atom, const int* shell_L,
                    const int* shell_nprim, const double* exps,
                    const double* coefs, cq_basis** out);

/* cq_basis_create_batch: many independent molecules in one basis (batched
 * execution of the Fock build and SCF).  atom_mol[natom] gives each atom's
 * molecule, as consecutive ids 0,..,0,1,..,1,...; shells must be ordered by
 * molecule.  Shell pairs and quartets are formed within a molecule only.
 * Every matrix argument of the batched basis (densities, J, K, one-electron
 * matrices, SCF densities) uses the batched layout: nmol slots of ld x ld
 * (ld = the largest molecule's function count, cq_basis_layout), element
 * (r, c) of molecule m at m*ld*ld + r*ld + c, padding elements zero.  A
 * single-molecule basis has nmol = 1 and ld = nbf (the plain layout). */
int cq_basis_create_batch(int natom, const double* xyz, const int* Z,
                          const int* atom_mol, int nshell,
                          const int* shell_atom, const int* shell_L,
                          const int* shell_nprim, const double* exps,
                          const double* coefs, cq_basis** out);

/* Molecule count, slot dimension ld and functions per molecule (host
 * array of nmol, may be NULL). */
int cq_basis_layout(const cq_basis* b, int* nmol, int* ld, int* mol_n);

/* Number of basis functions, shells, shell pairs. */
int cq_basis_info(const cq_basis* b, int* nbf, int* nshell, int* npair);

void cq_basis_destroy(cq_basis* b);

/* cq_boys: the Boys function F_m(T) = int_0^1 t^(2m) exp(-T t^2) dt,
 * m = 0..mmax (mmax <= 8), at n arguments, evaluated by the same device
 * code the integral kernels use (the [00|00]^(m) factor of the Obara-Saika
 * recurrence, Sec. "Reference Wave Functions" direct integral evaluation):
 * fp32 = 0 in FP64; fp32 = 1 in FP32 with the argument rounded to FP32 and
 * FP64 evaluation below T = 1/32 (the first table interval); fp32 = 2 in
 * double-float (pairs of FP32 numbers, about 48 significant bits).
 *   T: device, n doubles.  F: device, n x (mmax + 1) doubles, row-major
 *   (FP32 results widened).  The table lives in the basis handle b.
 *   Returns CQ_ERR_INVALID_ARG for mmax outside 0..8, fp32 outside 0..2,
 *   n < 0 or NULL arrays. */
int cq_boys(const cq_basis* b, int fp32, int mmax, int n, const double* T, double* F, void* stream);

/* cq_schwarz: Schwarz factors Q_ab = sqrt(max_{m in a, n in b} |(mn|mn)|)
 * (screening of the direct build, Sec. "Reference Wave Functions": LinK-like
 * screening).  Q: device, nshell*nshell doubles (row-major, symmetric), or
 * NULL to only (re)compute the internal table (a batched basis accepts only
 * NULL).  Enqueued on `stream`. */
int cq_schwarz(cq_basis* b, double* Q, void* stream);

typedef struct {
    double schwarz_tol;  /* skip a shell quartet when Q_ab Q_cd max|P| < tol (1e-14) */
    double mixed_tol;    /* CQ_PREC_MIXED: quartets with bound < mixed_tol in FP32 */
    int prec;            /* cq_prec */
    int want_J, want_K;  /* 0/1 */
    double fp64_tol;     /* CQ_PREC_MIXED: quartets with mixed_tol <= bound < fp64_tol in
                            double-float (pairs of FP32 values, ~48 bits, on the FP32
                            pipes); bound >= fp64_tol in FP64.  0 (or <= mixed_tol): no
                            double-float tier */
} cq_fock_opts;

typedef struct {
    unsigned long long quartets_fp64;  /* contracted shell quartets evaluated in FP64 */
    unsigned long long quartets_fp32;  /* ... in FP32 (mixed precision)             */
    unsigned long long prim_fp64, prim_fp32; /* primitive quartets                   */
    double ms;                          /* device time of the build (CUDA events)   */
    unsigned long long quartets_df, prim_df;  /* ... in double-float (fp64_tol tier) */
} cq_fock_stats;

/* cq_fock_build: J and K of a density (Eq. 2c_fock; Pauli components per
 * Eq. pauli_sep).  All pointers device, row-major:
 *   REAL_SYM:      P nbf^2 f64 (symmetric); J nbf^2 f64; K nbf^2 f64.
 *   COMPLEX_HERM:  P nbf^2 c128 (Hermitian); J nbf^2 f64 (J of Re P; J of the
 *                  antisymmetric Im P vanishes); K nbf^2 c128 (Hermitian).
 *   PAULI4:        P 4*nbf^2 c128 (P^0..P^3, each Hermitian); J nbf^2 f64 =
 *                  J[P^0]; K 4*nbf^2 c128 = K[P^0..P^3].
 *   REAL_GENERAL:  P nbf^2 f64 (any symmetry); J nbf^2 f64 (J of the
 *                  symmetric part; that of the antisymmetric part vanishes);
 *                  K nbf^2 f64 = K[P] = K[S] + K[A] (S, A the symmetric and
 *                  antisymmetric parts, built as the real and imaginary
 *                  parts of the Hermitian S + iA).
 * J or K may be NULL when opts->want_J / want_K is 0.  opts NULL = defaults
 * (schwarz_tol 1e-14, FP64, J and K).  stats may be NULL; when given, the
 * call synchronises `stream` to fill it.  Hermiticity of P is assumed, not
 * checked (except for REAL_GENERAL): only the symmetric part of Re P and
 * the antisymmetric part of Im P contribute. */
int cq_fock_build(cq_basis* b, int kind, const void* P, double* J, void* K,
                  const cq_fock_opts* opts, cq_fock_stats* stats, void* stream);

/* cq_fock_build_noalloc: the same J/K build as cq_fock_build for callers
 * that cannot have the library allocate device memory -- for example a host
 * program that hands out all device memory from its own pool or fixed
 * budget, or a loop that must not pay for cudaMalloc/cudaFree and the device
 * synchronisation they may cause.  The paper has no counterpart; this is an
 * interface of this library only.
 *   - Allocates nothing: its scratch (scaled densities, J'/K' accumulators,
 *     block maxima, counters) lives in one file-scope __device__ array of
 *     16 MiB (16777216 bytes) that every GPU loading the library holds until
 *     the library is unloaded.  cq_fock_noalloc_scratch_bytes(kind, nbf,
 *     nshell) gives the bytes a build on a single-molecule basis needs
 *     (about (3 nk + 2) nbf^2 doubles -- nk scaled densities plus the
 *     two-word J'/K' accumulators -- with nk = 1 / 2 / 8 for REAL_SYM /
 *     COMPLEX_HERM / PAULI4, so nbf up to about 647 / 512 / 284).  For a batched basis (cq_basis_create_batch)
 *     the need is that of nmol slots of the largest molecule, more than the
 *     query reports for the total nbf and nshell: the call itself checks the
 *     exact need.  A basis that needs more than the array is rejected with
 *     CQ_ERR_INVALID_ARG before any work is enqueued.
 *   - Arguments, layouts and results are those of cq_fock_build; there is no
 *     stats output.  The basis must come from cq_basis_create (which does
 *     allocate, once, ahead of time).
 *   - The first call on each device looks up the array's device address
 *     (cudaGetSymbolAddress) with that device current.  Under CUDA's lazy
 *     module loading (the default) that lookup is also what loads the code
 *     module holding the array, so the 16 MiB are reserved on the device by
 *     this first call, not when the library is loaded: make the first call
 *     at set-up -- before the caller's own allocator takes the rest of the
 *     device memory, and before any stream capture.  The first launch of the integral kernels in
 *     a process may also make the driver enlarge its per-thread local-memory
 *     reservation, so run one build before entering a region where no device
 *     memory may be reserved.
 *   - All calls share the one array, and it keeps the last call's contents
 *     (the accumulators are cleared at the start of each call).  Calls whose
 *     work overlaps on the GPU -- different streams, or different host
 *     threads -- race on it and give wrong results: serialise them. */
int cq_fock_build_noalloc(cq_basis* b, int kind, const void* P, double* J,
                          void* K, const cq_fock_opts* opts, void* stream);
size_t cq_fock_noalloc_scratch_bytes(int kind, int nbf, int nshell);

/* Per-class profile of cq_fock_build (instrumentation, off by default).
 * cq_fock_profile(b, 1) makes later builds record CUDA events around each
 * angular-momentum-class kernel.  cq_fock_class_stats returns, for the last
 * build, class qc (0..20, bra class X >= ket class Y, qc = X(X+1)/2 + Y with
 * pair classes ss,ps,pp,ds,dp,dd = 0..5) and precision (fp32: 0 FP64,
 * 1 FP32, 2 double-float): kernel
 * time in ms (0 if profiling was off), contracted and primitive quartets
 * evaluated.  Synchronises the device. */
int cq_fock_profile(cq_basis* b, int enable);
int cq_fock_class_stats(cq_basis* b, int qc, int fp32, double* ms,
                        unsigned long long* quartets, unsigned long long* prims);

/* Kernel variant used for one angular-momentum class (qc as for
 * cq_fock_class_stats) and precision (prec: 0 FP64, 1 FP32, 2 double-float):
 *   0 = lane-group kernel (lanes of a warp split one quartet's primitive
 *       quartets, generated straight-line recurrences); double-float only
 *       for classes of total angular momentum <= 3;
 *   1 = warp-cooperative kernel (one warp per quartet walking generated
 *       recurrence tables through shared memory) over one task per
 *       (class, bra pair), screening inside the kernel; FP64 and FP32 only;
 *   2 = axis-permutation lane groups (classes of total angular momentum
 *       >= 4 with a d shell, and (pp|pp); FP64 and double-float too except
 *       (dd|dp) and (dd|dd)): 3 or 6 lanes per quartet each run the
 *       vertical recurrence for a third or a sixth of the targets on
 *       axis-permuted inputs;
 *   3 = the warp-cooperative kernel over the build's screened quartet
 *       list, each quartet's primitive quartets split over up to four warps.
 * CQ_ERR_UNSUPPORTED where a class has no such kernel, CQ_ERR_INVALID_ARG
 * for arguments out of range.  All give the same J/K to rounding; the
 * choice only changes speed (set by the autotuner). */
int cq_fock_set_variant(cq_basis* b, int qc, int prec, int variant);

int cq_fock_get_variant(const cq_basis* b, int qc, int prec, int* variant);

/* Work split of variant 3 (the cooperative kernel on the screened list) at
 * precision prec: each quartet's primitive quartets are cut into
 * ceil(nprim / chunk) ranges, at most `split` (1..64), one warp task each
 * (every task repeats the HRR and the digestion).  Defaults: FP64 8 / 64,
 * FP32 and double-float 4 / 32.  CQ_ERR_INVALID_ARG out of range. */
int cq_fock_set_list_split(cq_basis* b, int prec, int split, int chunk);

/* Memory bound of the quartet lists (no paper counterpart).  A basis
 * created while the capacity is C keeps one list of min(C, candidates)
 * 8-byte entries, where candidates = the shell quartets of every class that
 * pass no screening yet (about npair^2 / 2).  When the candidates exceed C
 * (large bases), the basis uses one task per (class, bra pair) and every
 * build screens, lists and evaluates the quartets of each class in passes of
 * whole tasks that fit the list, one after the other on the caller's
 * stream; the cooperative kernel then reads its quartets from the list.
 * Results are the same up to the order of the FP64 sums.  Default
 * 3e9 entries (24 GB); CQ_ERR_INVALID_ARG below 1024.  Process-wide;
 * affects bases created afterwards. */
int cq_set_list_capacity(long long entries);
long long cq_get_list_capacity(void);

/* Autotuner: times every kernel variant a class has at every precision
 * the options use -- FP64; FP64 and FP32; or, when fp64_tol > mixed_tol,
 * FP32 and double-float (the FP64 tier of a three-tier build always runs
 * variant 3) -- on the given density (device, layout as for cq_fock_build)
 * with the given options (NULL: mixed precision, mixed_tol 1e-3), keeps the
 * fastest variant per class and precision in the basis, then tries the
 * runner-up variant of each of the eight costliest (class, precision)
 * kernels in turn and keeps it only if the median of three complete
 * (concurrent) builds gets more than 1 % faster.  Returns the choice in
 * table[3*qc + prec] and the best isolated kernel time in
 * ms_out[3*qc + prec] (0 for precisions not used; host arrays of 63, either
 * may be NULL).  Runs up to 39 builds; allocates and frees two output
 * buffers. */
int cq_autotune(cq_basis* b, int kind, const void* P, const cq_fock_opts* opts,
                int* table, double* ms_out, void* stream);

/* FMA throughput of the current device (FP64 if fp32 == 0, else FP32), in
 * floating-point operations per second (an FMA counts 2), from independent
 * FMA chains on every SM.  Measurement support for the roofline of the
 * integral kernels; allocates and frees a small output buffer. */
int cq_peak_fma(int fp32, int iters, double* flops_per_s, void* stream);

/* One-electron matrices (device, nbf^2 f64 each): overlap S, kinetic T,
 * nuclear attraction V (all nuclei of the basis) and dipole-moment integrals
 * M_d = <m| r_d - origin_d |n> (3*nbf^2, d = x,y,z; no charge sign), the
 * core Hamiltonian h = T + V of Eq. 2c_fock and the electric-dipole operator
 * of the real-time perturbation (Sec. "Real-Time Electronic Dynamics").
 * Any output may be NULL; origin: host double[3] or NULL for (0,0,0). */
int cq_one_electron(cq_basis* b, double* S, double* T, double* V, double* M,
                    const double* origin, void* stream);

/* RHF direct SCF (Sec. "Self-Consistent Field Optimization": DIIS
 * extrapolation of the Fock matrix; RS case of Eq. rh_1c), every Fock matrix
 * from cq_fock_build.  Loewdin orthogonalisation S^{-1/2}, canonical when an
 * overlap eigenvalue is below 1e-8.  Core-Hamiltonian guess unless D_in
 * (device, nbf^2, per-spin density C_occ C_occ^T) is given.  Converged when
 * |dE| < e_tol and rms(X^T (FDS - SDF) X) < d_tol after a full FP64 build.
 *   prec = CQ_PREC_MIXED: FP32 for quartets with bound < mixed_tol until the
 *   error rms drops below switch_tol, then full FP64 builds (final
 *   iterations).  incremental = 1: Fock matrices built from the density
 *   change, F_k = F_{k-1} + G[D_k - D_{k-1}], with a full rebuild every
 *   full_every iterations and before convergence is declared.
 * Outputs (device): D_out nbf^2 (required), F_out nbf^2 (may be NULL).
 * Returns CQ_ERR_NOT_CONVERGED (stats filled) if max_iter is reached,
 * CQ_ERR_NUMERIC on a non-finite energy.  Synchronises `stream` every
 * iteration (convergence test on the host). */
typedef struct {
    double e_tol;        /* 1e-10 */
    double d_tol;        /* 1e-8  */
    int max_iter;        /* 128 */
    int diis_size;       /* 1..8 */
    int prec;            /* cq_prec */
    double mixed_tol;    /* 1e-5 */
    double schwarz_tol;  /* 1e-14 */
    int incremental;     /* 0/1 */
    int full_every;      /* 8 */
    double switch_tol;   /* 1e-5 */
    int graph;           /* cq_scf_batch: 1 = capture the iteration as a CUDA graph */
    int guess_fallback;  /* cq_scf_batch with D_in: a molecule still open at this
                            iteration (> 1) restarts from the core guess with a
                            fresh DIIS subspace; 0 = never */
    double fp64_tol;     /* mixed builds: double-float tier for mixed_tol <= bound
                            < fp64_tol, as in cq_fock_opts; 0 = two tiers */
} cq_scf_opts;
typedef struct {
    double energy;
    int iterations, converged;
    double last_rms;
    unsigned long long quartets_fp64, quartets_fp32;  /* summed over iterations */
    double ms;
    int graph;           /* cq_scf_batch: 2 whole iteration replayed as a graph,
                            1 graphs around an eager eigensolver call, 0 eager */
    unsigned long long quartets_df;  /* double-float quartets, summed over iterations */
} cq_scf_stats;
int cq_scf(cq_basis* b, int nocc, const cq_scf_opts* opts, const double* D_in,
           double* D_out, double* F_out, cq_scf_stats* stats, void* stream);

/* Two-component (GHF) SCF in the Pauli representation (Eq. pauli_sep,
 * Eq. 2c_fock with the factor-2 reading of J): per iteration one Fock build
 * of kind CQ_DENS_PAULI4, F^0 = h + 2J[P^0] - K[P^0], F^k = -K[P^k]; the
 * 2n x 2n Fock matrix sum_I sigma_I (x) F^I is diagonalised in the
 * orthonormal basis diag(X, X) and the nelec lowest spinors give
 * P^{2C} = C C^+, whose Pauli components are the next density.
 * E = sum_I Re Tr[(h^I + F^I) P^I] + E_nuc (h^k = 0).  DIIS on
 * X^+(F P S - S P F)X with real B_ij = Re <e_i|e_j>.  Options as for cq_scf
 * (prec/mixed_tol/switch_tol as there; incremental builds, graph and
 * guess_fallback are not used).
 * P_in: device 4 x nbf^2 c128 Hermitian Pauli components (NULL: core guess,
 * which is collinear); P_out (required), F_out (may be NULL): device
 * 4 x nbf^2 c128.  Returns CQ_ERR_NOT_CONVERGED (stats filled) if max_iter
 * is reached.  Synchronises `stream` every iteration. */
int cq_scf_ghf(cq_basis* b, int nelec, const cq_scf_opts* opts, const void* P_in,
               void* P_out, void* F_out, cq_scf_stats* stats, void* stream);

/* Batched RHF SCF over the molecules of a batched basis
 * (cq_basis_create_batch): one Fock build for all molecules per iteration,
 * the dense steps as strided-batched GEMMs and a batched eigensolver on the
 * ld x ld slots.  nocc: host array of nmol occupied-orbital counts.  D_in
 * (device, batched layout, may be NULL for the core guess), D_out (device,
 * batched layout), E_out and iters_out (host arrays of nmol, may be NULL).
 * A supplied D_in need not be idempotent: the first iteration diagonalises
 * its Fock matrix without adding it to the DIIS subspace.
 * Options as for cq_scf (incremental builds are not used here).  Each
 * molecule converges on its own: its density is then frozen and later
 * builds skip its quartets.  With prec = CQ_PREC_MIXED a molecule's builds
 * move to all-FP64 once its orthogonal-basis commutator rms falls below
 * switch_tol, and convergence is only declared on an all-FP64 energy.
 * The state of an iteration (iteration number, DIIS ring, convergence
 * flags) lives on the device, so with opts->graph the iterations after the
 * first are captured once as a CUDA graph and replayed; the host reads the
 * number of open molecules one iteration behind (at most one extra, no-op
 * iteration).  With D_in and opts->guess_fallback = k > 1, a molecule not
 * converged after k iterations restarts from the core-Hamiltonian guess
 * (the supplied guess is then only a first try; the answer is judged by
 * the SCF either way).  Runs on a private stream ordered after `stream`; returns
 * after it has drained.  Returns CQ_ERR_NOT_CONVERGED if any molecule
 * reached max_iter.  stats->iterations is the number of batched iterations,
 * stats->converged the number of converged molecules, stats->energy the sum
 * of the energies, stats->graph how the iterations were launched. */
int cq_scf_batch(cq_basis* b, const int* nocc, const cq_scf_opts* opts,
                 const double* D_in, double* D_out, double* E_out,
                 int* iters_out, cq_scf_stats* stats, void* stream);

/* One closed-shell RT-TDHF step of the Liouville-von Neumann equation (Eq.
 * lvn), in the orthonormal (Loewdin) basis:
 *   MMUT  P_{k+1} = U P_{k-1} U^+,  U = exp(-2 i dt F(P_k, t_k));
 *   EM2   (step 0, and every restart_every steps)
 *         P_{k+1} = U P_k U^+,  U = exp(-i dt (F(P_k,t_k) + F(P_FE,t_{k+1}))/2),
 *         P_FE = U_FE P_k U_FE^+,  U_FE = exp(-i dt F(P_k, t_k)).
 * F(P, t) = h + 2J[P] - K[P] + E(t).M (Eq. td_pert; length gauge, electron
 * charge -1; E(t) = field on [t_on, t_off), else 0), t_k = step*dt.  The
 * exponentials are Taylor series with scaling and squaring (ZGEMMs).
 * P_prev, P_cur: device nbf^2 c128 AO densities (per spin); on return
 * P_prev <- P_cur and P_cur <- P_{k+1}.  P_prev may be NULL only for step 0.
 * obs (host, may be NULL): observables of P_k (the density on entry), from
 * the step's own Fock build: dipole = -2 Re Tr[M P] + sum_A Z_A R_A, Tr(PS),
 * field-free energy Re Tr[(h + F0) P] + E_nuc (Eq. td_expectation). */
typedef struct {
    double dt;
    double field[3];
    double t_on, t_off;
    int restart_every;   /* 50 */
    int prec;            /* cq_prec */
    double mixed_tol;
    double schwarz_tol;
    double fp64_tol;     /* mixed builds: double-float tier below it (cq_fock_opts); 0 = two tiers */
} cq_rt_opts;
typedef struct {
    double dipole[3];
    double trPS;
    double energy;
    int em2;             /* 1 if this step was an EM2 step */
} cq_rt_obs;
int cq_rt_step(cq_basis* b, const cq_rt_opts* opts, int step, void* P_prev,
               void* P_cur, cq_rt_obs* obs, void* stream);

/* Learned initial density (a build requirement; no paper counterpart -- the
 * paper's SCF starts from standard guesses).  An MLP (40 -> 256 -> 256 ->
 * 1472, SiLU) maps an atom-pair descriptor to that pair's density block in
 * the even-tempered s,p,d basis (H 3s1p = 6 functions, C/N/O 4s3p2d = 25);
 * heads: 0 H on-site, 1 heavy on-site, 2 H-H, 3 H-heavy (H rows), 4
 * heavy-heavy.  Parameters: device float array of cq_mlp_param_count().
 *   cq_mlp_init        seeded initialisation.
 *   cq_guess_dataset   descriptors X (npair x 40 f32), targets T (npair x
 *                      1472 f32, the converged D blocks) and heads (npair
 *                      i32) of every atom pair of a batched basis; D in the
 *                      batched layout (may be NULL with T NULL).  X, T,
 *                      head may be NULL to only count (*npair).
 *   cq_mlp_loss_grad   masked MSE and its gradient for n samples.
 *   cq_mlp_train       Adam over `epochs` shuffled passes (minibatch rows).
 *   cq_guess_density   guess D (batched layout) for every molecule:
 *                      assembled blocks (flags bit 0: on-site blocks only),
 *                      Tr(DS) = nocc[m], npurify McWeeny steps.  Pass it as D_in to cq_scf_batch; the SCF
 *                      decides the answer, the guess only changes the
 *                      iteration count.
 * Returns CQ_ERR_UNSUPPORTED if an atom does not carry that basis. */
size_t cq_mlp_param_count(void);
int cq_mlp_init(float* params, unsigned long long seed, void* stream);
int cq_guess_dataset(cq_basis* b, const double* D, float* X, float* T,
                     int* head, int* npair, void* stream);
int cq_mlp_loss_grad(const float* params, int n, const float* X,
                     const float* T, const int* head, float* grad,
                     double* loss, void* stream);
int cq_mlp_train(float* params, int n, const float* X, const float* T,
                 const int* head, int epochs, int batch, float lr,
                 unsigned long long seed, double* last_loss, void* stream);
int cq_guess_density(cq_basis* b, const float* params, const int* nocc,
                     int npurify, int flags, double* D, void* stream);

/* Number of orthonormal functions (columns of X) and dropped overlap
 * eigenvectors; computes the one-electron data on first use. */
int cq_dense_info(cq_basis* b, int* northo, int* ndropped, void* stream);

/* Nuclear repulsion energy of the basis' nuclei (host result; summed over
 * the molecules of a batched basis), and per molecule (host array of nmol). */
int cq_nuclear_repulsion(const cq_basis* b, double* E);
int cq_nuclear_repulsion_batch(const cq_basis* b, double* E);

const char* cq_last_error(void);

#ifdef __cplusplus
}
#endif
#endif /* CQ_H */
