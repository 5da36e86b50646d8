// Internal host-side state of the Fock-build library.
#pragma once
#include <cuda_runtime.h>

#include <string>
#include <vector>

#include "../../include/cq.h"
#include "cq_common.cuh"

namespace cq {

struct JKArgs;

// pair classes (la, lb), la >= lb: 00 10 11 20 21 22
constexpr int NPC = 6;
constexpr int NQC = 21;   // (bra class X) >= (ket class Y)
inline int pc_of(int la, int lb) { return la * (la + 1) / 2 + lb; }
// real density matrices a build contracts for each density kind
inline int dens_nk(int kind)
{
    return kind == CQ_DENS_REAL_SYM ? 1 : (kind == CQ_DENS_COMPLEX_HERM || kind == CQ_DENS_REAL_GENERAL) ? 2 : 8;
}
extern const int PC_L[NPC][2];

using LaunchJK = void (*)(const JKArgs&, int fp32, cudaStream_t);
using LaunchSchwarz = void (*)(const JKArgs&, int, int, float*, double*, cudaStream_t);
extern const LaunchJK JK_LAUNCH[NQC];          // index: X*(X+1)/2 + Y
extern const LaunchSchwarz SCHWARZ_LAUNCH[NPC];
void launch_coop(const JKArgs& a, int qc, int fp32, cudaStream_t s);
size_t coop_smem_bytes(int qc, int fp32);

// kernel variant per quartet class: 0 lane-group kernel, 1 warp-cooperative,
// 2 axis-permutation lane groups (classes with an entry in SYM_LAUNCH; FP64
// where SYM_F64)
constexpr int VARIANT_LANES = 0, VARIANT_COOP = 1, VARIANT_SYM = 2, VARIANT_COOP_LIST = 3, NVARIANT = 4;
// precision index of a class launch: 0 FP64, 1 FP32, 2 double-float
constexpr int PREC_DF = 2;
// counters of a build: 6 totals (quartets, primitive quartets of each
// precision), then 6 per class
constexpr int CNT_WORDS = 6 + 6 * NQC;
extern const LaunchJK SYM_LAUNCH[NQC];      // NULL where a class has no split kernel
extern const int SYM_F64[NQC];              // 1 where the split kernel also exists in FP64 and double-float
extern const int LANE_DF[NQC];              // 1 where the lane-group kernel exists in double-float
extern const int DEFAULT_VARIANT[NQC][3];   // [class][FP64, FP32, double-float]
bool variant_exists(int qc, int prec, int v);

void set_error(const std::string& msg);
int cuda_fail(cudaError_t e, const char* what);

#define CQ_CUDA(call)                                         \
    do {                                                      \
        cudaError_t _e = (call);                              \
        if (_e != cudaSuccess) return cq::cuda_fail(_e, #call); \
    } while (0)

template <typename T>
int dalloc(T** p, size_t n)
{
    *p = nullptr;
    if (n == 0) n = 1;
    cudaError_t e = cudaMalloc((void**)p, n * sizeof(T));
    if (e != cudaSuccess) {
        set_error(std::string("cudaMalloc failed: ") + cudaGetErrorString(e));
        return e == cudaErrorMemoryAllocation ? CQ_ERR_OOM : CQ_ERR_CUDA;
    }
    return CQ_OK;
}

}  // namespace cq

struct cq_basis {
    int device = 0;
    int natom = 0, nsh = 0, nbf = 0, npair = 0, nprim_pairs = 0;
    // molecules of a batched basis (one molecule for cq_basis_create): every
    // matrix is stored as nmol slots of ld x ld, shell blocks as lds x lds
    int nmol = 1, ld = 0, lds = 0;
    long long mstride = 0;
    std::vector<int> atom_mol, mol_atom_off, mol_sho, mol_bfo, mol_n, mol_nsh;
    std::vector<int> molcls_off;   // NPC x (nmol + 1) pair offsets per class and molecule
    int *d_mol_n = nullptr, *d_mol_bfo = nullptr, *d_mol_nsh = nullptr, *d_mol_sho = nullptr,
        *d_mol_atom_off = nullptr;
    std::pair<int, int> mol_range(int c, int m) const
    {
        return {molcls_off[c * (nmol + 1) + m], molcls_off[c * (nmol + 1) + m + 1]};
    }
    std::vector<double> xyz;
    std::vector<int> Z;
    std::vector<int> L, nprim, poff, atom, bfo;
    std::vector<double> exps, coefs;
    // pair classes
    int cls_off[cq::NPC + 1] = {0};
    std::vector<cq::PairHdr> pairs;
    // tasks per quartet class
    std::vector<int> task_off;   // NQC + 1
    // device data
    double* d_boys = nullptr;
    float* d_boysf = nullptr;
    cq::PairHdr* d_pairs = nullptr;
    cq::PrimPair* d_prims = nullptr;
    cq::PrimPairF* d_primsf = nullptr;
    cq::PrimPairX* d_primsx = nullptr;
    int4* d_tasks = nullptr;
    float* d_Qf = nullptr;
    double* d_Qd = nullptr;
    double* d_scale = nullptr;     // per-function Cartesian component factor
    double* d_ctr = nullptr;       // shell centres
    int* d_L = nullptr;
    int* d_nprim = nullptr;
    int* d_poff = nullptr;
    int* d_bfo = nullptr;
    double* d_exps = nullptr;
    double* d_coef = nullptr;      // normalised (x^L component) coefficients
    double* d_axyz = nullptr;
    double* d_Z = nullptr;
    // per-build scratch (grown on demand)
    int nk_cap = 0;
    double* d_Dp = nullptr;        // nk scaled densities
    cq::acc_t* d_Jp = nullptr;     // J' (two fx_add words per element)
    cq::acc_t* d_Kp = nullptr;     // nk K' (two fx_add words per element)
    float* d_Dmax = nullptr;       // nsh x nsh
    unsigned long long* d_cnt = nullptr;  // 4 totals + per class/precision (quartets, prims)
    cudaEvent_t ev0 = nullptr, ev1 = nullptr;
    // optional per-class profile of the last build
    int profile = 0;
    cudaEvent_t pev[cq::NQC][3][2] = {};   // [class][FP64, FP32, double-float][start, end]
    bool pev_used[cq::NQC][3] = {};
    // builds in passes: one event pair per pass and precision of a class
    std::vector<cudaEvent_t> pev_pass[cq::NQC][3];
    int pev_npass[cq::NQC][3] = {};
    unsigned long long pcnt[cq::NQC][2][2] = {};
    // dense drivers (SCF, RT): library handles and cached one-electron data
    void* blas = nullptr;          // cublasHandle_t
    void* solver = nullptr;        // cusolverDnHandle_t
    int dense_ready = 0;
    int northo = 0;                // columns of the orthogonaliser X (n x northo)
    int ndropped = 0;
    double enuc = 0.0;
    double* d_S = nullptr;
    double* d_H = nullptr;         // core Hamiltonian
    double* d_M = nullptr;         // 3 dipole matrices
    double* d_X = nullptr;         // orthogonaliser, n x northo
    double* d_Xinv = nullptr;      // X^T S, northo x n
    double* d_w = nullptr;         // eigenvalue workspace
    double* d_work = nullptr;      // cusolver workspace
    int lwork = 0;
    int* d_info = nullptr;
    std::vector<void*> dense_bufs; // other driver scratch, freed with the basis
    void* rt = nullptr;            // RT-TDHF buffers (cq_drivers.cu)
    int variant[cq::NQC][3] = {};  // kernel variant per class and precision (FP64, FP32, double-float)
    // cooperative kernel on the screened list, per precision: warp tasks per
    // quartet (at most) and primitive quartets per task (about)
    int list_split[3] = {8, 4, 4};
    int list_chunk[3] = {64, 32, 32};
    // tasks of the warp-cooperative kernel: (bra, ket, primitive range), built
    // for the classes that use it, rebuilt when the variant table changes
    std::vector<int> coop_off;     // NQC + 1
    // compacted quartet lists (per class: FP64 from the front, FP32 from the
    // back of its region), rebuilt on the device by every build
    std::vector<long long> qoff;   // NQC + 1
    int2* d_qlist = nullptr;
    unsigned int* d_qcount = nullptr;   // [NQC][3]
    int* d_task_off = nullptr;          // NQC + 1 (device copy)
    long long* d_qoff = nullptr;        // NQC + 1 (device copy)
    unsigned int* d_tcount = nullptr;   // 3 per task: survivors per precision
    unsigned int* d_toff = nullptr;     // 3 per task: offsets in the class lists
    // side streams for running the class kernels of a build concurrently
    static constexpr int NSIDE = 6;
    cudaStream_t side[NSIDE] = {};
    cudaEvent_t fork_ev = nullptr;
    cudaEvent_t join_ev[NSIDE] = {};
    int4* d_coop_tasks = nullptr;
    bool coop_dirty = true;
    bool coop_list = false;        // cooperative classes read the screened lists
    // large bases: one task per (class, bra pair) and a quartet list of
    // list_cap entries filled and drained in passes of whole tasks
    bool passes = false;
    long long list_cap = 0;
    std::vector<long long> task_cand;   // prefix sums of candidates over tasks (passes only)
    long long* d_pass_qoff = nullptr;   // {0, list_cap}
    // private stream of the batched SCF (graph capture needs a non-default stream)
    cudaStream_t batch_stream = nullptr;
    cudaEvent_t batch_ev = nullptr;
};

namespace cq {
// largest quartet list a basis allocates before switching to passes
// (settable through cq_set_list_capacity)
extern long long g_list_capacity;
constexpr int COOP_CHUNK = 64;   // primitive quartets per cooperative task
// candidate quartets of the cooperative classes above which the cooperative
// kernel reads the screened lists instead of a per-candidate task table
constexpr long long COOP_TASK_CANDIDATES = 4000000;
void launch_jk_class(const cq_basis* b, const JKArgs& a, int qc, int fp32, cudaStream_t s);
int ensure_coop_tasks(cq_basis* b);
int classify_and_launch(const cq_basis* b, JKArgs& a, const cq_fock_opts& o, bool profile, cudaStream_t s,
                        const int* mol_mode = nullptr);
// cq_fock_build with an optional device array of per-molecule modes (see
// ClassifyArgs::mol_mode) and an optional device accumulator of the four
// quartet/primitive totals; no host synchronisation unless stats is given
int fock_build_modes(cq_basis* b, int kind, const void* P, double* J, void* K, const cq_fock_opts* opts,
                     cq_fock_stats* stats, cudaStream_t s, const int* mol_mode, unsigned long long* acc);
}

namespace cq {
void dense_free(cq_basis* b);
}
