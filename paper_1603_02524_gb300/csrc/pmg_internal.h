// Internal data structures of the GB300 p-multigrid DG Poisson library.
//
// Method: Stiller, "Robust multigrid for high-order discontinuous Galerkin
// methods" (arXiv 1603.02524).  Host-side set-up (setup.cpp) builds, per
// p-level and axis, the 1-D operator blocks of Eq. (L:generic), the patch
// eigen-tables of the fast diagonalisation (Sec. 3.1) and the embedded
// interpolation (Sec. 3.2); the CUDA kernels (kernels_*.cu) run every
// per-iteration step; solver.cu orchestrates Algorithms 1 and 2.
#pragma once

#include <atomic>
#include <cstdint>
#include <mutex>
#include <string>
#include <vector>

#include <cuda_runtime.h>

#include "../../include/pmg.h"
#include "dfloat.cuh"

namespace pmg {

// process-wide count of kernel launches (pmg_kernel_launches)
extern std::atomic<unsigned long long> g_launches;
inline void count_launch() { g_launches.fetch_add(1, std::memory_order_relaxed); }

constexpr int kMaxLevels = 7;     // P <= 32 -> levels P_l = 1, 2, 4, ..., 32
constexpr int kMaxRhs = 64;       // right-hand sides of one hierarchy (pmg_options.nrhs)

// Launch-shape figures (SM count, resident blocks, kernel attributes) kept per
// device: a process may drive several GPUs, from several host threads.  with()
// runs fn(entry) under the lock, after init(entry, device) has filled the current
// device's entry on its first use; both return PMG_OK or an error status.
constexpr int kMaxDevices = 64;
template <typename T>
struct PerDevice {
  std::mutex mu;
  T val[kMaxDevices];
  bool ready[kMaxDevices] = {};
  template <typename Init, typename Fn>
  int with(Init&& init, Fn&& fn) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return PMG_ECUDA;
    if (dev < 0 || dev >= kMaxDevices) return PMG_EINVAL;
    std::lock_guard<std::mutex> lock(mu);
    if (!ready[dev]) {
      const int rc = init(val[dev], dev);
      if (rc != PMG_OK) return rc;
      ready[dev] = true;
    }
    return fn(val[dev]);
  }
};

// ---------------------------------------------------------------------------
// host-side 1-D discretisation of one axis at one order (Sec. 2.4)
// ---------------------------------------------------------------------------
struct Axis1DHost {
  int P = 0, NP = 0, Ne = 0;
  bool periodic = false;
  double beta = 0.0, mu_star = 1.0;
  std::vector<double> dx;        // element widths
  std::vector<double> eta, rho;  // GLL nodes / weights
  std::vector<double> D;         // D[i*NP+k] = phi_k'(eta_i)
  std::vector<double> Ls;        // standard stiffness
  // per element m: blocks of Eq. (L:generic) (walls folded into L0, reading C2)
  std::vector<double> L0, Lm, Lp;   // [Ne][NP][NP]
  std::vector<double> M;            // [Ne*NP] diagonal mass
  // rank form of the neighbour coupling used by the apply kernel:
  // (L^- u^-)_i = -aL D_{0,i} u^-_P + d_{i0} (bL (D u^-)_P - cL u^-_P)
  // (L^+ u^+)_i =  aR D_{P,i} u^+_0 - d_{iP} (bR (D u^+)_0 + cR u^+_0)
  std::vector<double> cpl;          // [Ne][8] = aL bL cL hasL aR bR cR hasR
  double entry(int I, int J) const; // global 1-D stiffness entry L(I, J)
};

// ---------------------------------------------------------------------------
// device tables of one level
// ---------------------------------------------------------------------------
template <typename T>
struct ApplyTables {
  // Per axis d and element index m along d:
  // (accumulate form of apply_rowform: rows transposed and padded to 16 bytes)
  const T* L0[3];     // [Ne_d][NP*pad(NP)] M_d^-1 L^0 (row-scaled); even-odd folded when sym
  const int* sym[3];  // [Ne_d]         1: M^-1 L^0 is centro-symmetric (folded form)
  const T* M[3];      // [Ne_d][NP]     diagonal mass M_d
  const T* cpl[3];    // [Ne_d][2pad(NP)+8] neighbour coupling, scaled by M_d^-1 (see setup)
  const T* D0;        // D_{0,k}
  const T* DP;        // D_{P,k}
  const double* D0d;  // the same rows in FP64 (the double-float apply's neighbour terms)
  const double* DPd;
};
// Host-side apply tables of one axis (built from Axis1DHost by apply_axis_tables).
struct ApplyAxisHost {
  std::vector<double> L0, cpl;
  std::vector<int> sym;
};
// fold_coupling: mirrored neighbour-coupling rows stored folded and flagged (the FP64 and
// double-float applies use them; the fp32 apply keeps the rows unfolded)
void apply_axis_tables(const Axis1DHost& a, ApplyAxisHost& t, bool fold_coupling = true);
// the same tables in the apply kernel's accumulate form, rows padded to W entries
void apply_rowform(const ApplyAxisHost& t, int NP, int W, std::vector<double>& L0r,
                   std::vector<double>& cplr);

// One axis of a family of patches (EA, or FA with this axis normal/lateral).
template <typename T>
struct FdmAxis {
  int n;          // patch length along this axis
  int count;      // number of patch positions
  int start0;     // first global 1-D index of patch p: start0 + p * NP
  int N;          // global 1-D size Ne * NP (1 for the trivial z axis in 2-D)
  int periodic;
  int phys;       // physical axis (0 x, 1 y, 2 z) this patch-buffer axis maps to
  const T* S;     // [count][n*n] forward table S[p][a][i]: node a, mode i
  const T* W;     // [count][n*n] backward table (diag(w) S)^T, mode-major (times omega on axis 0)
  const T* lam;   // [count][n] eigenvalues in mode order
  const int* sym; // [count] 1: centro-symmetric, tables stored in even-odd folded form
  // [count] (tcgen05 kernel; null elsewhere): the first position whose S, W and lam are
  // identical to this one's, so that a CTA walking consecutive positions reloads tables
  // only when they change (interior positions of a uniform axis all share one set)
  const int* tabid;
  // Several right-hand sides stack copies of the grid along its last axis, with walls
  // between the copies: there, positions come in blocks of bpos (0: no blocks), and
  // position p starts at start0 + (p - (p / bpos) * bskip) * NP (bskip = 1 for the face
  // family normal to that axis, whose blocks hold one face more than elements)
  int bpos;
  int bskip;
};
template <typename T>
__host__ __device__ __forceinline__ int patch_start(const FdmAxis<T>& ax, int p, int npp) {
  const int pe = ax.bpos ? p - (p / ax.bpos) * ax.bskip : p;
  return ax.start0 + pe * npp;
}

// Largest CTA any patch-kernel launch may use (the autotuner's candidates stay
// within it; it caps registers at 128 per thread).
constexpr int kFdmMaxThreads = 512;
// Smallest patch (nodes) that the tcgen05 patch kernel takes (PMG_PREC_MIXED_TF32);
// measured on GB300: 13^3 EA patches break even with the SIMT kernel, smaller
// ones run about 2x faster on the SIMT kernel.
constexpr long long kTcMinPatchNodes = 13 * 13 * 13;

template <typename T>
struct FdmFamily {
  FdmAxis<T> ax[3];    // patch-buffer axes a (fastest), b, c
  int count_total;
  int tc = 0;          // fp32 only: 1 = line passes on the tensor cores (tables unfolded)
  int threads = 0;     // CTA size chosen by the autotuner (0: the kernel's default)
  int variant = -1;    // fp32: 0 one patch per CTA, 1 pipelined persistent CTAs, -1 default
  // patches too large for shared memory (3-D, P = 32): the patch buffers of the
  // persistent CTAs in global memory, scratch_ctas buffers of scratch_stride entries
  T* scratch = nullptr;
  int scratch_ctas = 0;
  long long scratch_stride = 0;
  // FP64: 1 / (lambda_a + lambda_b + lambda_c) precomputed per combination of
  // distinct axis eigenvalue sets (uid[q][p]: set of position p on axis q; few
  // sets on uniform grids); null where the combinations would be too many
  const T* inv = nullptr;
  const int* uid[3] = {nullptr, nullptr, nullptr};
  int ucount[3] = {1, 1, 1};
  // device status word of the owning hierarchy: the tcgen05 kernel sets PMG_ETIMEOUT
  // there when a bounded wait gives up (null: counted only)
  int* status = nullptr;
  // test hook of the tcgen05 kernel (0 = off): its blocks wait on a barrier that
  // nothing completes and give up after stall_ns nanoseconds
  unsigned int stall_ns = 0;
};

struct LevelDims {
  int dim, P, NP, NPz;       // NPz = NP (3-D) or 1 (2-D)
  int ne[3];                 // elements per axis (ne[2] = 1 in 2-D)
  long long nelem, ndof;
  int periodic;
};

// all device allocations of one level, for one scalar type
template <typename T>
struct LevelDev {
  ApplyTables<T> at{};
  FdmFamily<T> ea{};
  FdmFamily<T> fa[3]{};
  T* u = nullptr;      // level solution / correction
  T* f = nullptr;      // level right-hand side
  T* r = nullptr;      // residual scratch
  std::vector<void*> owned;
};

struct CoarseFdm {            // exact global fast-diagonalisation solve at P = 1
  int N[3];                   // global 1-D sizes (2 Ne_d)
  double* S[3];               // [N][N] (node, mode)
  double* lam[3];             // [N]
  double* tmp[2];
  double lam_max;
};

// host patch tables along one axis (see FdmAxis): S, W^T, lambda, symmetry flags
struct AxisTables {
  int n = 0, count = 0, start0 = 0;
  int bpos = 0, bskip = 0;   // stacked copies (see FdmAxis)
  std::vector<double> S, W, lam;
  std::vector<int> sym;
};

struct Grid {
  int dim = 3, P = 1, bc_periodic = 0;
  int ne[3] = {1, 1, 1};
  std::vector<double> spacing[3];
  double mu_star = 1.0;
  double beta[3] = {0, 0, 0};
};

// Result of one device-resident solve, written by the device.
struct SolveResult {
  double r0, rn;
  int iterations, status;
};

struct Hier {
  Grid grid;
  pmg_options opt{};
  int L = 0;                       // finest level index
  int nrhs = 1;                    // right-hand sides (segments of every level vector)
  long long n1 = 0;                // finest-level unknowns of one right-hand side
  LevelDims dims[kMaxLevels];
  std::vector<Axis1DHost> axes[kMaxLevels];   // per level, per axis
  int No[kMaxLevels];
  LevelDev<double> d64[kMaxLevels];
  LevelDev<float> d32[kMaxLevels];
  bool has32 = false;
  // interpolation J_l (fine NP x coarse NP), l = 1..L; the host copy feeds the
  // even-odd folded coefficients that the transfer kernels take as parameters
  double* J64[kMaxLevels] = {};
  float* J32[kMaxLevels] = {};
  std::vector<double> Jhost[kMaxLevels];
  CoarseFdm coarse{};
  // host copies of the patch-table shapes and symmetry flags (S/W/lam cleared)
  std::vector<AxisTables> ec_shape[kMaxLevels], fc_shape[kMaxLevels];
  // MGCG work vectors (fine level, fp64)
  double *r = nullptr, *r_old = nullptr, *p = nullptr, *q = nullptr, *z = nullptr;
  double* scal = nullptr;          // device scalars
  double* partial = nullptr;       // reduction partials
  unsigned* counter = nullptr;     // last-block counter
  int* dstatus = nullptr;          // device status word
  int* duz = nullptr;              // 1 if the solve's initial u has a nonzero entry
  double* hscal = nullptr;         // pinned host mirror (host_mirror_bytes): control words, results
  double *g_host_stage = nullptr, *u_host_stage = nullptr;   // device buffers for solve_host
  std::vector<void*> owned;
  std::string err;
  int nsm = 152;
  // CUDA graph of the MGCG preconditioner (V-cycle r -> z on the fixed work
  // vectors), captured on first reuse on a private stream, replayed on the
  // caller's stream; state 0 = not yet, 1 = captured, -1 = capture unsupported
  cudaStream_t cap_stream = nullptr;
  cudaGraphExec_t pc_exec = nullptr;
  int pc_state = 0;
  int pc_calls = 0;
  unsigned long long pc_launches = 0;
  // Whole MGCG solve as one CUDA graph (a device-side `while` node runs the
  // iterations), captured for fixed (g, u, rtol) once the kernels have run
  // directly; state 0 = not yet, 1 = captured, -1 = conditional graphs unsupported
  cudaStream_t cap_stream2 = nullptr;
  cudaGraphExec_t sv_exec = nullptr;
  int sv_state = 0;
  const double* sv_g = nullptr;
  double* sv_u = nullptr;
  double sv_rtol = -1.0;
  unsigned long long sv_fixed = 0, sv_iter = 0;   // kernels outside / per iteration
  double* hist = nullptr;          // device residual history [max_iter + 1]
  SolveResult* dres = nullptr;     // device result of the captured solve
  bool coarse_split = false;       // coarse solve as separate launches (graph capture)
  ApplyTables<dfloat> at_df{};     // finest-level apply tables in double-float (outer_apply DF)
};

// scalar slots of one segment (right-hand side); reductions write two consecutive slots
enum { S_DELTA = 0, S_PQ = 2, S_RR = 4, S_ZR = 6, S_ZRO = 7, S_MEAN = 8, S_RR0 = 10, S_NUM = 16 };
// control words (int) of a solve over k segments: [C_STATUS] global status word (set by
// kernels whose failure concerns every segment, e.g. the tcgen05 patch kernel's timed-out
// waits), [C_ITER] iteration counter, [C_ACTIVE] segments still iterating; segment s at
// kCtrlSeg + 4 s: its status word, iterations, result and active flag (same C_* slots,
// C_RES the result)
enum { C_STATUS = 0, C_ITER = 1, C_RES = 2, C_ACTIVE = 3 };
constexpr int kCtrlSeg = 4;
// reduction partials of one segment (two per block, at most 152 x 8 blocks)
constexpr int kPartialStride = 2 * 152 * 8 + 64;
// pinned host mirror of a hierarchy with k segments: room for the control words or the
// k solve results
inline size_t host_mirror_bytes(int k) {
  const size_t a = sizeof(int) * (size_t)(kCtrlSeg + 4 * k), b = sizeof(SolveResult) * (size_t)k;
  return (a > b ? a : b) + 64;
}

// ----------------------------------------------------------------------------
// set-up (setup.cpp)
// ----------------------------------------------------------------------------
void build_axis(Axis1DHost& a, int P, const std::vector<double>& dx, bool periodic, double beta,
                double mu_star);
void gll_nodes(int P, std::vector<double>& eta, std::vector<double>& rho);
void lagrange_matrix(const std::vector<double>& nodes, const std::vector<double>& x,
                     std::vector<double>& B);
int sym_eig_jacobi(int n, std::vector<double>& A, std::vector<double>& V, std::vector<double>& lam);
int overlap_nodes(int P_l, int policy);
double transition(double x, int weighting);
void ec_axis_tables(const Axis1DHost& a, int No, int weighting, double tau, AxisTables& t);
void fc_axis_tables(const Axis1DHost& a, int weighting, double tau, AxisTables& t);
void unfold_tables(AxisTables& t);
void global_axis_eig(const Axis1DHost& a, std::vector<double>& S, std::vector<double>& lam);
// k copies of an axis (or of its patch tables) one after the other, separated by walls
void stack_axis(const Axis1DHost& a, int k, Axis1DHost& out);
void stack_tables(const AxisTables& t, int k, int skip, AxisTables& out);

// ----------------------------------------------------------------------------
// kernels (launch wrappers)
// ----------------------------------------------------------------------------
// unz (optional): a device word, 0 if u is identically zero (any_nonzero found no
// nonzero entry); the kernel then forms v = f (or 0) without the apply
template <typename T>
int launch_apply(const LevelDims& dm, const ApplyTables<T>& at, const T* u, const T* f, T* v,
                 cudaStream_t s, const int* unz = nullptr);
// Transfers: J the device copy of J_l (used where the kernels contract densely,
// 3-D P = 32 <-> 16), Jh the host copy (fine x coarse, row-major), folded into the
// kernel parameters of the others.
template <typename T>
int launch_residual_restrict(const LevelDims& dm, const ApplyTables<T>& at, const T* u, const T* f,
                             const T* J, const double* Jh, T* fc, cudaStream_t s);
template <typename T>
int launch_fdm(const LevelDims& dm, const FdmFamily<T>& fam, const T* r, T* u, cudaStream_t s);
template <typename T>
int launch_restrict(const LevelDims& fine, const LevelDims& coarse, const T* J, const double* Jh,
                    const T* rf, T* fc, cudaStream_t s);
template <typename T>
int launch_prolong(const LevelDims& fine, const LevelDims& coarse, const T* J, const double* Jh,
                   const T* uc, T* uf, cudaStream_t s);
// *flag = 1 if x[0..n) has an entry != 0 (flag zeroed by the caller)
void launch_any_nonzero(const double* x, long long n, int* flag, cudaStream_t s);
int launch_apply_df(const LevelDims& dm, const ApplyTables<dfloat>& at, const double* u,
                    const double* f, double* v, cudaStream_t s, const int* unz = nullptr);
int launch_coarse_fdm(const LevelDims& dm, const CoarseFdm& c, const double* f, double* u,
                      cudaStream_t s, bool cooperative = true);
template <typename Ta, typename Tb>
void launch_convert(const Ta* in, Tb* out, long long n, cudaStream_t s);
void launch_dot(const double* x, const double* y, const double* y2, long long n, int k, double* partial,
                unsigned* counter, double* out, int nblocks, cudaStream_t s);
void launch_cg_update(double* u, double* r, double* r_old, const double* p, const double* q,
                      const double* scal, int save_old, long long n, int k, double* partial,
                      unsigned* counter, int* ctrl, int nblocks, cudaStream_t s, const int* it_dev = nullptr);
void launch_p_update(double* p, const double* z, const double* scal, int first, long long n, int k,
                     cudaStream_t s, const int* it_dev = nullptr, const int* ctrl = nullptr);
void launch_set_delta(double* scal, int* ctrl, int k, cudaStream_t s);
void launch_solve_begin(double* scal, int* ctrl, double* hist, int hstride, int k,
                        const cudaGraphConditionalHandle* cond, cudaStream_t s);
void launch_solve_control(const double* scal, int* ctrl, double* hist, int hstride, int k, double rtol,
                          int max_iter, const cudaGraphConditionalHandle* cond, cudaStream_t s);
void launch_solve_result(const double* scal, const int* ctrl, SolveResult* out, int k, cudaStream_t s);
void launch_sub_mean(double* x, long long n, double* partial, unsigned* counter, double* scal,
                     int nblocks, cudaStream_t s);
void launch_mass(const LevelDims& dm, const ApplyTables<double>& at, const double* f, double* g,
                 cudaStream_t s);

}  // namespace pmg
