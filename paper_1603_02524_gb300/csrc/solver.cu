// C ABI, hierarchy construction, V-cycle (Algorithm 1) and inexact
// multigrid-preconditioned CG (Algorithm 2) of Stiller, arXiv 1603.02524.
//
// Every per-iteration step is a kernel launched on the caller's stream.  The
// first solve of a hierarchy sequences its iterations from the host (reading the
// residual norm once per iteration); later solves and batches replay CUDA graphs
// whose iteration loop and convergence test run on the device.
#include <algorithm>
#include <array>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <exception>
#include <map>
#include <mutex>
#include <new>

#include "dfloat.cuh"
#include "pmg_internal.h"

namespace pmg {

std::atomic<unsigned long long> g_launches{0};

int fdm_dispatch_d3(const LevelDims&, const FdmFamily<double>&, const double*, double*, cudaStream_t);
int fdm_dispatch_d2(const LevelDims&, const FdmFamily<double>&, const double*, double*, cudaStream_t);
int fdm_dispatch_f3(const LevelDims&, const FdmFamily<float>&, const float*, float*, cudaStream_t);
int tc_timeouts_take(unsigned int* out);
int fdm_dispatch_f2(const LevelDims&, const FdmFamily<float>&, const float*, float*, cudaStream_t);

template <>
int launch_fdm<double>(const LevelDims& dm, const FdmFamily<double>& fam, const double* r,
                       double* u, cudaStream_t s) {
  return dm.dim == 3 ? fdm_dispatch_d3(dm, fam, r, u, s) : fdm_dispatch_d2(dm, fam, r, u, s);
}
template <>
int launch_fdm<float>(const LevelDims& dm, const FdmFamily<float>& fam, const float* r, float* u,
                      cudaStream_t s) {
  return dm.dim == 3 ? fdm_dispatch_f3(dm, fam, r, u, s) : fdm_dispatch_f2(dm, fam, r, u, s);
}

namespace {

struct CudaError : std::exception {
  int code;
  std::string msg;
  CudaError(int c, std::string m) : code(c), msg(std::move(m)) {}
};

#define PMG_CUDA(call)                                                                   \
  do {                                                                                   \
    cudaError_t e_ = (call);                                                             \
    if (e_ != cudaSuccess)                                                               \
      throw CudaError(e_ == cudaErrorMemoryAllocation ? PMG_ENOMEM : PMG_ECUDA,          \
                      std::string(#call) + ": " + cudaGetErrorString(e_));               \
  } while (0)

#define PMG_CHECK(expr)                                                                  \
  do {                                                                                   \
    int st_ = (expr);                                                                    \
    if (st_ != PMG_OK) throw CudaError(st_, std::string(#expr) + " failed");             \
  } while (0)

template <typename T>
T* dev_alloc(std::vector<void*>& owned, size_t count) {
  void* p = nullptr;
  PMG_CUDA(cudaMalloc(&p, count * sizeof(T) + 16));
  owned.push_back(p);
  return static_cast<T*>(p);
}

template <typename T>
T* dev_upload(std::vector<void*>& owned, const std::vector<double>& host) {
  std::vector<T> tmp(host.begin(), host.end());
  T* d = dev_alloc<T>(owned, tmp.size() ? tmp.size() : 1);
  if (!tmp.empty()) PMG_CUDA(cudaMemcpy(d, tmp.data(), tmp.size() * sizeof(T), cudaMemcpyHostToDevice));
  return d;
}

int* dev_upload_int(std::vector<void*>& owned, const std::vector<int>& host) {
  int* d = dev_alloc<int>(owned, host.size() ? host.size() : 1);
  if (!host.empty()) PMG_CUDA(cudaMemcpy(d, host.data(), host.size() * sizeof(int), cudaMemcpyHostToDevice));
  return d;
}

// per-level smoother parameters (0 selects the default)
double level_omega(const pmg_options& o, int l) {
  return (l >= 1 && l < 8 && o.omega_level[l] > 0.0) ? o.omega_level[l] : o.omega;
}
double level_tau(const pmg_options& o, int l) {
  return (l >= 1 && l < 8 && o.tau_level[l] > 0.0) ? o.tau_level[l] : 1.0;
}

// trivial third axis of a 2-D patch family
template <typename T>
FdmAxis<T> trivial_axis(std::vector<void*>& owned) {
  FdmAxis<T> ax{};
  ax.n = 1;
  ax.count = 1;
  ax.start0 = 0;
  ax.N = 1;
  ax.periodic = 0;
  ax.phys = 2;
  ax.S = dev_upload<T>(owned, {1.0});
  ax.W = dev_upload<T>(owned, {1.0});
  ax.lam = dev_upload<T>(owned, {0.0});
  ax.sym = dev_upload_int(owned, {0});
  return ax;
}

// x rounded to the nearest tf32 value (8 exponent bits, 10 stored mantissa bits;
// ties to even), as an fp32 value in a double
double round_to_tf32(double x) {
  float f = (float)x;
  uint32_t u;
  std::memcpy(&u, &f, 4);
  if ((u & 0x7f800000u) != 0x7f800000u) {
    u += 0xFFFu + ((u >> 13) & 1u);
    u &= 0xFFFFE000u;
  }
  std::memcpy(&f, &u, 4);
  return (double)f;
}

// scale: omega for the first patch-buffer axis (folds the damping into W), 1 otherwise;
// tf32: tables rounded to tf32 for the tensor-core patch kernel
template <typename T>
FdmAxis<T> upload_axis(std::vector<void*>& owned, const AxisTables& t, const Axis1DHost& a, int phys,
                       double scale, bool tf32 = false) {
  FdmAxis<T> ax{};
  ax.n = t.n;
  ax.count = t.count;
  ax.start0 = t.start0;
  ax.bpos = t.bpos;
  ax.bskip = t.bskip;
  ax.N = a.Ne * a.NP;
  ax.periodic = a.periodic ? 1 : 0;
  ax.phys = phys;
  std::vector<double> S(t.S), W(t.W);
  for (double& x : W) x *= scale;
  if (tf32) {
    for (double& x : S) x = round_to_tf32(x);
    for (double& x : W) x = round_to_tf32(x);
  }
  ax.S = dev_upload<T>(owned, S);
  ax.W = dev_upload<T>(owned, W);
  ax.lam = dev_upload<T>(owned, t.lam);
  ax.sym = dev_upload_int(owned, t.sym);
  if (tf32) {
    // table identity of each position: the first earlier position with the same values
    const size_t nn = (size_t)t.n * t.n;
    std::vector<int> id(t.count), reps;
    for (int p = 0; p < t.count; ++p) {
      id[p] = p;
      for (int q : reps) {
        if (std::equal(S.begin() + p * nn, S.begin() + (p + 1) * nn, S.begin() + q * nn) &&
            std::equal(W.begin() + p * nn, W.begin() + (p + 1) * nn, W.begin() + q * nn) &&
            std::equal(t.lam.begin() + (size_t)p * t.n, t.lam.begin() + (size_t)(p + 1) * t.n,
                       t.lam.begin() + (size_t)q * t.n)) {
          id[p] = q;
          break;
        }
      }
      if (id[p] == p) reps.push_back(p);
    }
    ax.tabid = dev_upload_int(owned, id);
  }
  return ax;
}

// operator-apply tables of level l in arithmetic T
template <typename T>
ApplyTables<T> build_apply_tables(Hier& h, int l, std::vector<void*>& own) {
  const LevelDims& dm = h.dims[l];
  auto& ax = h.axes[l];
  ApplyTables<T> at{};
  for (int d = 0; d < 3; ++d) {
    int dd = d < dm.dim ? d : 0;
    ApplyAxisHost t;
    apply_axis_tables(ax[dd], t, sizeof(T) == 8);
    std::vector<double> L0r, cplr;
    apply_rowform(t, dm.NP, 16 / (int)sizeof(T), L0r, cplr);
    at.L0[d] = dev_upload<T>(own, L0r);
    at.sym[d] = dev_upload_int(own, t.sym);
    at.M[d] = dev_upload<T>(own, ax[dd].M);
    at.cpl[d] = dev_upload<T>(own, cplr);
  }
  std::vector<double> D0(dm.NP), DP(dm.NP);
  for (int k = 0; k < dm.NP; ++k) {
    D0[k] = ax[0].D[0 * dm.NP + k];
    DP[k] = ax[0].D[(size_t)(dm.NP - 1) * dm.NP + k];
  }
  at.D0 = dev_upload<T>(own, D0);
  at.DP = dev_upload<T>(own, DP);
  at.D0d = dev_upload<double>(own, D0);
  at.DPd = dev_upload<double>(own, DP);
  return at;
}

// Shared memory the one-patch-per-CTA kernel needs for a patch of n0 x n1 x n2
// (as fdm_smem_bytes); beyond 227 KB the patch buffers go to global scratch.
template <typename T>
size_t patch_smem_bytes(int n0, int n1, int n2) {
  const int W = 16 / (int)sizeof(T);
  auto pad = [W](long long n) { return (n + W - 1) / W * W; };
  const long long NN = (long long)n0 * n1 * n2;
  const long long tf = (long long)n0 * pad(n0) + (long long)n1 * pad(n1) + (long long)n2 * pad(n2);
  return sizeof(long long) * (size_t)((n0 + n1 + n2 + 1) / 2 * 2 + ((long long)n1 * n2 + 1) / 2 * 2) +
         sizeof(T) * (size_t)(pad(NN) + 2 * tf + n0 + n1 + n2);
}

template <typename T>
void attach_scratch(Hier& h, FdmFamily<T>& fam, std::vector<void*>& own) {
  const int n0 = fam.ax[0].n, n1 = fam.ax[1].n, n2 = fam.ax[2].n;
  if (patch_smem_bytes<T>(n0, n1, n2) <= 227 * 1024) return;
  fam.scratch_stride = ((long long)n0 * n1 * n2 + 31) / 32 * 32;
  // two CTAs per SM, fewer (down to one per SM) when their buffers would not stay
  // within ~96 MB of the 126 MB L2
  const long long per = fam.scratch_stride * (long long)sizeof(T);
  long long ctas = (96LL << 20) / per;
  if (ctas > 2 * h.nsm) ctas = 2 * h.nsm;
  if (ctas < h.nsm) ctas = h.nsm;
  fam.scratch_ctas = (int)ctas;
  fam.scratch = dev_alloc<T>(own, (size_t)fam.scratch_ctas * fam.scratch_stride);
}

// FP64 families: precompute 1 / ((lambda_a + lambda_b) + lambda_c) (the kernel's sum
// order, IEEE division) for every combination of distinct per-axis eigenvalue sets;
// on uniform grids an axis has at most three (the two walls, the interior), so the
// table is small and the patch kernel replaces a Newton reciprocal per node by one
// load.  Skipped when the combinations would take more than 32 MB.
template <typename T>
void attach_inverse_table(FdmFamily<T>& fam, const AxisTables* const (&tab)[3], std::vector<void*>& own) {
  if (sizeof(T) != 8 || fam.tc) return;
  std::vector<int> uid[3];
  std::vector<std::vector<double>> rep[3];
  long long combos = 1;
  for (int q = 0; q < 3; ++q) {
    const int n = fam.ax[q].n, count = fam.ax[q].count;
    std::map<std::vector<double>, int> ids;
    uid[q].resize(count);
    for (int p = 0; p < count; ++p) {
      std::vector<double> lam = tab[q] ? std::vector<double>(tab[q]->lam.begin() + (size_t)p * n,
                                                             tab[q]->lam.begin() + (size_t)(p + 1) * n)
                                       : std::vector<double>(1, 0.0);
      auto it = ids.find(lam);
      if (it == ids.end()) {
        it = ids.emplace(lam, (int)rep[q].size()).first;
        rep[q].push_back(lam);
      }
      uid[q][p] = it->second;
    }
    combos *= (long long)rep[q].size();
  }
  const int na = fam.ax[0].n, nb = fam.ax[1].n, nc = fam.ax[2].n;
  const long long nn = (long long)na * nb * nc;
  if (combos * nn * (long long)sizeof(T) > (32LL << 20)) return;
  std::vector<double> inv((size_t)(combos * nn));
  for (int i2 = 0; i2 < (int)rep[2].size(); ++i2)
    for (int i1 = 0; i1 < (int)rep[1].size(); ++i1)
      for (int i0 = 0; i0 < (int)rep[0].size(); ++i0) {
        const long long combo = ((long long)i2 * (long long)rep[1].size() + i1) * (long long)rep[0].size() + i0;
        double* dst = &inv[(size_t)(combo * nn)];
        for (int c = 0; c < nc; ++c)
          for (int b = 0; b < nb; ++b)
            for (int a = 0; a < na; ++a)
              dst[((size_t)c * nb + b) * na + a] = 1.0 / ((rep[0][i0][a] + rep[1][i1][b]) + rep[2][i2][c]);
      }
  fam.inv = dev_upload<T>(own, inv);
  for (int q = 0; q < 3; ++q) {
    fam.uid[q] = dev_upload_int(own, uid[q]);
    fam.ucount[q] = (int)rep[q].size();
  }
}

template <typename T>
void build_level_dev(Hier& h, int l, LevelDev<T>& dev, const std::vector<AxisTables>& ec,
                     const std::vector<AxisTables>& fc) {
  const LevelDims& dm = h.dims[l];
  auto& ax = h.axes[l];
  auto& own = dev.owned;
  dev.at = build_apply_tables<T>(h, l, own);
  dev.u = dev_alloc<T>(own, dm.ndof);
  dev.f = dev_alloc<T>(own, dm.ndof);
  dev.r = dev_alloc<T>(own, dm.ndof);
  if (l == 0) return;
  // tensor-core line passes (fp32, 3-D) apply the full tables: unfold even-odd ones
  int tc = (sizeof(T) == 4 && dm.dim == 3)
               ? (h.opt.precision == PMG_PREC_MIXED_TC ? 1 : (h.opt.precision == PMG_PREC_MIXED_TF32 ? 2 : 0))
               : 0;
  if (tc == 2) {
    // the tcgen05 kernel pays a fixed latency per line pass; small patches stay on
    // the SIMT kernel (folded tables), which is faster there
    const long long nn = (long long)(h.opt.smoother == PMG_SMOOTHER_EA ? ec[0].n : fc[0].n) * ec[1].n * ec[2].n;
    if (nn < kTcMinPatchNodes) tc = 0;
  }
  std::vector<AxisTables> ecu, fcu;
  const std::vector<AxisTables>& E = tc ? (ecu = ec) : ec;
  const std::vector<AxisTables>& F = tc ? (fcu = fc) : fc;
  if (tc) {
    for (auto& t : ecu) unfold_tables(t);
    for (auto& t : fcu) unfold_tables(t);
  }
  if (h.opt.smoother == PMG_SMOOTHER_EA) {
    FdmFamily<T> fam{};
    fam.count_total = 1;
    fam.tc = tc;
    for (int q = 0; q < 3; ++q) {
      if (q < dm.dim) {
        fam.ax[q] = upload_axis<T>(own, E[q], ax[q], q, q == 0 ? level_omega(h.opt, l) : 1.0, tc == 2);
        fam.count_total *= E[q].count;
      } else {
        fam.ax[q] = trivial_axis<T>(own);
      }
    }
    attach_scratch<T>(h, fam, own);
    const AxisTables* tab[3] = {nullptr, nullptr, nullptr};
    for (int q = 0; q < dm.dim; ++q) tab[q] = &E[q];
    attach_inverse_table<T>(fam, tab, own);
    dev.ea = fam;
  } else {
    for (int nrm = 0; nrm < dm.dim; ++nrm) {
      FdmFamily<T> fam{};
      fam.tc = tc;
      fam.ax[0] = upload_axis<T>(own, F[nrm], ax[nrm], nrm, level_omega(h.opt, l), tc == 2);
      fam.count_total = F[nrm].count;
      int q = 1;
      for (int d = 0; d < dm.dim; ++d) {
        if (d == nrm) continue;
        fam.ax[q] = upload_axis<T>(own, E[d], ax[d], d, 1.0, tc == 2);
        fam.count_total *= E[d].count;
        ++q;
      }
      for (; q < 3; ++q) fam.ax[q] = trivial_axis<T>(own);
      attach_scratch<T>(h, fam, own);
      const AxisTables* tab[3] = {&F[nrm], nullptr, nullptr};
      for (int d = 0, qq = 1; d < dm.dim; ++d)
        if (d != nrm) tab[qq++] = &E[d];
      attach_inverse_table<T>(fam, tab, own);
      dev.fa[nrm] = fam;
    }
  }
}

int reduce_blocks(long long n) {
  long long b = (n + 255) / 256;
  if (b > 152 * 8) b = 152 * 8;
  if (b < 1) b = 1;
  return (int)b;
}

// ---------------------------------------------------------------------------
// smoothing, V-cycle
// ---------------------------------------------------------------------------
template <typename T>
LevelDev<T>& lev(Hier& h, int l);
template <>
LevelDev<double>& lev<double>(Hier& h, int l) { return h.d64[l]; }
template <>
LevelDev<float>& lev<float>(Hier& h, int l) { return h.d32[l]; }

// nsteps Schwarz iterations on level l: u updated in place; u_zero says that u
// is known to be 0 on entry (then the first residual is f itself).
template <typename T>
void smooth_level(Hier& h, int l, T* u, const T* f, int nsteps, bool u_zero, cudaStream_t s) {
  LevelDev<T>& d = lev<T>(h, l);
  const LevelDims& dm = h.dims[l];
  for (int st = 0; st < nsteps; ++st) {
    if (h.opt.smoother == PMG_SMOOTHER_EA) {
      const T* r = f;
      if (!(u_zero && st == 0)) {
        PMG_CHECK(launch_apply<T>(dm, d.at, u, f, d.r, s));
        r = d.r;
      }
      PMG_CHECK(launch_fdm<T>(dm, d.ea, r, u, s));
    } else {
      for (int nrm = 0; nrm < dm.dim; ++nrm) {       // reading C12: same order pre and post
        const T* r = f;
        if (!(u_zero && st == 0 && nrm == 0)) {
          PMG_CHECK(launch_apply<T>(dm, d.at, u, f, d.r, s));
          r = d.r;
        }
        PMG_CHECK(launch_fdm<T>(dm, d.fa[nrm], r, u, s));
      }
    }
  }
}

int ns_level(const Hier& h, int l, bool post) {
  int base = post ? h.opt.ns_post : h.opt.ns_pre;
  return h.opt.variable_v ? base << (h.L - l) : base;
}

// Algorithm 1 with u_L = 0 on entry: uL = MultigridCycle(0, fL).
template <typename T>
void vcycle(Hier& h, const T* fL, T* uL, cudaStream_t s) {
  const int L = h.L;
  const T* f[kMaxLevels];
  T* u[kMaxLevels];
  for (int l = 0; l < L; ++l) {
    f[l] = lev<T>(h, l).f;
    u[l] = lev<T>(h, l).u;
  }
  f[L] = fL;
  u[L] = uL;
  for (int l = L; l >= 1; --l) {
    LevelDev<T>& d = lev<T>(h, l);
    PMG_CUDA(cudaMemsetAsync(u[l], 0, sizeof(T) * h.dims[l].ndof, s));
    smooth_level<T>(h, l, u[l], f[l], ns_level(h, l, false), true, s);
    T* J = nullptr;
    if constexpr (sizeof(T) == 8) J = (T*)h.J64[l]; else J = (T*)h.J32[l];
    // f_{l-1} = I^T (f_l - A u_l): one fused kernel, else residual and restriction apart
    const int rr = launch_residual_restrict<T>(h.dims[l], d.at, u[l], f[l], J, h.Jhost[l].data(),
                                               lev<T>(h, l - 1).f, s);
    if (rr == PMG_EINVAL) {
      PMG_CHECK(launch_apply<T>(h.dims[l], d.at, u[l], f[l], d.r, s));
      PMG_CHECK(launch_restrict<T>(h.dims[l], h.dims[l - 1], J, h.Jhost[l].data(), d.r, lev<T>(h, l - 1).f, s));
    } else {
      PMG_CHECK(rr);
    }
  }
  // coarse grid solution in fp64 (Algorithm 1, A_0^+ f_0)
  if constexpr (sizeof(T) == 8) {
    PMG_CHECK(launch_coarse_fdm(h.dims[0], h.coarse, h.d64[0].f, h.d64[0].u, s, !h.coarse_split));
  } else {
    launch_convert<float, double>(h.d32[0].f, h.d64[0].f, h.dims[0].ndof, s);
    PMG_CHECK(launch_coarse_fdm(h.dims[0], h.coarse, h.d64[0].f, h.d64[0].u, s, !h.coarse_split));
    launch_convert<double, float>(h.d64[0].u, h.d32[0].u, h.dims[0].ndof, s);
  }
  for (int l = 1; l <= L; ++l) {
    T* J = nullptr;
    if constexpr (sizeof(T) == 8) J = (T*)h.J64[l]; else J = (T*)h.J32[l];
    PMG_CHECK(launch_prolong<T>(h.dims[l], h.dims[l - 1], J, h.Jhost[l].data(), u[l - 1], u[l], s));
    smooth_level<T>(h, l, u[l], f[l], ns_level(h, l, true), false, s);
  }
}

// z = V-cycle(r) in the hierarchy's precision, fp64 in and out.
void precondition(Hier& h, const double* r, double* z, cudaStream_t s) {
  if (h.opt.preconditioner == PMG_PC_NONE) {         // plain CG: z = r
    PMG_CUDA(cudaMemcpyAsync(z, r, sizeof(double) * h.dims[h.L].ndof, cudaMemcpyDeviceToDevice, s));
    return;
  }
  if (h.opt.precision != PMG_PREC_FP64) {
    const long long n = h.dims[h.L].ndof;
    launch_convert<double, float>(r, h.d32[h.L].f, n, s);
    vcycle<float>(h, h.d32[h.L].f, h.d32[h.L].u, s);
    launch_convert<float, double>(h.d32[h.L].u, z, n, s);
  } else {
    vcycle<double>(h, r, z, s);
  }
}

// z = V-cycle(r) on the MGCG work vectors, replayed from a CUDA graph after the
// first direct call (the direct call also performs one-time kernel set-up).
void precondition_graph(Hier& h, cudaStream_t s) {
  if (h.pc_state == 1) {
    PMG_CUDA(cudaGraphLaunch(h.pc_exec, s));
    g_launches.fetch_add(h.pc_launches, std::memory_order_relaxed);
    return;
  }
  if (h.pc_state == 0 && h.pc_calls++ >= 1) {
    if (!h.cap_stream) PMG_CUDA(cudaStreamCreateWithFlags(&h.cap_stream, cudaStreamNonBlocking));
    const unsigned long long c0 = g_launches.load();
    bool ok = cudaStreamBeginCapture(h.cap_stream, cudaStreamCaptureModeThreadLocal) == cudaSuccess;
    if (ok) {
      try {
        precondition(h, h.r, h.z, h.cap_stream);
      } catch (const CudaError&) {
        ok = false;
      }
      cudaGraph_t graph = nullptr;
      ok = (cudaStreamEndCapture(h.cap_stream, &graph) == cudaSuccess) && ok && graph;
      if (ok) ok = cudaGraphInstantiate(&h.pc_exec, graph, 0) == cudaSuccess;
      if (graph) cudaGraphDestroy(graph);
    }
    cudaGetLastError();                     // clear a failed capture
    g_launches.store(c0);                   // captured launches did not run
    if (ok) {
      h.pc_state = 1;                        // pc_launches: kernels per V-cycle, from the direct call
      precondition_graph(h, s);
      return;
    }
    h.pc_state = -1;
  }
  const unsigned long long c0 = g_launches.load();
  precondition(h, h.r, h.z, s);
  if (h.pc_state == 0) h.pc_launches = g_launches.load() - c0;
}

// The outer CG's operator apply on the finest level: v = A u, or v = f - A u
// (f non-null); FP64, or double-float on the FP32 pipes (outer_apply option).
void outer_apply(Hier& h, const double* u, const double* f, double* v, cudaStream_t s,
                 const int* unz = nullptr) {
  const LevelDims& dm = h.dims[h.L];
  if (h.opt.outer_apply == PMG_OUTER_DF) {
    PMG_CHECK(launch_apply_df(dm, h.at_df, u, f, v, s, unz));
  } else {
    PMG_CHECK(launch_apply<double>(dm, h.d64[h.L].at, u, f, v, s, unz));
  }
}
// Algorithm 2 in three pieces shared by the host-driven solve and the captured one, for
// all nrhs right-hand sides (segments) of the hierarchy at once; each segment has its
// own scalars, convergence test and result, the V-cycle and operator applies run on
// all segments together.
//   cg_begin:     r = g - A u (periodic: projected), ||r_0|| per segment, r_old = 0
//   cg_iteration: z = V-cycle(r), beta and p (the first iteration: p = z), delta,
//                 q = A p, alpha, the u and r updates, the tests ||r|| <= rtol ||r_0||
//   cg_end:       periodic: zero-mean u; results to res[0..nrhs)
// A captured solve runs cg_iteration as the body of a device-side `while` node whose
// condition the tests set (cond); the host-driven solve reads the control words after
// each iteration and replays the V-cycle from its own graph (direct).
void cg_begin(Hier& h, const double* g, double* u, const cudaGraphConditionalHandle* cond, cudaStream_t s) {
  const long long n = h.n1;
  const int k = h.nrhs, nb = reduce_blocks(n);
  PMG_CUDA(cudaMemsetAsync(h.dstatus, 0, (kCtrlSeg + 4 * k) * sizeof(int), s));
  // r = g - A u; from a zero initial guess (checked on the device, so that a captured
  // solve keeps the test) the apply kernel forms r = g without the apply
  PMG_CUDA(cudaMemsetAsync(h.duz, 0, sizeof(int), s));
  launch_any_nonzero(u, n * k, h.duz, s);
  outer_apply(h, u, g, h.r, s, h.duz);
  if (h.dims[h.L].periodic) launch_sub_mean(h.r, n, h.partial, h.counter, h.scal, nb, s);   // nrhs = 1
  launch_dot(h.r, h.r, nullptr, n, k, h.partial, h.counter, h.scal + S_RR0, nb, s);
  PMG_CUDA(cudaMemsetAsync(h.r_old, 0, (size_t)k * n * sizeof(double), s));
  launch_solve_begin(h.scal, h.dstatus, h.hist, h.opt.max_iter + 1, k, cond, s);
}

void cg_iteration(Hier& h, double* u, double rtol, const cudaGraphConditionalHandle* cond, bool direct,
                  cudaStream_t s) {
  const long long n = h.n1;
  const int k = h.nrhs, nb = reduce_blocks(n);
  const int* it_dev = h.dstatus + C_ITER;
  if (direct) precondition_graph(h, s);
  else precondition(h, h.r, h.z, s);
  launch_dot(h.z, h.r, h.r_old, n, k, h.partial, h.counter, h.scal + S_ZR, nb, s);
  launch_p_update(h.p, h.z, h.scal, 0, n, k, s, it_dev, h.dstatus);
  launch_set_delta(h.scal, h.dstatus, k, s);
  outer_apply(h, h.p, nullptr, h.q, s);
  launch_dot(h.p, h.q, nullptr, n, k, h.partial, h.counter, h.scal + S_PQ, nb, s);
  launch_cg_update(u, h.r, h.r_old, h.p, h.q, h.scal, 0, n, k, h.partial, h.counter, h.dstatus, nb, s,
                   it_dev);
  launch_solve_control(h.scal, h.dstatus, h.hist, h.opt.max_iter + 1, k, rtol, h.opt.max_iter, cond, s);
}

void cg_end(Hier& h, double* u, SolveResult* res, cudaStream_t s) {
  if (h.dims[h.L].periodic) launch_sub_mean(u, h.n1, h.partial, h.counter, h.scal, reduce_blocks(h.n1), s);
  launch_solve_result(h.scal, h.dstatus, res, h.nrhs, s);
}

// Appends one whole MGCG solve of h on (g, u) to `graph` as an independent branch:
// cg_begin, the iterations as a device-side `while` node, cg_end writing res.  The
// coarse solve is captured as separate launches, so branches of one graph may run
// concurrently.  Returns the kernel counts outside the loop and per iteration.
void capture_solve(Hier& h, cudaGraph_t graph, const double* g, double* u, double rtol,
                   SolveResult* res, unsigned long long* fixed, unsigned long long* per_iter) {
  if (!h.cap_stream) PMG_CUDA(cudaStreamCreateWithFlags(&h.cap_stream, cudaStreamNonBlocking));
  if (!h.cap_stream2) PMG_CUDA(cudaStreamCreateWithFlags(&h.cap_stream2, cudaStreamNonBlocking));
  cudaStream_t cs = h.cap_stream, cb = h.cap_stream2;
  cudaGraphConditionalHandle cond;
  PMG_CUDA(cudaGraphConditionalHandleCreate(&cond, graph, 0, cudaGraphCondAssignDefault));
  const unsigned long long c0 = g_launches.load();
  unsigned long long c1 = 0, c2 = 0;
  h.coarse_split = true;
  bool outer = false, inner = false;
  try {
    PMG_CUDA(cudaStreamBeginCaptureToGraph(cs, graph, nullptr, nullptr, 0,
                                           cudaStreamCaptureModeRelaxed));
    outer = true;
    cg_begin(h, g, u, &cond, cs);
    cudaStreamCaptureStatus cst;
    const cudaGraphNode_t* deps = nullptr;
    const cudaGraphEdgeData* edges = nullptr;
    size_t ndeps = 0;
    PMG_CUDA(cudaStreamGetCaptureInfo(cs, &cst, nullptr, nullptr, &deps, &edges, &ndeps));
    cudaGraphNodeParams cp = {};
    cp.type = cudaGraphNodeTypeConditional;
    cp.conditional.handle = cond;
    cp.conditional.type = cudaGraphCondTypeWhile;
    cp.conditional.size = 1;
    cudaGraphNode_t loop = nullptr;
    PMG_CUDA(cudaGraphAddNode(&loop, graph, deps, edges, ndeps, &cp));
    cudaGraph_t body = cp.conditional.phGraph_out[0];
    c1 = g_launches.load();
    PMG_CUDA(cudaStreamBeginCaptureToGraph(cb, body, nullptr, nullptr, 0,
                                           cudaStreamCaptureModeRelaxed));
    inner = true;
    cg_iteration(h, u, rtol, &cond, false, cb);
    cudaGraph_t body_out = nullptr;
    inner = false;
    PMG_CUDA(cudaStreamEndCapture(cb, &body_out));
    c2 = g_launches.load();
    PMG_CUDA(cudaStreamUpdateCaptureDependencies(cs, &loop, nullptr, 1,
                                                 cudaStreamSetCaptureDependencies));
    cg_end(h, u, res, cs);
    cudaGraph_t out = nullptr;
    outer = false;
    PMG_CUDA(cudaStreamEndCapture(cs, &out));
  } catch (...) {
    cudaGraph_t tmp = nullptr;
    if (inner) cudaStreamEndCapture(cb, &tmp);
    if (outer) cudaStreamEndCapture(cs, &tmp);
    cudaGetLastError();
    h.coarse_split = false;
    g_launches.store(c0);
    throw;
  }
  h.coarse_split = false;
  *per_iter = c2 - c1;
  *fixed = (g_launches.load() - c0) - *per_iter;
  g_launches.store(c0);                     // captured launches did not run
}

// Capture (or re-capture for new g, u, rtol) the single-solve graph of h.
void build_solve_graph(Hier& h, const double* g, double* u, double rtol) {
  if (h.sv_exec) cudaGraphExecDestroy(h.sv_exec);
  h.sv_exec = nullptr;
  h.sv_state = 0;
  cudaGraph_t graph = nullptr;
  try {
    PMG_CUDA(cudaGraphCreate(&graph, 0));
    capture_solve(h, graph, g, u, rtol, h.dres, &h.sv_fixed, &h.sv_iter);
    PMG_CUDA(cudaGraphInstantiate(&h.sv_exec, graph, 0));
    h.sv_state = 1;
    h.sv_g = g;
    h.sv_u = u;
    h.sv_rtol = rtol;
  } catch (const CudaError& e) {
    h.err = "device-resident solve unavailable, host-driven iterations used: " + e.msg;
    h.sv_exec = nullptr;
    h.sv_state = -1;
  }
  if (graph) cudaGraphDestroy(graph);
  cudaGetLastError();
}

void fill_stats(pmg_stats* st, const SolveResult& r, const double* hist, int device_loop, cudaStream_t s) {
  if (!st) return;
  st->iterations = r.iterations;
  st->r0 = r.r0;
  st->rn = r.rn;
  st->status = r.status;
  st->device_loop = device_loop;
  if (st->history) {
    PMG_CUDA(cudaMemcpyAsync(st->history, hist, sizeof(double) * (r.iterations + 1),
                             cudaMemcpyDeviceToHost, s));
    PMG_CUDA(cudaStreamSynchronize(s));
  }
}

// Statistics of the nrhs segments (st: nrhs entries, may be null); returns the status
// of the first segment that failed, else PMG_OK.
int report_results(Hier& h, const SolveResult* r, pmg_stats* st, int device_loop, cudaStream_t s) {
  int first = PMG_OK;
  for (int sg = 0; sg < h.nrhs; ++sg) {
    if (st) fill_stats(&st[sg], r[sg], h.hist + (size_t)sg * (h.opt.max_iter + 1), device_loop, s);
    if (first == PMG_OK && r[sg].status != PMG_OK) first = r[sg].status;
  }
  return first;
}

// Largest iteration count of a solve's segments (the number of loop iterations run).
int loop_iterations(const SolveResult* r, int k) {
  int m = 0;
  for (int sg = 0; sg < k; ++sg) m = r[sg].iterations > m ? r[sg].iterations : m;
  return m;
}

int solve_graph_run(Hier& h, pmg_stats* st, cudaStream_t s) {
  PMG_CUDA(cudaGraphLaunch(h.sv_exec, s));
  PMG_CUDA(cudaMemcpyAsync(h.hscal, h.dres, sizeof(SolveResult) * h.nrhs, cudaMemcpyDeviceToHost, s));
  PMG_CUDA(cudaStreamSynchronize(s));
  std::vector<SolveResult> r(h.nrhs);
  std::memcpy(r.data(), h.hscal, sizeof(SolveResult) * h.nrhs);
  g_launches.fetch_add(h.sv_fixed + (unsigned long long)loop_iterations(r.data(), h.nrhs) * h.sv_iter,
                       std::memory_order_relaxed);
  return report_results(h, r.data(), st, 1, s);
}

// ---------------------------------------------------------------------------
// Autotuner of the patch kernel's CTA size.  Every line pass strides over its
// lines by the CTA size, so any multiple of 32 up to kFdmMaxThreads computes
// the same result; the best size depends on the patch shape (shared memory
// per CTA, lines per pass) and on the number of patches.  Each family is timed
// on its own level with CUDA events; results are cached per shape for the
// process, so many hierarchies of one shape tune once.
// ---------------------------------------------------------------------------
std::mutex g_tune_mu;
std::map<std::array<int, 6>, int> g_tune_cache;

template <typename T>
int tune_family(Hier& h, int l, FdmFamily<T>& fam, LevelDev<T>& d, cudaStream_t s) {
  int lg = 0;
  while ((1 << (lg + 1)) <= fam.count_total) ++lg;
  const std::array<int, 6> key = {(int)sizeof(T), fam.ax[0].n, fam.ax[1].n, fam.ax[2].n, fam.tc, lg};
  {
    std::lock_guard<std::mutex> lock(g_tune_mu);
    auto it = g_tune_cache.find(key);
    if (it != g_tune_cache.end()) {
      fam.variant = it->second / 1000;
      return fam.threads = it->second % 1000;
    }
  }
  const LevelDims& dm = h.dims[l];
  PMG_CUDA(cudaMemsetAsync(d.f, 0, sizeof(T) * dm.ndof, s));
  PMG_CUDA(cudaMemsetAsync(d.u, 0, sizeof(T) * dm.ndof, s));
  static const int cand_simt[] = {64, 96, 128, 160, 192, 256, 320, 384, 448, 512};
  static const int cand_tc[] = {128, 256, 384, 512};  // tcgen05 kernel: whole warp quarters
  const bool tc5 = sizeof(T) == 4 && fam.tc == 2 && dm.dim == 3;
  const int* cand = tc5 ? cand_tc : cand_simt;
  const int ncand = tc5 ? 4 : 10;
  cudaEvent_t e0, e1;
  PMG_CUDA(cudaEventCreate(&e0));
  PMG_CUDA(cudaEventCreate(&e1));
  int best = 0, best_v = -1;
  float best_ms = 1e30f;
  // fp32 families: both kernel forms (one patch per CTA, pipelined persistent CTAs);
  // patches too large for shared memory (a scratch buffer attached): scratch or slab form
  const int nvar = (sizeof(T) == 4 && !fam.tc) || fam.scratch ? 2 : 1;
  try {
    for (int v = 0; v < nvar; ++v) {
      for (int ci = 0; ci < ncand; ++ci) {
        const int c = cand[ci];
        if (c > kFdmMaxThreads) continue;
        fam.threads = c;
        fam.variant = nvar == 2 ? v : -1;
        PMG_CHECK(launch_fdm<T>(dm, fam, d.f, d.u, s));            // warm-up
        PMG_CUDA(cudaEventRecord(e0, s));
        for (int rep = 0; rep < 3; ++rep) PMG_CHECK(launch_fdm<T>(dm, fam, d.f, d.u, s));
        PMG_CUDA(cudaEventRecord(e1, s));
        PMG_CUDA(cudaEventSynchronize(e1));
        float ms = 0.0f;
        PMG_CUDA(cudaEventElapsedTime(&ms, e0, e1));
        if (ms < best_ms) {
          best_ms = ms;
          best = c;
          best_v = fam.variant;
        }
      }
    }
  } catch (...) {
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    fam.threads = 0;
    fam.variant = -1;
    throw;
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  fam.threads = best;
  fam.variant = best_v;
  std::lock_guard<std::mutex> lock(g_tune_mu);
  g_tune_cache[key] = best + 1000 * (best_v < 0 ? 0 : best_v);
  return best;
}

template <typename T>
void tune_level(Hier& h, int l, LevelDev<T>& d, cudaStream_t s) {
  if (h.opt.smoother == PMG_SMOOTHER_EA) {
    tune_family<T>(h, l, d.ea, d, s);
  } else {
    for (int q = 0; q < h.dims[l].dim; ++q) tune_family<T>(h, l, d.fa[q], d, s);
  }
}

// Algorithm 2.  The first solve of a hierarchy runs its iterations from the
// host (one synchronisation per iteration; it also sets the kernels up); later
// solves replay the whole solve as one CUDA graph with a device-side loop.
int solve_host_loop(Hier& h, const double* g, double* u, double rtol, pmg_stats* st,
                    cudaStream_t s);

int solve_impl(Hier& h, const double* g, double* u, double rtol, pmg_stats* st, cudaStream_t s) {
  if (h.pc_calls >= 1 && h.sv_state >= 0) {
    if (h.sv_state == 0 || h.sv_g != g || h.sv_u != u || h.sv_rtol != rtol)
      build_solve_graph(h, g, u, rtol);
    if (h.sv_state == 1) return solve_graph_run(h, st, s);
  }
  return solve_host_loop(h, g, u, rtol, st, s);
}

int solve_host_loop(Hier& h, const double* g, double* u, double rtol, pmg_stats* st,
                    cudaStream_t s) {
  const int k = h.nrhs;
  int* ctrl = reinterpret_cast<int*>(h.hscal);
  auto read_ctrl = [&] {
    PMG_CUDA(cudaMemcpyAsync(ctrl, h.dstatus, (kCtrlSeg + 4 * k) * sizeof(int), cudaMemcpyDeviceToHost, s));
    PMG_CUDA(cudaStreamSynchronize(s));
  };
  cg_begin(h, g, u, nullptr, s);
  read_ctrl();
  for (int it = 1; it <= h.opt.max_iter && ctrl[C_ACTIVE] > 0; ++it) {
    cg_iteration(h, u, rtol, nullptr, true, s);
    read_ctrl();
  }
  cg_end(h, u, h.dres, s);
  PMG_CUDA(cudaMemcpyAsync(h.hscal, h.dres, sizeof(SolveResult) * k, cudaMemcpyDeviceToHost, s));
  PMG_CUDA(cudaStreamSynchronize(s));
  std::vector<SolveResult> r(k);
  std::memcpy(r.data(), h.hscal, sizeof(SolveResult) * k);
  PMG_CUDA(cudaGetLastError());
  return report_results(h, r.data(), st, 0, s);
}

// A batch of independent solves captured as one CUDA graph: one branch per
// (hierarchy, g, u), each with its own device-side iteration loop.
struct Batch {
  std::vector<Hier*> h;
  std::vector<const double*> g;
  std::vector<double*> u;
  double rtol = 0.0;
  cudaGraphExec_t exec = nullptr;
  SolveResult* dres = nullptr;     // device [total segments]
  SolveResult* hres = nullptr;     // pinned host [total segments]
  std::vector<int> off;            // first segment of solve i
  std::vector<unsigned long long> fixed, per_iter;
  std::vector<void*> owned;
  std::string err;
};

void free_batch(Batch* b) {
  if (b->exec) cudaGraphExecDestroy(b->exec);
  for (void* p : b->owned) cudaFree(p);
  if (b->hres) cudaFreeHost(b->hres);
  delete b;
}

Hier* H(pmg_hier h) { return reinterpret_cast<Hier*>(h); }
Grid* G(pmg_grid g) { return reinterpret_cast<Grid*>(g); }

template <typename F>
int guarded(Hier* h, F&& fn) {
  try {
    return fn();
  } catch (const CudaError& e) {
    if (h) h->err = e.msg;
    return e.code;
  } catch (const std::bad_alloc&) {
    if (h) h->err = "host allocation failed";
    return PMG_ENOMEM;
  } catch (const std::exception& e) {
    if (h) h->err = e.what();
    return PMG_EINVAL;
  }
}

void free_all(Hier* h) {
  for (int l = 0; l < kMaxLevels; ++l) {
    for (void* p : h->d64[l].owned) cudaFree(p);
    for (void* p : h->d32[l].owned) cudaFree(p);
  }
  for (void* p : h->owned) cudaFree(p);
  if (h->hscal) cudaFreeHost(h->hscal);
  if (h->pc_exec) cudaGraphExecDestroy(h->pc_exec);
  if (h->sv_exec) cudaGraphExecDestroy(h->sv_exec);
  if (h->cap_stream) cudaStreamDestroy(h->cap_stream);
  if (h->cap_stream2) cudaStreamDestroy(h->cap_stream2);
}

}  // namespace
}  // namespace pmg

using namespace pmg;

extern "C" {

void pmg_options_default(pmg_options* opt) {
  if (!opt) return;
  opt->smoother = PMG_SMOOTHER_EA;
  opt->overlap = PMG_OVERLAP_LEVEL;
  opt->weighting = PMG_WEIGHT_QUINTIC;
  opt->ns_pre = 1;
  opt->ns_post = 1;
  opt->variable_v = 0;
  opt->omega = 1.0;
  opt->precision = PMG_PREC_FP64;
  opt->max_iter = 100;
  for (int l = 0; l < 8; ++l) opt->omega_level[l] = opt->tau_level[l] = 0.0;
  opt->nrhs = 1;
  opt->preconditioner = PMG_PC_VCYCLE;
  opt->outer_apply = PMG_OUTER_FP64;
}

int pmg_grid_create(int dim, int P, const int n_elem[3], const double* const spacing[3],
                    int periodic, double mu_star, const double beta[3], pmg_grid* out) {
  if (!out || !n_elem || !spacing) return PMG_EINVAL;
  *out = nullptr;
  if (dim != 2 && dim != 3) return PMG_EINVAL;
  if (P < 1 || (P & (P - 1)) != 0 || P > 32) return PMG_EINVAL;
  if (!(mu_star > -1.0)) return PMG_EINVAL;
  try {
    Grid* g = new Grid();
    g->dim = dim;
    g->P = P;
    g->bc_periodic = periodic ? 1 : 0;
    g->mu_star = mu_star;
    for (int d = 0; d < 3; ++d) {
      g->ne[d] = d < dim ? n_elem[d] : 1;
      g->beta[d] = (beta && d < dim) ? beta[d] : 0.0;
      if (d >= dim) continue;
      if (g->ne[d] < (periodic ? 2 : 1) || !spacing[d]) { delete g; return PMG_EINVAL; }
      g->spacing[d].assign(spacing[d], spacing[d] + g->ne[d]);
      for (double w : g->spacing[d])
        if (!(w > 0.0) || !std::isfinite(w)) { delete g; return PMG_EINVAL; }
    }
    *out = reinterpret_cast<pmg_grid>(g);
    return PMG_OK;
  } catch (...) {
    return PMG_ENOMEM;
  }
}

void pmg_grid_destroy(pmg_grid g) { delete G(g); }

int pmg_grid_coords(pmg_grid g, int axis, double* out) {
  Grid* gr = G(g);
  if (!gr || !out || axis < 0 || axis >= gr->dim) return PMG_EINVAL;
  std::vector<double> eta, rho;
  gll_nodes(gr->P, eta, rho);
  double left = 0.0;
  for (int m = 0; m < gr->ne[axis]; ++m) {
    double w = gr->spacing[axis][m];
    for (int i = 0; i <= gr->P; ++i) out[m * (gr->P + 1) + i] = left + 0.5 * (eta[i] + 1.0) * w;
    left += w;
  }
  return PMG_OK;
}

int pmg_hierarchy_build(pmg_grid g, const pmg_options* opt, pmg_hier* out) {
  if (!g || !out) return PMG_EINVAL;
  *out = nullptr;
  Grid* gr = G(g);
  pmg_options o;
  if (opt) o = *opt; else pmg_options_default(&o);
  if (o.smoother != PMG_SMOOTHER_EA && o.smoother != PMG_SMOOTHER_FA) return PMG_EINVAL;
  if (o.overlap < 0 || o.overlap > 2) return PMG_EINVAL;
  if (o.weighting != 0 && o.weighting != 1 && o.weighting != 3 && o.weighting != 5) return PMG_EINVAL;
  if (o.ns_pre < 0 || o.ns_post < 0 || o.max_iter < 1 || !(o.omega > 0.0)) return PMG_EINVAL;
  for (int l = 0; l < 8; ++l)
    if (!(o.omega_level[l] >= 0.0) || !(o.tau_level[l] >= 0.0) || o.tau_level[l] > 1.0) return PMG_EINVAL;
  if (o.precision != PMG_PREC_FP64 && o.precision != PMG_PREC_MIXED && o.precision != PMG_PREC_MIXED_TC &&
      o.precision != PMG_PREC_MIXED_TF32)
    return PMG_EINVAL;
  if (o.preconditioner != PMG_PC_VCYCLE && o.preconditioner != PMG_PC_NONE) return PMG_EINVAL;
  if (o.outer_apply != PMG_OUTER_FP64 && o.outer_apply != PMG_OUTER_DF) return PMG_EINVAL;
  // several right-hand sides stack copies of the grid along its last axis, separated by walls
  if (o.nrhs < 1 || o.nrhs > kMaxRhs || (o.nrhs > 1 && gr->bc_periodic)) return PMG_EINVAL;
  Hier* h = nullptr;
  try {
    h = new Hier();
  } catch (...) {
    return PMG_ENOMEM;
  }
  h->grid = *gr;
  h->opt = o;
  const int k = o.nrhs;
  h->nrhs = k;
  int L = 0;
  while ((1 << L) < gr->P) ++L;
  h->L = L;
  int rc = guarded(h, [&]() -> int {
    int dev = 0;
    PMG_CUDA(cudaGetDevice(&dev));
    PMG_CUDA(cudaDeviceGetAttribute(&h->nsm, cudaDevAttrMultiProcessorCount, dev));
    const int dim = gr->dim;
    for (int l = 0; l <= L; ++l) {
      const int Pl = 1 << l;
      LevelDims& dm = h->dims[l];
      dm.dim = dim;
      dm.P = Pl;
      dm.NP = Pl + 1;
      dm.NPz = dim == 3 ? Pl + 1 : 1;
      dm.nelem = 1;
      for (int d = 0; d < 3; ++d) {
        dm.ne[d] = gr->ne[d];
        dm.nelem *= gr->ne[d];
      }
      // several right-hand sides: k copies of the grid stacked along its last axis
      // with walls between them, so every level vector holds the k vectors back to back
      dm.ne[dim - 1] *= k;
      dm.nelem *= k;
      dm.ndof = dm.nelem * dm.NP * dm.NP * dm.NPz;
      dm.periodic = gr->bc_periodic;
      h->axes[l].resize(dim);
      std::vector<Axis1DHost> single(dim);
      for (int d = 0; d < dim; ++d) {
        build_axis(single[d], Pl, gr->spacing[d], gr->bc_periodic != 0, gr->beta[d], gr->mu_star);
        if (k > 1 && d == dim - 1) stack_axis(single[d], k, h->axes[l][d]);
        else h->axes[l][d] = single[d];
      }
      h->No[l] = overlap_nodes(Pl, o.overlap);
      std::vector<AxisTables> ec(dim), fc(dim);
      if (l > 0) {
        for (int d = 0; d < dim; ++d) {
          ec_axis_tables(single[d], h->No[l], o.weighting, level_tau(o, l), ec[d]);
          if (o.smoother == PMG_SMOOTHER_FA) {
            fc_axis_tables(single[d], o.weighting, level_tau(o, l), fc[d]);
          }
          if (k > 1 && d == dim - 1) {
            AxisTables t;
            stack_tables(ec[d], k, 0, t);
            ec[d] = t;
            if (o.smoother == PMG_SMOOTHER_FA) {
              stack_tables(fc[d], k, 1, t);
              fc[d] = t;
            }
          }
        }
      }
      build_level_dev<double>(*h, l, h->d64[l], ec, fc);
      if (o.precision != PMG_PREC_FP64) build_level_dev<float>(*h, l, h->d32[l], ec, fc);
      for (auto& t : ec) { t.S.clear(); t.W.clear(); t.lam.clear(); }
      for (auto& t : fc) { t.S.clear(); t.W.clear(); t.lam.clear(); }
      h->ec_shape[l] = ec;
      h->fc_shape[l] = fc;
      if (l > 0) {
        std::vector<double> J;
        lagrange_matrix(h->axes[l - 1][0].eta, h->axes[l][0].eta, J);
        h->J64[l] = dev_upload<double>(h->owned, J);
        h->J32[l] = dev_upload<float>(h->owned, J);
        h->Jhost[l] = J;
      }
    }
    h->has32 = o.precision != PMG_PREC_FP64;
    if (o.outer_apply == PMG_OUTER_DF) h->at_df = build_apply_tables<dfloat>(*h, L, h->owned);
    // exact coarse solve tables (global 1-D eigen-pairs at P = 1)
    CoarseFdm& c = h->coarse;
    c.lam_max = 0.0;
    for (int d = 0; d < 3; ++d) {
      int dd = d < dim ? d : 0;
      std::vector<double> S, lam;
      global_axis_eig(h->axes[0][dd], S, lam);
      c.N[d] = (int)lam.size();
      c.S[d] = dev_upload<double>(h->owned, S);
      c.lam[d] = dev_upload<double>(h->owned, lam);
      for (double v : lam) c.lam_max = std::max(c.lam_max, std::fabs(v));
    }
    c.tmp[0] = dev_alloc<double>(h->owned, h->dims[0].ndof);
    c.tmp[1] = dev_alloc<double>(h->owned, h->dims[0].ndof);
    const long long n = h->dims[L].ndof;
    h->n1 = n / k;
    h->r = dev_alloc<double>(h->owned, n);
    h->r_old = dev_alloc<double>(h->owned, n);
    h->p = dev_alloc<double>(h->owned, n);
    h->q = dev_alloc<double>(h->owned, n);
    h->z = dev_alloc<double>(h->owned, n);
    h->scal = dev_alloc<double>(h->owned, (size_t)S_NUM * k);
    h->partial = dev_alloc<double>(h->owned, (size_t)kPartialStride * k);
    h->counter = dev_alloc<unsigned>(h->owned, k);
    h->dstatus = dev_alloc<int>(h->owned, kCtrlSeg + 4 * k);
    h->duz = dev_alloc<int>(h->owned, 1);
    h->hist = dev_alloc<double>(h->owned, (size_t)(o.max_iter + 1) * k);
    h->dres = dev_alloc<SolveResult>(h->owned, k);
    PMG_CUDA(cudaMemset(h->counter, 0, k * sizeof(unsigned)));
    PMG_CUDA(cudaMemset(h->dstatus, 0, (kCtrlSeg + 4 * k) * sizeof(int)));
    PMG_CUDA(cudaMemset(h->scal, 0, (size_t)S_NUM * k * sizeof(double)));
    PMG_CUDA(cudaMallocHost(&h->hscal, host_mirror_bytes(k)));
    // patch kernels that can detect a failed bounded wait report it in the hierarchy's
    // status word, which pmg_solve reads (and pmg_device_status for the other calls)
    for (int l = 1; l <= L; ++l) {
      h->d32[l].ea.status = h->dstatus;
      for (int q = 0; q < 3; ++q) h->d32[l].fa[q].status = h->dstatus;
    }
    PMG_CUDA(cudaDeviceSynchronize());
    return PMG_OK;
  });
  if (rc != PMG_OK) {
    std::fprintf(stderr, "pmg_hierarchy_build: %s\n", h->err.c_str());
    free_all(h);
    delete h;
    return rc;
  }
  *out = reinterpret_cast<pmg_hier>(h);
  return PMG_OK;
}

void pmg_hierarchy_destroy(pmg_hier hh) {
  Hier* h = H(hh);
  if (!h) return;
  cudaDeviceSynchronize();
  free_all(h);
  delete h;
}

int pmg_num_levels(pmg_hier hh) { return hh ? H(hh)->L + 1 : PMG_EINVAL; }

int pmg_level_info(pmg_hier hh, int level, int* P_l, long long* ndof) {
  Hier* h = H(hh);
  if (!h || level < 0 || level > h->L) return PMG_EINVAL;
  if (P_l) *P_l = h->dims[level].P;
  if (ndof) *ndof = h->dims[level].ndof;
  return PMG_OK;
}

int pmg_apply(pmg_hier hh, int level, const double* u, double* Au, void* stream) {
  Hier* h = H(hh);
  if (!h || level < 0 || level > h->L || !u || !Au) return PMG_EINVAL;
  return guarded(h, [&] {
    if (level == h->L) {
      outer_apply(*h, u, nullptr, Au, (cudaStream_t)stream);
      return (int)PMG_OK;
    }
    return launch_apply<double>(h->dims[level], h->d64[level].at, u, nullptr, Au, (cudaStream_t)stream);
  });
}

int pmg_residual(pmg_hier hh, int level, const double* u, const double* f, double* r, void* stream) {
  Hier* h = H(hh);
  if (!h || level < 0 || level > h->L || !u || !f || !r) return PMG_EINVAL;
  return guarded(h, [&] {
    if (level == h->L) {
      outer_apply(*h, u, f, r, (cudaStream_t)stream);
      return (int)PMG_OK;
    }
    return launch_apply<double>(h->dims[level], h->d64[level].at, u, f, r, (cudaStream_t)stream);
  });
}

int pmg_rhs(pmg_hier hh, const double* f, double* g, void* stream) {
  Hier* h = H(hh);
  if (!h || !f || !g) return PMG_EINVAL;
  return guarded(h, [&] {
    launch_mass(h->dims[h->L], h->d64[h->L].at, f, g, (cudaStream_t)stream);
    PMG_CUDA(cudaGetLastError());
    return PMG_OK;
  });
}

int pmg_smooth(pmg_hier hh, int level, double* u, const double* f, int nsteps, void* stream) {
  Hier* h = H(hh);
  if (!h || level < 1 || level > h->L || !u || !f || nsteps < 0) return PMG_EINVAL;
  return guarded(h, [&] {
    cudaStream_t s = (cudaStream_t)stream;
    if (h->opt.precision != PMG_PREC_FP64) {
      const long long n = h->dims[level].ndof;
      // level vectors of the V-cycle serve as fp32 staging buffers
      float* uf = h->d32[level].u;
      float* ff = h->d32[level].f;
      launch_convert<double, float>(u, uf, n, s);
      launch_convert<double, float>(f, ff, n, s);
      smooth_level<float>(*h, level, uf, ff, nsteps, false, s);
      launch_convert<float, double>(uf, u, n, s);
    } else {
      smooth_level<double>(*h, level, u, f, nsteps, false, s);
    }
    PMG_CUDA(cudaGetLastError());
    return PMG_OK;
  });
}

int pmg_restrict(pmg_hier hh, int level, const double* rf, double* fc, void* stream) {
  Hier* h = H(hh);
  if (!h || level < 1 || level > h->L || !rf || !fc) return PMG_EINVAL;
  return guarded(h, [&] {
    return launch_restrict<double>(h->dims[level], h->dims[level - 1], h->J64[level], h->Jhost[level].data(),
                                   rf, fc, (cudaStream_t)stream);
  });
}

int pmg_prolong(pmg_hier hh, int level, const double* uc, double* uf, void* stream) {
  Hier* h = H(hh);
  if (!h || level < 1 || level > h->L || !uc || !uf) return PMG_EINVAL;
  return guarded(h, [&] {
    return launch_prolong<double>(h->dims[level], h->dims[level - 1], h->J64[level], h->Jhost[level].data(),
                                  uc, uf, (cudaStream_t)stream);
  });
}

int pmg_coarse_solve(pmg_hier hh, const double* f0, double* u0, void* stream) {
  Hier* h = H(hh);
  if (!h || !f0 || !u0) return PMG_EINVAL;
  return guarded(h, [&] { return launch_coarse_fdm(h->dims[0], h->coarse, f0, u0, (cudaStream_t)stream); });
}

int pmg_vcycle(pmg_hier hh, const double* f, double* u, void* stream) {
  Hier* h = H(hh);
  if (!h || !f || !u) return PMG_EINVAL;
  return guarded(h, [&] {
    precondition(*h, f, u, (cudaStream_t)stream);
    PMG_CUDA(cudaGetLastError());
    return PMG_OK;
  });
}

int pmg_solve(pmg_hier hh, const double* g, double* u, double rtol, pmg_stats* st, void* stream) {
  Hier* h = H(hh);
  if (!h || !g || !u || !(rtol >= 0.0)) return PMG_EINVAL;
  return guarded(h, [&] { return solve_impl(*h, g, u, rtol, st, (cudaStream_t)stream); });
}

int pmg_solve_host(pmg_hier hh, const double* g_host, double* u_host, double rtol, pmg_stats* st,
                   void* stream) {
  Hier* h = H(hh);
  if (!h || !g_host || !u_host || !(rtol >= 0.0)) return PMG_EINVAL;
  return guarded(h, [&] {
    cudaStream_t s = (cudaStream_t)stream;
    const long long n = h->dims[h->L].ndof;
    if (!h->g_host_stage) {               // first call: device staging buffers
      h->g_host_stage = dev_alloc<double>(h->owned, n);
      h->u_host_stage = dev_alloc<double>(h->owned, n);
    }
    PMG_CUDA(cudaMemcpyAsync(h->g_host_stage, g_host, n * sizeof(double), cudaMemcpyHostToDevice, s));
    PMG_CUDA(cudaMemcpyAsync(h->u_host_stage, u_host, n * sizeof(double), cudaMemcpyHostToDevice, s));
    int rc = solve_impl(*h, h->g_host_stage, h->u_host_stage, rtol, st, s);
    PMG_CUDA(cudaMemcpyAsync(u_host, h->u_host_stage, n * sizeof(double), cudaMemcpyDeviceToHost, s));
    PMG_CUDA(cudaStreamSynchronize(s));
    return rc;
  });
}

int pmg_batch_create(int count, const pmg_hier* hiers, const double* const* g_dev,
                     double* const* u_dev, double rtol, pmg_batch* out) {
  if (!out) return PMG_EINVAL;
  *out = nullptr;
  if (count < 1 || !hiers || !g_dev || !u_dev || !(rtol >= 0.0)) return PMG_EINVAL;
  std::vector<Hier*> hs(count);
  for (int i = 0; i < count; ++i) {
    hs[i] = H(hiers[i]);
    if (!hs[i] || !g_dev[i] || !u_dev[i]) return PMG_EINVAL;
    for (int j = 0; j < i; ++j)
      if (hs[j] == hs[i]) return PMG_EINVAL;   // one workspace per concurrent solve
  }
  Batch* b = nullptr;
  try {
    b = new Batch();
  } catch (...) {
    return PMG_ENOMEM;
  }
  b->h = hs;
  b->g.assign(g_dev, g_dev + count);
  b->u.assign(u_dev, u_dev + count);
  b->rtol = rtol;
  b->fixed.assign(count, 0);
  b->per_iter.assign(count, 0);
  cudaGraph_t graph = nullptr;
  int rc = PMG_OK;
  try {
    // one direct V-cycle per hierarchy that has not run yet (kernel set-up)
    for (Hier* h : hs) {
      if (h->pc_calls >= 1) continue;
      PMG_CUDA(cudaMemsetAsync(h->r, 0, sizeof(double) * h->dims[h->L].ndof, 0));
      precondition_graph(*h, 0);
    }
    PMG_CUDA(cudaStreamSynchronize(0));
    int total = 0;
    for (Hier* h : hs) {
      b->off.push_back(total);
      total += h->nrhs;
    }
    b->dres = dev_alloc<SolveResult>(b->owned, total);
    PMG_CUDA(cudaMallocHost(&b->hres, sizeof(SolveResult) * total));
    PMG_CUDA(cudaGraphCreate(&graph, 0));
    for (int i = 0; i < count; ++i)
      capture_solve(*hs[i], graph, b->g[i], b->u[i], rtol, b->dres + b->off[i], &b->fixed[i],
                    &b->per_iter[i]);
    PMG_CUDA(cudaGraphInstantiate(&b->exec, graph, 0));
  } catch (const CudaError& e) {
    b->err = e.msg;
    rc = e.code;
  } catch (const std::bad_alloc&) {
    rc = PMG_ENOMEM;
  }
  if (graph) cudaGraphDestroy(graph);
  if (rc != PMG_OK) {
    std::fprintf(stderr, "pmg_batch_create: %s\n", b->err.c_str());
    cudaGetLastError();
    free_batch(b);
    return rc;
  }
  *out = reinterpret_cast<pmg_batch>(b);
  return PMG_OK;
}

int pmg_batch_solve(pmg_batch bb, pmg_stats* stats, void* stream) {
  Batch* b = reinterpret_cast<Batch*>(bb);
  if (!b) return PMG_EINVAL;
  cudaStream_t s = (cudaStream_t)stream;
  const int count = (int)b->h.size();
  const int total = b->off[count - 1] + b->h[count - 1]->nrhs;
  int first_bad = PMG_OK;
  try {
    PMG_CUDA(cudaGraphLaunch(b->exec, s));
    PMG_CUDA(cudaMemcpyAsync(b->hres, b->dres, sizeof(SolveResult) * total,
                             cudaMemcpyDeviceToHost, s));
    PMG_CUDA(cudaStreamSynchronize(s));
    for (int i = 0; i < count; ++i) {
      const SolveResult* r = b->hres + b->off[i];
      g_launches.fetch_add(b->fixed[i] + (unsigned long long)loop_iterations(r, b->h[i]->nrhs) * b->per_iter[i],
                           std::memory_order_relaxed);
      const int st = report_results(*b->h[i], r, stats ? stats + b->off[i] : nullptr, 1, s);
      if (first_bad == PMG_OK && st != PMG_OK) first_bad = st;
    }
  } catch (const CudaError& e) {
    b->err = e.msg;
    return e.code;
  }
  return first_bad;
}

void pmg_batch_destroy(pmg_batch bb) {
  Batch* b = reinterpret_cast<Batch*>(bb);
  if (!b) return;
  cudaDeviceSynchronize();
  free_batch(b);
}

const char* pmg_batch_last_error(pmg_batch bb) {
  return bb ? reinterpret_cast<Batch*>(bb)->err.c_str() : "";
}

int pmg_hierarchy_autotune(pmg_hier hh, void* stream) {
  Hier* h = H(hh);
  if (!h) return PMG_EINVAL;
  return guarded(h, [&] {
    cudaStream_t s = (cudaStream_t)stream;
    for (int l = 1; l <= h->L; ++l) {
      if (h->opt.precision == PMG_PREC_FP64) tune_level<double>(*h, l, h->d64[l], s);
      else tune_level<float>(*h, l, h->d32[l], s);
    }
    // captured graphs hold the old launch shapes: capture again on next use
    if (h->sv_exec) cudaGraphExecDestroy(h->sv_exec);
    h->sv_exec = nullptr;
    if (h->sv_state == 1) h->sv_state = 0;
    if (h->pc_exec) cudaGraphExecDestroy(h->pc_exec);
    h->pc_exec = nullptr;
    if (h->pc_state == 1) h->pc_state = 0;
    return (int)PMG_OK;
  });
}

int pmg_tuned_threads(pmg_hier hh, int level, int family) {
  Hier* h = H(hh);
  if (!h || level < 1 || level > h->L) return PMG_EINVAL;
  const bool ea = h->opt.smoother == PMG_SMOOTHER_EA;
  if (ea ? family != -1 : (family < 0 || family >= h->dims[level].dim)) return PMG_EINVAL;
  if (h->opt.precision == PMG_PREC_FP64) {
    const FdmFamily<double>& f = ea ? h->d64[level].ea : h->d64[level].fa[family];
    return f.threads;
  }
  const FdmFamily<float>& f = ea ? h->d32[level].ea : h->d32[level].fa[family];
  return f.threads;
}

const char* pmg_status_string(int status) {
  switch (status) {
    case PMG_OK: return "ok";
    case PMG_EINVAL: return "invalid argument or unsupported configuration";
    case PMG_ENOMEM: return "out of memory";
    case PMG_ECUDA: return "CUDA error";
    case PMG_ENOCONV: return "no convergence within max_iter";
    case PMG_EBREAKDOWN: return "CG breakdown (p^T A p <= 0 or delta <= 0)";
    case PMG_ENAN: return "non-finite residual";
    case PMG_ETIMEOUT: return "device wait timed out";
    default: return "unknown status";
  }
}

const char* pmg_last_error(pmg_hier hh) { return hh ? H(hh)->err.c_str() : ""; }

unsigned long long pmg_kernel_launches(void) { return g_launches.load(); }

int pmg_tc_timeouts(unsigned int* count) {
  if (!count) return PMG_EINVAL;
  return tc_timeouts_take(count);
}

int pmg_device_status(pmg_hier hh, void* stream, int* status) {
  Hier* h = H(hh);
  if (!h || !status) return PMG_EINVAL;
  return guarded(h, [&] {
    cudaStream_t s = (cudaStream_t)stream;
    int v = 0;
    PMG_CUDA(cudaMemcpyAsync(h->hscal, h->dstatus + C_STATUS, sizeof(int), cudaMemcpyDeviceToHost, s));
    PMG_CUDA(cudaStreamSynchronize(s));
    std::memcpy(&v, h->hscal, sizeof(int));
    PMG_CUDA(cudaMemsetAsync(h->dstatus + C_STATUS, 0, sizeof(int), s));
    PMG_CUDA(cudaStreamSynchronize(s));
    *status = v;
    return (int)PMG_OK;
  });
}

int pmg_test_stall_tc_waits(pmg_hier hh, unsigned int limit_us) {
  Hier* h = H(hh);
  if (!h || limit_us > 1000000u) return PMG_EINVAL;
  const unsigned int ns = limit_us * 1000u;
  for (int l = 1; l <= h->L; ++l) {
    h->d32[l].ea.stall_ns = ns;
    for (int q = 0; q < 3; ++q) h->d32[l].fa[q].stall_ns = ns;
  }
  // captured graphs hold the old kernel parameters: capture again on next use
  return guarded(h, [&] {
    PMG_CUDA(cudaDeviceSynchronize());
    if (h->sv_exec) cudaGraphExecDestroy(h->sv_exec);
    h->sv_exec = nullptr;
    if (h->sv_state == 1) h->sv_state = 0;
    if (h->pc_exec) cudaGraphExecDestroy(h->pc_exec);
    h->pc_exec = nullptr;
    if (h->pc_state == 1) h->pc_state = 0;
    return (int)PMG_OK;
  });
}

int pmg_schwarz_sweep_native(pmg_hier hh, int level, int family, void* stream) {
  Hier* h = H(hh);
  if (!h || level < 1 || level > h->L) return PMG_EINVAL;
  const LevelDims& dm = h->dims[level];
  const bool ea = h->opt.smoother == PMG_SMOOTHER_EA;
  if (ea ? family != -1 : (family < 0 || family >= dm.dim)) return PMG_EINVAL;
  return guarded(h, [&] {
    cudaStream_t s = (cudaStream_t)stream;
    if (h->opt.precision != PMG_PREC_FP64) {
      LevelDev<float>& d = h->d32[level];
      PMG_CHECK(launch_fdm<float>(dm, ea ? d.ea : d.fa[family], d.f, d.u, s));
    } else {
      LevelDev<double>& d = h->d64[level];
      PMG_CHECK(launch_fdm<double>(dm, ea ? d.ea : d.fa[family], d.f, d.u, s));
    }
    PMG_CUDA(cudaGetLastError());
    return PMG_OK;
  });
}

int pmg_schwarz_sweep_fma(pmg_hier hh, int level, int family, double* fma) {
  Hier* h = H(hh);
  if (!h || !fma || level < 1 || level > h->L) return PMG_EINVAL;
  const LevelDims& dm = h->dims[level];
  const bool ea = h->opt.smoother == PMG_SMOOTHER_EA;
  if (ea ? family != -1 : (family < 0 || family >= dm.dim)) return PMG_EINVAL;
  // patch-buffer axes of the family, in kernel order
  const AxisTables* ax[3] = {nullptr, nullptr, nullptr};
  if (ea) {
    for (int q = 0; q < dm.dim; ++q) ax[q] = &h->ec_shape[level][q];
  } else {
    ax[0] = &h->fc_shape[level][family];
    int q = 1;
    for (int d = 0; d < dm.dim; ++d)
      if (d != family) ax[q++] = &h->ec_shape[level][d];
  }
  const int nd = dm.dim;
  // per axis: sum over positions of the multiply-adds of one line pass (even-odd: NE^2 + NO^2)
  double per_axis[3] = {0, 0, 0}, count[3] = {1, 1, 1}, n[3] = {1, 1, 1};
  for (int q = 0; q < nd; ++q) {
    const int nn = ax[q]->n, H = nn / 2, NE = nn - H;
    n[q] = nn;
    count[q] = ax[q]->count;
    for (int p = 0; p < ax[q]->count; ++p) per_axis[q] += ax[q]->sym[p] ? double(NE * NE + H * H) : double(nn * nn);
  }
  double total = 0.0;
  for (int q = 0; q < nd; ++q) {
    double lines = 1.0, others = 1.0;     // lines of a patch along q, and patch count of the other axes
    for (int r = 0; r < nd; ++r)
      if (r != q) {
        lines *= n[r];
        others *= count[r];
      }
    total += 2.0 * lines * others * per_axis[q];        // forward + backward pass
  }
  *fma = total;
  return PMG_OK;
}

int pmg_schwarz_sweep(pmg_hier hh, int level, int family, const double* r, double* u, void* stream) {
  Hier* h = H(hh);
  if (!h || level < 1 || level > h->L || !r || !u) return PMG_EINVAL;
  const LevelDims& dm = h->dims[level];
  const bool ea = h->opt.smoother == PMG_SMOOTHER_EA;
  if (ea ? family != -1 : (family < 0 || family >= dm.dim)) return PMG_EINVAL;
  return guarded(h, [&] {
    cudaStream_t s = (cudaStream_t)stream;
    if (h->opt.precision != PMG_PREC_FP64) {
      LevelDev<float>& d = h->d32[level];
      launch_convert<double, float>(r, d.r, dm.ndof, s);
      launch_convert<double, float>(u, d.u, dm.ndof, s);
      PMG_CHECK(launch_fdm<float>(dm, ea ? d.ea : d.fa[family], d.r, d.u, s));
      launch_convert<float, double>(d.u, u, dm.ndof, s);
    } else {
      LevelDev<double>& d = h->d64[level];
      PMG_CHECK(launch_fdm<double>(dm, ea ? d.ea : d.fa[family], r, u, s));
    }
    PMG_CUDA(cudaGetLastError());
    return PMG_OK;
  });
}

}  // extern "C"
