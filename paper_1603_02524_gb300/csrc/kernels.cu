// CUDA kernels of the p-multigrid DG Poisson solver (sm_103a): operator apply,
// mass, restriction / prolongation, exact coarse solve, CG vector kernels.
// The Schwarz patch kernel lives in fdm_kernel.cuh.
//
// Paper: Stiller, arXiv 1603.02524 (Sec. 2.4 operator, Sec. 3.2 transfers,
// Algorithm 2 vector steps).
#include <cstdio>

#include <cooperative_groups.h>

#include "apply_kernel.cuh"

namespace pmg {

template <typename T>
int launch_apply(const LevelDims& dm, const ApplyTables<T>& at, const T* u, const T* f, T* v,
                 cudaStream_t s, const int* unz) {
  if (dm.nelem == 0) return PMG_OK;
#define PMG_APPLY_CASE(DIMV, NPV) \
  if (dm.dim == DIMV && dm.NP == NPV) return apply_dispatch<T, DIMV, NPV>(dm, at, u, f, v, s, unz);
  PMG_APPLY_CASE(3, 2) PMG_APPLY_CASE(3, 3) PMG_APPLY_CASE(3, 5) PMG_APPLY_CASE(3, 9)
  PMG_APPLY_CASE(3, 17)
  if (dm.dim == 3 && dm.NP == 33) return apply_dispatch_axes<T, 33, T>(dm, at, u, f, v, s, unz);
  PMG_APPLY_CASE(2, 2) PMG_APPLY_CASE(2, 3) PMG_APPLY_CASE(2, 5) PMG_APPLY_CASE(2, 9)
  PMG_APPLY_CASE(2, 17) PMG_APPLY_CASE(2, 33)
#undef PMG_APPLY_CASE
  return PMG_EINVAL;
}
// fc = I^T (f - A u) in one kernel (the residual is not stored); PMG_EINVAL for
// shapes without the fused kernel (3-D P = 32), where the caller runs the two.
template <typename T>
int launch_residual_restrict(const LevelDims& dm, const ApplyTables<T>& at, const T* u, const T* f,
                             const T* /*J*/, const double* Jh, T* fc, cudaStream_t s) {
  if (dm.nelem == 0) return PMG_OK;
  if (!Jh) return PMG_EINVAL;
#define PMG_RR_CASE(DIMV, NPV, NPCV) \
  if (dm.dim == DIMV && dm.NP == NPV) return residual_restrict_dispatch<T, DIMV, NPV, NPCV>(dm, at, u, f, Jh, fc, s);
  PMG_RR_CASE(3, 3, 2) PMG_RR_CASE(3, 5, 3) PMG_RR_CASE(3, 9, 5) PMG_RR_CASE(3, 17, 9)
  PMG_RR_CASE(2, 3, 2) PMG_RR_CASE(2, 5, 3) PMG_RR_CASE(2, 9, 5) PMG_RR_CASE(2, 17, 9) PMG_RR_CASE(2, 33, 17)
#undef PMG_RR_CASE
  return PMG_EINVAL;
}
template int launch_residual_restrict<double>(const LevelDims&, const ApplyTables<double>&, const double*,
                                              const double*, const double*, const double*, double*,
                                              cudaStream_t);
template int launch_residual_restrict<float>(const LevelDims&, const ApplyTables<float>&, const float*,
                                             const float*, const float*, const double*, float*, cudaStream_t);

template int launch_apply<double>(const LevelDims&, const ApplyTables<double>&, const double*,
                                  const double*, double*, cudaStream_t, const int*);
template int launch_apply<float>(const LevelDims&, const ApplyTables<float>&, const float*,
                                 const float*, float*, cudaStream_t, const int*);

// *flag = 1 if some x[i] != 0 (a NaN counts as nonzero); the caller zeroes the flag
__global__ void __launch_bounds__(256) any_nonzero_kernel(const double* __restrict__ x, long long n, int* flag) {
  bool nz = false;
  for (long long i = blockIdx.x * 256LL + threadIdx.x; i < n; i += (long long)gridDim.x * 256) nz |= !(x[i] == 0.0);
  if (__syncthreads_or(nz) && threadIdx.x == 0) *flag = 1;
}
void launch_any_nonzero(const double* x, long long n, int* flag, cudaStream_t s) {
  if (n <= 0) return;
  long long blocks = (n + 255) / 256;
  if (blocks > 4096) blocks = 4096;
  count_launch();
  any_nonzero_kernel<<<(unsigned)blocks, 256, 0, s>>>(x, n, flag);
}

// ---------------------------------------------------------------------------
// g = M f: diagonal GLL mass (Sec. 2.4 right-hand side)
// ---------------------------------------------------------------------------
__global__ void mass_kernel(LevelDims dm, ApplyTables<double> at, const double* __restrict__ f,
                            double* __restrict__ g) {
  const int NP = dm.NP;
  const long long nodes = (dm.dim == 3) ? (long long)NP * NP * NP : (long long)NP * NP;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < dm.ndof;
       t += (long long)gridDim.x * blockDim.x) {
    long long e = t / nodes;
    int n = (int)(t % nodes);
    int i = n % NP, j = (n / NP) % NP, k = n / (NP * NP);
    int mx = (int)(e % dm.ne[0]), my = (int)((e / dm.ne[0]) % dm.ne[1]);
    int mz = (int)(e / ((long long)dm.ne[0] * dm.ne[1]));
    double s = at.M[0][(size_t)mx * NP + i] * at.M[1][(size_t)my * NP + j];
    if (dm.dim == 3) s *= at.M[2][(size_t)mz * NP + k];
    g[t] = s * f[t];
  }
}

void launch_mass(const LevelDims& dm, const ApplyTables<double>& at, const double* f, double* g,
                 cudaStream_t s) {
  long long blocks = (dm.ndof + 255) / 256;
  if (blocks > 65535 * 8) blocks = 65535 * 8;
  count_launch(); mass_kernel<<<(unsigned)blocks, 256, 0, s>>>(dm, at, f, g);
}

// ---------------------------------------------------------------------------
// Transfers (Sec. 3.2): prolongation u_f += (J (x) J (x) J) u_c, restriction
// f_c = (J (x) J (x) J)^T r_f, element by element, with J even-odd folded (FoldedJ
// in apply_kernel.cuh).  One CTA per element; three passes through shared memory,
// one thread per line of a pass.
// ---------------------------------------------------------------------------
template <typename T, int DIM, int NPF, int NPC, bool PROLONG>
__global__ void __launch_bounds__(256)
transfer_kernel(long long nelem, FoldedJ<T, NPF, NPC> J, const T* __restrict__ in, T* __restrict__ out) {
  constexpr int NIN = PROLONG ? NPC : NPF;      // per-axis size of the input
  constexpr int NOUT = PROLONG ? NPF : NPC;
  constexpr int NZI = (DIM == 3) ? NIN : 1;
  constexpr int NZO = (DIM == 3) ? NOUT : 1;
  extern __shared__ __align__(16) unsigned char tr_smem[];
  T* b0 = reinterpret_cast<T*>(tr_smem);
  T* b1 = b0 + NIN * NIN * NZI;
  T* b2 = b1 + NOUT * NIN * NZI;
  const long long e = blockIdx.x;
  // FP64: the coefficients from a shared-memory copy (as constant operands the
  // compiler keeps all of them in registers, 130 per thread, one CTA per SM)
  __shared__ FoldedJ<T, NPF, NPC> sJ;
  if constexpr (sizeof(T) == 8) {
    if (threadIdx.x == 0) sJ = J;
  }
  for (int t = threadIdx.x; t < NIN * NIN * NZI; t += blockDim.x)
    b0[t] = in[e * (NIN * NIN * NZI) + t];
  __syncthreads();
  // one axis line: NIN inputs `sstride` apart -> NOUT outputs (even-odd folded J),
  // each handed to put(index, value)
  auto line = [&](const T* src, int sstride, auto&& put) {
    T x[NIN];
#pragma unroll
    for (int a = 0; a < NIN; ++a) x[a] = src[a * sstride];
    const FoldedJ<T, NPF, NPC>* jp = &J;
    if constexpr (sizeof(T) == 8) {
      jp = &sJ;
      asm volatile("" : "+l"(jp));             // opaque per line: loaded as used, not hoisted
    }
    if constexpr (PROLONG) fold_prolong<T, NPF, NPC>(*jp, x, put);
    else fold_restrict<T, NPF, NPC>(*jp, x, put);
  };
#pragma unroll 1
  for (int r = threadIdx.x; r < NIN * NZI; r += blockDim.x) {          // x: lines (y, z)
    T* dst = b1 + r * NOUT;
    line(b0 + r * NIN, 1, [&](int o, T v) { dst[o] = v; });
  }
  __syncthreads();
#pragma unroll 1
  for (int t = threadIdx.x; t < NOUT * NZI; t += blockDim.x) {         // y: lines (x', z)
    const int i = t % NOUT, c = t / NOUT;
    if (DIM == 2) {
      T* dst = out + e * (NOUT * NOUT) + i;
      line(b1 + c * NIN * NOUT + i, NOUT, [&](int o, T v) {
        if (PROLONG) dst[o * NOUT] += v;
        else dst[o * NOUT] = v;
      });
    } else {
      T* dst = b2 + c * NOUT * NOUT + i;
      line(b1 + c * NIN * NOUT + i, NOUT, [&](int o, T v) { dst[o * NOUT] = v; });
    }
  }
  if (DIM == 2) return;
  __syncthreads();
#pragma unroll 1
  for (int ij = threadIdx.x; ij < NOUT * NOUT; ij += blockDim.x) {     // z: lines (x', y')
    T* dst = out + e * (NOUT * NOUT * NZO) + ij;
    line(b2 + ij, NOUT * NOUT, [&](int o, T v) {
      if (PROLONG) dst[o * NOUT * NOUT] += v;
      else dst[o * NOUT * NOUT] = v;
    });
  }
}

// 3-D transfers between P = 32 and P = 16 (33 and 17 nodes per axis): the
// three element-sized buffers of transfer_kernel do not fit shared memory, so the
// passes share one buffer of 17 x 33 x 33 entries: the first pass reads global
// memory, the middle pass works in place line by line (a thread holds its whole
// line in registers before it writes it), the last pass writes global memory.
template <typename T, bool PROLONG>
__global__ void __launch_bounds__(256)
transfer_big_kernel(long long nelem, const T* __restrict__ J, const T* __restrict__ in,
                    T* __restrict__ out) {
  constexpr int F = 33, C = 17;
  extern __shared__ __align__(16) unsigned char trb_smem[];
  T* sJ = reinterpret_cast<T*>(trb_smem);          // J[f][c]
  T* b = sJ + F * C;                                // [C][F][F]
  const long long e = blockIdx.x;
  for (int t = threadIdx.x; t < F * C; t += blockDim.x) sJ[t] = J[t];
  __syncthreads();
  if (!PROLONG) {
    const T* ie = in + e * (F * F * F);
    for (int t = threadIdx.x; t < C * F * F; t += blockDim.x) {   // z: F -> C
      const int oz = t / (F * F), rem = t - oz * F * F;
      T s = T(0);
#pragma unroll 1
      for (int k = 0; k < F; ++k) s = fma(sJ[k * C + oz], ie[k * F * F + rem], s);
      b[t] = s;
    }
    __syncthreads();
    for (int l = threadIdx.x; l < C * F; l += blockDim.x) {       // y: F -> C, in place
      const int oz = l / F, i = l - oz * F;
      T v[F];
#pragma unroll
      for (int j = 0; j < F; ++j) v[j] = b[(oz * F + j) * F + i];
#pragma unroll
      for (int oj = 0; oj < C; ++oj) {
        T s = T(0);
#pragma unroll
        for (int j = 0; j < F; ++j) s = fma(sJ[j * C + oj], v[j], s);
        b[(oz * F + oj) * F + i] = s;
      }
    }
    __syncthreads();
    for (int t = threadIdx.x; t < C * C * C; t += blockDim.x) {   // x: F -> C, to global
      const int ox = t % C, oj = (t / C) % C, oz = t / (C * C);
      const T* row = b + (oz * F + oj) * F;
      T s = T(0);
#pragma unroll
      for (int i = 0; i < F; ++i) s = fma(sJ[i * C + ox], row[i], s);
      out[e * (C * C * C) + t] = s;
    }
  } else {
    const T* ie = in + e * (C * C * C);
    for (int t = threadIdx.x; t < C * C * F; t += blockDim.x) {   // x: C -> F
      const int xo = t % F, jc = (t / F) % C, kc = t / (F * C);
      const T* row = ie + (kc * C + jc) * C;
      T s = T(0);
#pragma unroll
      for (int ic = 0; ic < C; ++ic) s = fma(sJ[xo * C + ic], row[ic], s);
      b[(kc * F + jc) * F + xo] = s;
    }
    __syncthreads();
    for (int l = threadIdx.x; l < C * F; l += blockDim.x) {       // y: C -> F, in place
      const int kc = l / F, xo = l - kc * F;
      T v[C];
#pragma unroll
      for (int jc = 0; jc < C; ++jc) v[jc] = b[(kc * F + jc) * F + xo];
#pragma unroll
      for (int yo = 0; yo < F; ++yo) {
        T s = T(0);
#pragma unroll
        for (int jc = 0; jc < C; ++jc) s = fma(sJ[yo * C + jc], v[jc], s);
        b[(kc * F + yo) * F + xo] = s;
      }
    }
    __syncthreads();
    for (int t = threadIdx.x; t < F * F * F; t += blockDim.x) {   // z: C -> F, add to global
      const int xy = t % (F * F), zo = t / (F * F);
      T s = T(0);
#pragma unroll
      for (int kc = 0; kc < C; ++kc) s = fma(sJ[zo * C + kc], b[kc * F * F + xy], s);
      out[e * (F * F * F) + t] += s;
    }
  }
}

template <typename T, bool PROLONG>
static int transfer_launch(const LevelDims& fine, const LevelDims& coarse, const T* J, const double* Jh,
                           const T* in, T* out, cudaStream_t s) {
  if (fine.nelem == 0) return PMG_OK;
  unsigned blocks = (unsigned)fine.nelem;
#define PMG_TR_CASE(DIMV, NPF, NPC) \
  if (fine.dim == DIMV && fine.NP == NPF && coarse.NP == NPC) { \
    if (!Jh) return PMG_EINVAL; \
    constexpr int NIN = PROLONG ? NPC : NPF, NOUT = PROLONG ? NPF : NPC; \
    constexpr int NZI = DIMV == 3 ? NIN : 1; \
    const size_t smem = sizeof(T) * (NIN * NIN * NZI + NOUT * NIN * NZI + NOUT * NOUT * NZI); \
    if (!set_smem(transfer_kernel<T, DIMV, NPF, NPC, PROLONG>, smem)) return PMG_ECUDA; \
    count_launch(); \
    transfer_kernel<T, DIMV, NPF, NPC, PROLONG><<<blocks, 256, smem, s>>>( \
        fine.nelem, fold_interpolation<T, NPF, NPC>(Jh), in, out); \
    return cudaGetLastError() == cudaSuccess ? PMG_OK : PMG_ECUDA; }
  PMG_TR_CASE(3, 3, 2) PMG_TR_CASE(3, 5, 3) PMG_TR_CASE(3, 9, 5) PMG_TR_CASE(3, 17, 9)
  PMG_TR_CASE(2, 3, 2) PMG_TR_CASE(2, 5, 3) PMG_TR_CASE(2, 9, 5) PMG_TR_CASE(2, 17, 9)
  PMG_TR_CASE(2, 33, 17)
#undef PMG_TR_CASE
  if (fine.dim == 3 && fine.NP == 33 && coarse.NP == 17) {
    const size_t smem = sizeof(T) * (33 * 17 + 17 * 33 * 33);
    if (!set_smem(transfer_big_kernel<T, PROLONG>, smem)) return PMG_ECUDA;
    count_launch(); transfer_big_kernel<T, PROLONG><<<blocks, 256, smem, s>>>(fine.nelem, J, in, out);
    return cudaGetLastError() == cudaSuccess ? PMG_OK : PMG_ECUDA;
  }
  return PMG_EINVAL;
}

template <typename T>
int launch_restrict(const LevelDims& fine, const LevelDims& coarse, const T* J, const double* Jh,
                    const T* rf, T* fc, cudaStream_t s) {
  return transfer_launch<T, false>(fine, coarse, J, Jh, rf, fc, s);
}
template <typename T>
int launch_prolong(const LevelDims& fine, const LevelDims& coarse, const T* J, const double* Jh,
                   const T* uc, T* uf, cudaStream_t s) {
  return transfer_launch<T, true>(fine, coarse, J, Jh, uc, uf, s);
}
template int launch_restrict<double>(const LevelDims&, const LevelDims&, const double*, const double*,
                                     const double*, double*, cudaStream_t);
template int launch_restrict<float>(const LevelDims&, const LevelDims&, const float*, const double*,
                                    const float*, float*, cudaStream_t);
template int launch_prolong<double>(const LevelDims&, const LevelDims&, const double*, const double*,
                                    const double*, double*, cudaStream_t);
template int launch_prolong<float>(const LevelDims&, const LevelDims&, const float*, const double*,
                                   const float*, float*, cudaStream_t);

// ---------------------------------------------------------------------------
// Exact coarse solve at P = 1 (A_0^+ f_0): the coarse operator is
// M3(x)M2(x)L1 + M3(x)L2(x)M1 + L3(x)M2(x)M1 with global 1-D factors, so
// A_0^{-1} = (S3(x)S2(x)S1) (sum Lambda)^{-1} (S3(x)S2(x)S1)^T  -- the fast
// diagonalisation of Sec. 3.1 applied to the whole coarse grid.  The zero mode
// of a periodic grid (all three lambda = 0) is dropped (pseudo-inverse).
// ---------------------------------------------------------------------------
__device__ __forceinline__ long long coarse_off(const LevelDims& dm, int X, int Y, int Z) {
  int ex = X >> 1, i = X & 1, ey = Y >> 1, j = Y & 1;
  if (dm.dim == 2) return ((long long)ey * dm.ne[0] + ex) * 4 + j * 2 + i;
  int ez = Z >> 1, k = Z & 1;
  return (((long long)ez * dm.ne[1] + ey) * dm.ne[0] + ex) * 8 + (k * 2 + j) * 2 + i;
}

// One axis transform of the coarse solve, grid-stride over all outputs.
__device__ __forceinline__ void coarse_axis_pass(const LevelDims& dm, int axis, bool transpose,
                                                 const double* __restrict__ S, int N,
                                                 const double* in, double* out) {
  const int NX = dm.ne[0] * 2, NY = dm.ne[1] * 2, NZ = (dm.dim == 3) ? dm.ne[2] * 2 : 1;
  const long long total = (long long)NX * NY * NZ;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < total;
       t += (long long)gridDim.x * blockDim.x) {
    const int X = (int)(t % NX), Y = (int)((t / NX) % NY), Z = (int)(t / ((long long)NX * NY));
    const int o = axis == 0 ? X : (axis == 1 ? Y : Z);
    double s = 0.0;
#pragma unroll 8
    for (int a = 0; a < N; ++a) {
      const int XX = axis == 0 ? a : X, YY = axis == 1 ? a : Y, ZZ = axis == 2 ? a : Z;
      const double m = transpose ? S[(size_t)a * N + o] : S[(size_t)o * N + a];
      s = fma(m, in[coarse_off(dm, XX, YY, ZZ)], s);
    }
    out[coarse_off(dm, X, Y, Z)] = s;
  }
}

// The whole coarse solve in one cooperative launch: forward transforms along
// each axis, scale by the eigenvalue sums, backward transforms; grid-wide
// synchronisation between the passes replaces seven separate launches.
__global__ void __launch_bounds__(256)
coarse_fdm_fused_kernel(LevelDims dm, CoarseFdm c, const double* f, double* u, double tol) {
  cooperative_groups::grid_group grid = cooperative_groups::this_grid();
  const double* src = f;
  int cur = 0;
  for (int d = 0; d < dm.dim; ++d) {
    coarse_axis_pass(dm, d, true, c.S[d], c.N[d], src, c.tmp[cur]);
    grid.sync();
    src = c.tmp[cur];
    cur ^= 1;
  }
  {
    const int NX = dm.ne[0] * 2, NY = dm.ne[1] * 2, NZ = (dm.dim == 3) ? dm.ne[2] * 2 : 1;
    const long long total = (long long)NX * NY * NZ;
    double* x = c.tmp[cur ^ 1];
    for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < total;
         t += (long long)gridDim.x * blockDim.x) {
      const int X = (int)(t % NX), Y = (int)((t / NX) % NY), Z = (int)(t / ((long long)NX * NY));
      const double l = c.lam[0][X] + c.lam[1][Y] + (dm.dim == 3 ? c.lam[2][Z] : 0.0);
      const long long o = coarse_off(dm, X, Y, Z);
      x[o] = (l > tol) ? x[o] / l : 0.0;
    }
    grid.sync();
  }
  for (int d = dm.dim - 1; d >= 0; --d) {
    double* dst = (d == 0) ? u : c.tmp[cur];
    coarse_axis_pass(dm, d, false, c.S[d], c.N[d], src, dst);
    if (d > 0) grid.sync();
    src = dst;
    cur ^= 1;
  }
}

// The same passes as separate launches, for CUDA graphs whose branches run
// concurrently (no grid-wide co-residency needed).
__global__ void __launch_bounds__(256)
coarse_pass_kernel(LevelDims dm, int axis, int transpose, const double* __restrict__ S, int N,
                   const double* in, double* out) {
  coarse_axis_pass(dm, axis, transpose != 0, S, N, in, out);
}
__global__ void __launch_bounds__(256)
coarse_scale_kernel(LevelDims dm, CoarseFdm c, double* x, double tol) {
  const int NX = dm.ne[0] * 2, NY = dm.ne[1] * 2, NZ = (dm.dim == 3) ? dm.ne[2] * 2 : 1;
  const long long total = (long long)NX * NY * NZ;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < total;
       t += (long long)gridDim.x * blockDim.x) {
    const int X = (int)(t % NX), Y = (int)((t / NX) % NY), Z = (int)(t / ((long long)NX * NY));
    const double l = c.lam[0][X] + c.lam[1][Y] + (dm.dim == 3 ? c.lam[2][Z] : 0.0);
    const long long o = coarse_off(dm, X, Y, Z);
    x[o] = (l > tol) ? x[o] / l : 0.0;
  }
}

static int launch_coarse_split(const LevelDims& dm, const CoarseFdm& c, const double* f, double* u,
                               int blocks, double tol, cudaStream_t s) {
  const double* src = f;
  int cur = 0;
  for (int d = 0; d < dm.dim; ++d) {
    count_launch(); coarse_pass_kernel<<<blocks, 256, 0, s>>>(dm, d, 1, c.S[d], c.N[d], src, c.tmp[cur]);
    src = c.tmp[cur];
    cur ^= 1;
  }
  count_launch(); coarse_scale_kernel<<<blocks, 256, 0, s>>>(dm, c, c.tmp[cur ^ 1], tol);
  for (int d = dm.dim - 1; d >= 0; --d) {
    double* dst = (d == 0) ? u : c.tmp[cur];
    count_launch(); coarse_pass_kernel<<<blocks, 256, 0, s>>>(dm, d, 0, c.S[d], c.N[d], src, dst);
    src = dst;
    cur ^= 1;
  }
  return cudaGetLastError() == cudaSuccess ? PMG_OK : PMG_ECUDA;
}

int launch_coarse_fdm(const LevelDims& dm, const CoarseFdm& c, const double* f, double* u,
                      cudaStream_t s, bool cooperative) {
  struct Shape { int per_sm, nsm; };
  static PerDevice<Shape> shapes;
  int per_sm = 0, nsm = 0;
  const int rc = shapes.with(
      [](Shape& sh, int dev) {
        return (cudaDeviceGetAttribute(&sh.nsm, cudaDevAttrMultiProcessorCount, dev) == cudaSuccess &&
                cudaOccupancyMaxActiveBlocksPerMultiprocessor(&sh.per_sm, coarse_fdm_fused_kernel, 256, 0) ==
                    cudaSuccess)
                   ? (int)PMG_OK
                   : (int)PMG_ECUDA;
      },
      [&](Shape& sh) {
        per_sm = sh.per_sm;
        nsm = sh.nsm;
        return (int)PMG_OK;
      });
  if (rc != PMG_OK) return rc;
  long long want = (dm.ndof + 255) / 256;
  long long cap = (long long)per_sm * nsm;
  int blocks = (int)(want < cap ? want : cap);
  if (blocks < 1) blocks = 1;
  double tol = 1e-13 * c.lam_max;
  if (!cooperative) return launch_coarse_split(dm, c, f, u, blocks, tol, s);
  LevelDims dmv = dm;
  CoarseFdm cv = c;
  const double* fv = f;
  double* uv = u;
  void* args[] = {&dmv, &cv, &fv, &uv, &tol};
  count_launch();
  cudaError_t e = cudaLaunchCooperativeKernel((const void*)coarse_fdm_fused_kernel, dim3(blocks),
                                              dim3(256), args, 0, s);
  return e == cudaSuccess ? PMG_OK : PMG_ECUDA;
}

// ---------------------------------------------------------------------------
// Vector kernels of Algorithm 2.  Reductions are deterministic: fixed grid,
// per-block partial sums in a fixed order, final sum by the last block to
// finish (threadfence + counter), also in a fixed order.
// ---------------------------------------------------------------------------
template <typename Ta, typename Tb>
__global__ void convert_kernel(const Ta* __restrict__ in, Tb* __restrict__ out, long long n) {
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < n;
       t += (long long)gridDim.x * blockDim.x)
    out[t] = (Tb)in[t];
}
template <typename Ta, typename Tb>
void launch_convert(const Ta* in, Tb* out, long long n, cudaStream_t s) {
  long long blocks = (n + 255) / 256;
  if (blocks > 152 * 32) blocks = 152 * 32;
  if (blocks < 1) blocks = 1;
  count_launch(); convert_kernel<Ta, Tb><<<(unsigned)blocks, 256, 0, s>>>(in, out, n);
}
template void launch_convert<double, float>(const double*, float*, long long, cudaStream_t);
template void launch_convert<float, double>(const float*, double*, long long, cudaStream_t);

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  return v;
}

// Block-level sum of two values in fixed order; result valid in thread 0.
__device__ __forceinline__ void block_sum2(double& a, double& b) {
  __shared__ double sa[32], sb[32];
  a = warp_sum(a);
  b = warp_sum(b);
  int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  if (l == 0) { sa[w] = a; sb[w] = b; }
  __syncthreads();
  if (w == 0) {
    int nw = blockDim.x >> 5;
    a = l < nw ? sa[l] : 0.0;
    b = l < nw ? sb[l] : 0.0;
    a = warp_sum(a);
    b = warp_sum(b);
  }
}

// Final reduction of the per-block partials by the last block; out[0..1].
__device__ void finish_reduce(double a, double b, double* partial, unsigned* counter, double* out,
                              int* status, int check) {
  __shared__ bool last;
  if (threadIdx.x == 0) {
    partial[2 * blockIdx.x] = a;
    partial[2 * blockIdx.x + 1] = b;
    __threadfence();
    unsigned prev = atomicAdd(counter, 1u);
    last = (prev == gridDim.x - 1);
  }
  __syncthreads();
  if (!last) return;
  __threadfence();
  double sa = 0.0, sb = 0.0;
  for (int i = threadIdx.x; i < (int)gridDim.x; i += blockDim.x) {
    sa += ((volatile double*)partial)[2 * i];
    sb += ((volatile double*)partial)[2 * i + 1];
  }
  block_sum2(sa, sb);
  if (threadIdx.x == 0) {
    out[0] = sa;
    out[1] = sb;
    if (check && status && *status == 0 && !(sa == sa && sa < 1e300)) *status = PMG_ENAN;
    *counter = 0u;
  }
}

// The CG vector kernels below run on `k` segments at once (one per right-hand side of
// the hierarchy; vectors hold the segments back to back, n entries each): grid.y = k,
// segment s = blockIdx.y with its own scalars (scal + s S_NUM), reduction partials
// (partial + s kPartialStride, counter + s) and control words (ctrl + kCtrlSeg + 4 s).
// A segment whose solve has finished (its active word is 0) is left untouched.
__device__ __forceinline__ int* seg_ctrl(int* ctrl, int s) { return ctrl + kCtrlSeg + 4 * s; }
__device__ __forceinline__ bool seg_active(const int* ctrl, int s) {
  return ctrl == nullptr || ctrl[kCtrlSeg + 4 * s + C_ACTIVE] != 0;
}

// out[0] = x.y ; out[1] = x.y2 (y2 may be null -> 0), per segment (out + s S_NUM)
__global__ void dot_kernel(const double* __restrict__ x, const double* __restrict__ y,
                           const double* __restrict__ y2, long long n, double* partial,
                           unsigned* counter, double* out) {
  const long long o = (long long)blockIdx.y * n;
  double a = 0.0, b = 0.0;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < n;
       t += (long long)gridDim.x * blockDim.x) {
    double xv = x[o + t];
    a = fma(xv, y[o + t], a);
    if (y2) b = fma(xv, y2[o + t], b);
  }
  block_sum2(a, b);
  finish_reduce(a, b, partial + blockIdx.y * kPartialStride, counter + blockIdx.y, out + blockIdx.y * S_NUM,
                nullptr, 0);
}

void launch_dot(const double* x, const double* y, const double* y2, long long n, int k, double* partial,
                unsigned* counter, double* out, int nblocks, cudaStream_t s) {
  count_launch(); dot_kernel<<<dim3(nblocks, k), 256, 0, s>>>(x, y, y2, n, partial, counter, out);
}

// alpha = delta / (p.q); u += alpha p; [r_old = r]; r -= alpha q; scal[S_RR] = r.r
__global__ void cg_update_kernel(double* __restrict__ u, double* __restrict__ r,
                                 double* __restrict__ r_old, const double* __restrict__ p,
                                 const double* __restrict__ q, const double* __restrict__ scal_all,
                                 int save_old, long long n, double* partial, unsigned* counter,
                                 int* ctrl, const int* it_dev) {
  const int sg = blockIdx.y;
  if (!seg_active(ctrl, sg)) return;                // uniform over the segment's blocks
  const double* scal = scal_all + sg * S_NUM;
  int* status = ctrl ? seg_ctrl(ctrl, sg) + C_STATUS : nullptr;
  if (it_dev) save_old = *it_dev >= 2;
  const double pq = scal[S_PQ];
  const double alpha = scal[S_DELTA] / pq;
  if (blockIdx.x == 0 && threadIdx.x == 0 && status && *status == 0) {   // the first status stays
    if (!(pq > 0.0) || !(scal[S_DELTA] > 0.0)) *status = (pq == pq) ? PMG_EBREAKDOWN : PMG_ENAN;
  }
  const long long o = (long long)sg * n;
  double a = 0.0;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < n;
       t += (long long)gridDim.x * blockDim.x) {
    u[o + t] = fma(alpha, p[o + t], u[o + t]);
    double rv = r[o + t];
    if (save_old) r_old[o + t] = rv;
    rv = fma(-alpha, q[o + t], rv);
    r[o + t] = rv;
    a = fma(rv, rv, a);
  }
  double b = 0.0;
  block_sum2(a, b);
  finish_reduce(a, b, partial + sg * kPartialStride, counter + sg, const_cast<double*>(scal) + S_RR, status, 1);
}

void launch_cg_update(double* u, double* r, double* r_old, const double* p, const double* q,
                      const double* scal, int save_old, long long n, int k, double* partial,
                      unsigned* counter, int* ctrl, int nblocks, cudaStream_t s, const int* it_dev) {
  count_launch();
  cg_update_kernel<<<dim3(nblocks, k), 256, 0, s>>>(u, r, r_old, p, q, scal, save_old, n, partial, counter,
                                                    ctrl, it_dev);
}

// beta = (z.r - z.r_old) / delta_old ; p = z + beta p   (reading C8; first: r_old = 0).
// With it_dev (device iteration counter): iteration 1 sets the first direction p = z,
// later iterations take z.r_old from the dot (r_old is zero until iteration 2
// saves it, so the first beta is again Fletcher-Reeves).
__global__ void p_update_kernel(double* __restrict__ p, const double* __restrict__ z,
                                const double* __restrict__ scal_all, int first, long long n,
                                const int* it_dev, const int* ctrl) {
  const int sg = blockIdx.y;
  if (!seg_active(ctrl, sg)) return;
  const double* scal = scal_all + sg * S_NUM;
  const bool copy = it_dev && *it_dev == 1;
  const double zro = first ? 0.0 : scal[S_ZRO];
  const double beta = (scal[S_ZR] - zro) / scal[S_DELTA];
  const long long o = (long long)sg * n;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < n;
       t += (long long)gridDim.x * blockDim.x)
    p[o + t] = copy ? z[o + t] : fma(beta, p[o + t], z[o + t]);
}

void launch_p_update(double* p, const double* z, const double* scal, int first, long long n, int k,
                     cudaStream_t s, const int* it_dev, const int* ctrl) {
  long long blocks = (n + 255) / 256;
  if (blocks > 152 * 32) blocks = 152 * 32;
  count_launch();
  p_update_kernel<<<dim3((unsigned)blocks, k), 256, 0, s>>>(p, z, scal, first, n, it_dev, ctrl);
}

// delta <- z.r (after the p update, which still needed the old delta), per segment
__global__ void set_delta_kernel(double* scal_all, int* ctrl, int k) {
  for (int sg = threadIdx.x; sg < k; sg += blockDim.x) {
    if (!seg_active(ctrl, sg)) continue;
    double* scal = scal_all + sg * S_NUM;
    scal[S_DELTA] = scal[S_ZR];
    int* status = ctrl ? seg_ctrl(ctrl, sg) + C_STATUS : nullptr;
    if (status && *status == 0 && !(scal[S_ZR] > 0.0))
      *status = (scal[S_ZR] == scal[S_ZR]) ? PMG_EBREAKDOWN : PMG_ENAN;
  }
}
void launch_set_delta(double* scal, int* ctrl, int k, cudaStream_t s) {
  count_launch(); set_delta_kernel<<<1, 32, 0, s>>>(scal, ctrl, k);
}

// MGCG control (Algorithm 2 with the convergence tests on the device), for k segments:
// ctrl[C_ITER] = current iteration, ctrl[C_ACTIVE] = segments still iterating; per
// segment its status word, iterations, result and active flag.  Host-driven solves
// read the control words after each iteration; a captured solve's loop is a graph
// `while` node whose condition these kernels set (GRAPH).
template <bool GRAPH>
__global__ void solve_begin_kernel(double* scal_all, int* ctrl, double* hist, int hstride, int k,
                                   cudaGraphConditionalHandle cond) {
  if (threadIdx.x != 0) return;
  int active = 0;
  for (int sg = 0; sg < k; ++sg) {
    double* scal = scal_all + sg * S_NUM;
    int* c = seg_ctrl(ctrl, sg);
    const double rr0 = scal[S_RR0];
    const double r0 = sqrt(rr0);
    hist[sg * hstride] = r0;
    scal[S_RR] = rr0;
    const bool go = (r0 == r0) && r0 != 0.0;
    c[C_ACTIVE] = go ? 1 : 0;
    c[C_ITER] = 0;
    c[C_RES] = (r0 == r0) ? (go ? PMG_ENOCONV : PMG_OK) : PMG_ENAN;
    active += go;
  }
  ctrl[C_ITER] = active ? 1 : 0;
  ctrl[C_ACTIVE] = active;
  if constexpr (GRAPH) cudaGraphSetConditional(cond, active ? 1u : 0u);
}

// After iteration ctrl[C_ITER]: record every active segment's ||r||; a segment stops on
// the global status word (a failure of a kernel shared by all segments), on its own
// status word, on ||r|| <= rtol ||r_0|| or at max_iter; the loop goes on while any
// segment is active.
template <bool GRAPH>
__global__ void solve_control_kernel(const double* scal_all, int* ctrl, double* hist, int hstride, int k,
                                     double rtol, int max_iter, cudaGraphConditionalHandle cond) {
  if (threadIdx.x != 0) return;
  const int it = ctrl[C_ITER];
  int active = 0;
  for (int sg = 0; sg < k; ++sg) {
    int* c = seg_ctrl(ctrl, sg);
    if (!c[C_ACTIVE]) continue;
    const double* scal = scal_all + sg * S_NUM;
    const double rn = sqrt(scal[S_RR]);
    const double r0 = sqrt(scal[S_RR0]);
    hist[sg * hstride + it] = rn;
    c[C_ITER] = it;
    int res = 1;
    if (ctrl[C_STATUS] != 0) res = ctrl[C_STATUS];
    else if (c[C_STATUS] != 0) res = c[C_STATUS];
    else if (rn <= rtol * r0) res = PMG_OK;
    else if (it >= max_iter) res = PMG_ENOCONV;
    if (res != 1) {
      c[C_RES] = res;
      c[C_ACTIVE] = 0;
    } else {
      ++active;
    }
  }
  ctrl[C_ACTIVE] = active;
  if (active) ctrl[C_ITER] = it + 1;
  if constexpr (GRAPH) cudaGraphSetConditional(cond, active ? 1u : 0u);
}

__global__ void solve_result_kernel(const double* scal_all, const int* ctrl, SolveResult* out, int k) {
  for (int sg = threadIdx.x; sg < k; sg += blockDim.x) {
    const double* scal = scal_all + sg * S_NUM;
    const int* c = ctrl + kCtrlSeg + 4 * sg;
    out[sg].r0 = sqrt(scal[S_RR0]);
    out[sg].rn = sqrt(scal[S_RR]);
    out[sg].iterations = c[C_ITER];
    out[sg].status = c[C_RES];
  }
}

void launch_solve_result(const double* scal, const int* ctrl, SolveResult* out, int k, cudaStream_t s) {
  count_launch(); solve_result_kernel<<<1, 32, 0, s>>>(scal, ctrl, out, k);
}

void launch_solve_begin(double* scal, int* ctrl, double* hist, int hstride, int k, const cudaGraphConditionalHandle* cond,
                        cudaStream_t s) {
  count_launch();
  if (cond) solve_begin_kernel<true><<<1, 1, 0, s>>>(scal, ctrl, hist, hstride, k, *cond);
  else solve_begin_kernel<false><<<1, 1, 0, s>>>(scal, ctrl, hist, hstride, k, cudaGraphConditionalHandle{});
}
void launch_solve_control(const double* scal, int* ctrl, double* hist, int hstride, int k, double rtol,
                          int max_iter, const cudaGraphConditionalHandle* cond, cudaStream_t s) {
  count_launch();
  if (cond) solve_control_kernel<true><<<1, 1, 0, s>>>(scal, ctrl, hist, hstride, k, rtol, max_iter, *cond);
  else
    solve_control_kernel<false><<<1, 1, 0, s>>>(scal, ctrl, hist, hstride, k, rtol, max_iter,
                                                cudaGraphConditionalHandle{});
}

// x -= mean(x)   (projection onto range(A) for periodic grids)
__global__ void sum_kernel(const double* __restrict__ x, long long n, double* partial,
                           unsigned* counter, double* out) {
  double a = 0.0, b = 0.0;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < n;
       t += (long long)gridDim.x * blockDim.x)
    a += x[t];
  block_sum2(a, b);
  finish_reduce(a, b, partial, counter, out, nullptr, 0);
}
__global__ void sub_kernel(double* __restrict__ x, long long n, const double* __restrict__ sum) {
  const double m = sum[0] / (double)n;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < n;
       t += (long long)gridDim.x * blockDim.x)
    x[t] -= m;
}
void launch_sub_mean(double* x, long long n, double* partial, unsigned* counter, double* scal,
                     int nblocks, cudaStream_t s) {
  count_launch(); sum_kernel<<<nblocks, 256, 0, s>>>(x, n, partial, counter, scal + S_MEAN);
  long long blocks = (n + 255) / 256;
  if (blocks > 152 * 32) blocks = 152 * 32;
  count_launch(); sub_kernel<<<(unsigned)blocks, 256, 0, s>>>(x, n, scal + S_MEAN);
}

}  // namespace pmg
