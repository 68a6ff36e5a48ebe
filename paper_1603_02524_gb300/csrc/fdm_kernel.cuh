// Weighted additive Schwarz patch solve by fast diagonalisation (Sec. 3.1).
//
// One CTA per subdomain.  The kernel serves both the element-centred (EA) and
// the face-centred (FA) families: every patch is a tensor product of three
// contiguous global 1-D index ranges (one per axis, wrapped on periodic axes,
// truncated at Dirichlet walls), and every axis carries its own eigen-table
// (S, lambda) of L_{s,d} S = M_{s,d} S Lambda and weight vector w.
//
//   gather   r_s = R_s r                          (0 outside the domain)
//   forward  t = (S_c^T (x) S_b^T (x) S_a^T) r_s   three in-place line passes
//   scale    t /= lambda_a + lambda_b + lambda_c
//   backward t = (S_c (x) S_b (x) S_a) t
//   scatter  u += omega * (w_c (x) w_b (x) w_a) t   (atomic: patches overlap)
//
// Positions outside the domain carry a decoupled identity in the eigen-table
// and weight 0, so the tensor algebra needs no special cases.  Each thread of
// a line pass owns one whole line: it loads the line into registers, then
// writes the transformed line back over the same shared-memory locations.
#pragma once

#include "pmg_internal.h"

namespace pmg {

// In-place transform of the lines of `buf` along one axis of length N.
// FORWARD: out_i = sum_a S[a][i] v_a  (S^T); else out_a = sum_i S[a][i] v_i.
template <typename T, int N, bool FORWARD>
__device__ __forceinline__ void line_pass(T* buf, const T* S, int nlines, int line_stride_lo,
                                          int lo_count, int line_stride_hi, int stride) {
  for (int l = threadIdx.x; l < nlines; l += blockDim.x) {
    const int base = (l % lo_count) * line_stride_lo + (l / lo_count) * line_stride_hi;
    T v[N];
#pragma unroll
    for (int a = 0; a < N; ++a) v[a] = buf[base + a * stride];
#pragma unroll 1
    for (int i = 0; i < N; ++i) {
      T s = T(0);
#pragma unroll
      for (int a = 0; a < N; ++a) s = fma(FORWARD ? S[a * N + i] : S[i * N + a], v[a], s);
      buf[base + i * stride] = s;
    }
  }
}

template <typename T>
__device__ __forceinline__ void atomic_add_t(T* p, T v) {
  atomicAdd(p, v);
}

template <typename T, int NA, int NB, int NC>
__global__ void __launch_bounds__(256)
fdm_kernel(LevelDims dm, FdmFamily<T> fam, const T* __restrict__ r, T* __restrict__ u, T omega) {
  constexpr int NN = NA * NB * NC;
  extern __shared__ __align__(16) unsigned char fdm_smem[];
  T* buf = reinterpret_cast<T*>(fdm_smem);
  T* Sa = buf + NN;
  T* Sb = Sa + NA * NA;
  T* Sc = Sb + NB * NB;
  T* la = Sc + NC * NC;
  T* lb = la + NA;
  T* lc = lb + NB;
  T* wa = lc + NC;
  T* wb = wa + NA;
  T* wc = wb + NB;

  const int ca = fam.ax[0].count, cb = fam.ax[1].count;
  const int pid = blockIdx.x;
  const int pa = pid % ca, pb = (pid / ca) % cb, pc = pid / (ca * cb);
  const int pidx[3] = {pa, pb, pc};

  // eigen-tables and weights of this patch
  {
    const T* gS[3] = {fam.ax[0].S + (size_t)pa * NA * NA, fam.ax[1].S + (size_t)pb * NB * NB,
                      fam.ax[2].S + (size_t)pc * NC * NC};
    for (int t = threadIdx.x; t < NA * NA; t += blockDim.x) Sa[t] = gS[0][t];
    for (int t = threadIdx.x; t < NB * NB; t += blockDim.x) Sb[t] = gS[1][t];
    for (int t = threadIdx.x; t < NC * NC; t += blockDim.x) Sc[t] = gS[2][t];
    if (threadIdx.x < NA) {
      la[threadIdx.x] = fam.ax[0].lam[(size_t)pa * NA + threadIdx.x];
      wa[threadIdx.x] = fam.ax[0].w[(size_t)pa * NA + threadIdx.x];
    }
    if (threadIdx.x < NB) {
      lb[threadIdx.x] = fam.ax[1].lam[(size_t)pb * NB + threadIdx.x];
      wb[threadIdx.x] = fam.ax[1].w[(size_t)pb * NB + threadIdx.x];
    }
    if (threadIdx.x < NC) {
      lc[threadIdx.x] = fam.ax[2].lam[(size_t)pc * NC + threadIdx.x];
      wc[threadIdx.x] = fam.ax[2].w[(size_t)pc * NC + threadIdx.x];
    }
  }

  // per buffer axis: first global 1-D index, size, node count of the physical axis
  int start[3], gN[3], npp[3], phys[3], per[3];
#pragma unroll
  for (int q = 0; q < 3; ++q) {
    phys[q] = fam.ax[q].phys;
    npp[q] = (phys[q] == 2) ? dm.NPz : dm.NP;
    start[q] = fam.ax[q].start0 + pidx[q] * npp[q];
    gN[q] = fam.ax[q].N;
    per[q] = fam.ax[q].periodic;
  }
  const long long nodes_el = (long long)dm.NP * dm.NP * dm.NPz;

  // element-major offset of buffer position (a, b, c), or -1 outside the domain
  auto offset = [&](int a, int b, int c) -> long long {
    const int loc[3] = {a, b, c};
    int X[3] = {0, 0, 0};
#pragma unroll
    for (int q = 0; q < 3; ++q) {
      int G = start[q] + loc[q];
      if (per[q]) {
        G %= gN[q];
        if (G < 0) G += gN[q];
      } else if (G < 0 || G >= gN[q]) {
        return -1;
      }
      X[phys[q]] = G;
    }
    const int NP = dm.NP;
    const int ex = X[0] / NP, i = X[0] % NP, ey = X[1] / NP, j = X[1] % NP;
    const int ez = X[2] / dm.NPz, k = X[2] % dm.NPz;
    return (((long long)ez * dm.ne[1] + ey) * dm.ne[0] + ex) * nodes_el + ((long long)k * NP + j) * NP + i;
  };

  for (int t = threadIdx.x; t < NN; t += blockDim.x) {
    const int a = t % NA, b = (t / NA) % NB, c = t / (NA * NB);
    const long long o = offset(a, b, c);
    buf[t] = o >= 0 ? r[o] : T(0);
  }
  __syncthreads();

  // forward transforms
  line_pass<T, NA, true>(buf, Sa, NB * NC, NA, NB * NC, 0, 1);
  __syncthreads();
  line_pass<T, NB, true>(buf, Sb, NA * NC, 1, NA, NA * NB, NA);
  __syncthreads();
  if (NC > 1) {
    line_pass<T, NC, true>(buf, Sc, NA * NB, 1, NA * NB, 0, NA * NB);
    __syncthreads();
  }
  for (int t = threadIdx.x; t < NN; t += blockDim.x) {
    const int a = t % NA, b = (t / NA) % NB, c = t / (NA * NB);
    buf[t] = buf[t] / (la[a] + lb[b] + lc[c]);
  }
  __syncthreads();
  if (NC > 1) {
    line_pass<T, NC, false>(buf, Sc, NA * NB, 1, NA * NB, 0, NA * NB);
    __syncthreads();
  }
  line_pass<T, NB, false>(buf, Sb, NA * NC, 1, NA, NA * NB, NA);
  __syncthreads();
  line_pass<T, NA, false>(buf, Sa, NB * NC, NA, NB * NC, 0, 1);
  __syncthreads();

  for (int t = threadIdx.x; t < NN; t += blockDim.x) {
    const int a = t % NA, b = (t / NA) % NB, c = t / (NA * NB);
    const T wt = wa[a] * wb[b] * wc[c];
    if (wt != T(0)) {
      const long long o = offset(a, b, c);
      if (o >= 0) atomic_add_t(u + o, omega * wt * buf[t]);
    }
  }
}

template <typename T, int NA, int NB, int NC>
int fdm_launch(const LevelDims& dm, const FdmFamily<T>& fam, const T* r, T* u, T omega,
               cudaStream_t s) {
  const size_t smem =
      sizeof(T) * ((size_t)NA * NB * NC + NA * NA + NB * NB + NC * NC + 2 * (NA + NB + NC));
  static bool attr_done = false;
  if (!attr_done && smem > 48 * 1024) {
    if (cudaFuncSetAttribute(fdm_kernel<T, NA, NB, NC>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)smem) != cudaSuccess)
      return PMG_ECUDA;
  }
  attr_done = true;
  if (fam.count_total <= 0) return PMG_OK;
  count_launch(); fdm_kernel<T, NA, NB, NC><<<fam.count_total, 256, smem, s>>>(dm, fam, r, u, omega);
  return cudaGetLastError() == cudaSuccess ? PMG_OK : PMG_ECUDA;
}

}  // namespace pmg
