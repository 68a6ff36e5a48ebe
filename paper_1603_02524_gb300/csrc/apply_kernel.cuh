// Sum-factorised DG operator apply (shared by the FP64 / fp32 library
// kernels and the double-float outer apply).
//
// Paper: Stiller, arXiv 1603.02524, Sec. 2.4 (1-D blocks of Eq. L:generic) and
// the tensor form of the discrete problem (Sec. 2.2, reading C1 in 3-D).
#pragma once

#include <type_traits>

#include "pmg_internal.h"

namespace pmg {

// table / vector loads through the read-only path (dfloat: one 8-byte load)
template <typename T>
__device__ __forceinline__ T ldg(const T* p) { return __ldg(p); }

// c + a * b, fused (dfloat: the accumulate form of dfloat.cuh)
__device__ __forceinline__ double madd(double a, double b, double c) { return ::fma(a, b, c); }
__device__ __forceinline__ float madd(float a, float b, float c) { return fmaf(a, b, c); }

// 16-byte vector of T read through the read-only path (dfloat: two values per vector)
template <typename T> struct AVec;
template <> struct AVec<float> {
  using V = float4;
  static constexpr int W = 4;
  __device__ static float get(const float4& v, int k) { return k == 0 ? v.x : k == 1 ? v.y : k == 2 ? v.z : v.w; }
};
template <> struct AVec<double> {
  using V = double2;
  static constexpr int W = 2;
  __device__ static double get(const double2& v, int k) { return k == 0 ? v.x : v.y; }
};
template <> struct AVec<dfloat> {
  using V = float4;
  static constexpr int W = 2;
  __device__ static dfloat get(const float4& v, int k) { return k == 0 ? dfloat(v.x, v.y) : dfloat(v.z, v.w); }
};
template <typename T>
__host__ __device__ constexpr int apad(int n) { return (n + AVec<T>::W - 1) / AVec<T>::W * AVec<T>::W; }

// acc[0..N) += row[0..N) * x, row a 16-byte aligned, padded row of a global table
template <typename T, int N>
__device__ __forceinline__ void apply_axpy(T (&acc)[N], const T* row, T x) {
  using A = AVec<T>;
  const typename A::V* r = reinterpret_cast<const typename A::V*>(row);
#pragma unroll
  for (int c = 0; c < apad<T>(N) / A::W; ++c) {
    const typename A::V w = __ldg(r + c);
#pragma unroll
    for (int k = 0; k < A::W; ++k)
      if (c * A::W + k < N) acc[c * A::W + k] = madd(A::get(w, k), x, acc[c * A::W + k]);
  }
}

// ---------------------------------------------------------------------------
// Transfers between orders (Sec. 3.2): J (NF x NC, J[a][o] = coarse basis function
// o at fine GLL node a) is centro-symmetric, J[NF-1-a][NC-1-o] = J[a][o], because
// both node sets are symmetric about the element centre.  Along one axis the
// restriction y = J^T x and the prolongation y = J x then split into an even part
// on the sums x[i] + x[n-1-i] and an odd part on the differences (the middle node,
// where there is one, enters the even part alone):
//   e[a][o] = (J[a][o] + J[a][NC-1-o]) / 2   (a <= middle, o <= middle)
//   d[a][o] = (J[a][o] - J[a][NC-1-o]) / 2   (a, o below the middle)
// about half the multiply-adds of the dense contraction.  The folded coefficients
// are kernel parameters: the contractions below index them with compile-time
// indices only, so they are read as constant operands, with no load instruction.
// ---------------------------------------------------------------------------
template <typename T, int NF, int NC>
struct FoldedJ {
  static constexpr int HF = NF / 2, HC = NC / 2, EF = NF - HF, EC = NC - HC;
  T e[EF * EC];
  T d[(HF * HC) > 0 ? HF * HC : 1];
};
template <typename T, int NF>
struct FoldedJ<T, NF, 0> {};

// host: the folded coefficients of J (row-major NF x NC, FP64), rounded to T
template <typename T, int NF, int NC>
FoldedJ<T, NF, NC> fold_interpolation(const double* J) {
  using F = FoldedJ<T, NF, NC>;
  F f{};
  for (int a = 0; a < F::EF; ++a)
    for (int o = 0; o < F::EC; ++o) f.e[a * F::EC + o] = T(0.5 * (J[a * NC + o] + J[a * NC + (NC - 1 - o)]));
  for (int a = 0; a < F::HF; ++a)
    for (int o = 0; o < F::HC; ++o) f.d[a * F::HC + o] = T(0.5 * (J[a * NC + o] - J[a * NC + (NC - 1 - o)]));
  return f;
}

// y[0..NC) = J^T x[0..NF) along one axis; each output is handed to put(index, value)
// as soon as it is formed (an output pair at a time), so no output array is held
template <typename T, int NF, int NC, typename Put>
__device__ __forceinline__ void fold_restrict(const FoldedJ<T, NF, NC>& J, const T (&x)[NF], Put&& put) {
  using F = FoldedJ<T, NF, NC>;
  T sp[F::EF], sm[F::HF > 0 ? F::HF : 1];
#pragma unroll
  for (int a = 0; a < F::HF; ++a) {
    sp[a] = x[a] + x[NF - 1 - a];
    sm[a] = x[a] - x[NF - 1 - a];
  }
  if constexpr (F::EF > F::HF) sp[F::HF] = x[F::HF];
#pragma unroll
  for (int o = 0; o < F::EC; ++o) {
    T ev = T(0);
#pragma unroll
    for (int a = 0; a < F::EF; ++a) ev = madd(J.e[a * F::EC + o], sp[a], ev);
    if (o < F::HC) {
      T od = T(0);
#pragma unroll
      for (int a = 0; a < F::HF; ++a) od = madd(J.d[a * F::HC + o], sm[a], od);
      put(o, ev + od);
      put(NC - 1 - o, ev - od);
    } else {
      put(o, ev);
    }
  }
}

// y[0..NF) = J x[0..NC) along one axis, outputs handed to put(index, value)
template <typename T, int NF, int NC, typename Put>
__device__ __forceinline__ void fold_prolong(const FoldedJ<T, NF, NC>& J, const T (&x)[NC], Put&& put) {
  using F = FoldedJ<T, NF, NC>;
  T sp[F::EC], sm[F::HC > 0 ? F::HC : 1];
#pragma unroll
  for (int o = 0; o < F::HC; ++o) {
    sp[o] = x[o] + x[NC - 1 - o];
    sm[o] = x[o] - x[NC - 1 - o];
  }
  if constexpr (F::EC > F::HC) sp[F::HC] = x[F::HC];
#pragma unroll
  for (int a = 0; a < F::EF; ++a) {
    T ev = T(0);
#pragma unroll
    for (int o = 0; o < F::EC; ++o) ev = madd(J.e[a * F::EC + o], sp[o], ev);
    if (a < F::HF) {
      T od = T(0);
#pragma unroll
      for (int o = 0; o < F::HC; ++o) od = madd(J.d[a * F::HC + o], sm[o], od);
      put(a, ev + od);
      put(NF - 1 - a, ev - od);
    } else {
      put(a, ev);
    }
  }
}

// Allow `bytes` of dynamic shared memory for kernel `fn` (once per kernel).
template <typename K>
static bool set_smem(K fn, size_t bytes) {
  if (bytes <= 48 * 1024) return true;
  return cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes) ==
         cudaSuccess;
}

// ---------------------------------------------------------------------------
// Operator apply: v = A u or v = f - A u  (Eq. discrete problem, 3-D tensor form)
//
// One thread owns one nodal line of one element per axis pass.  The element is
// staged in shared memory; the line is contracted with the element's dense
// 1-D block L^0 (Eq. L:generic); the neighbour blocks L^-/L^+ have rank <= 3
// and need only the neighbour line's end value and end derivative
// (sum_k D_{P,k} u_k^{m-1}, sum_k D_{0,k} u_k^{m+1}), which the thread reads
// from global memory (L2-resident: neighbouring CTAs read the same elements).
// Each pass result is scaled by the diagonal masses of the two other axes and
// accumulated in shared memory.
// ---------------------------------------------------------------------------
// y = M_d^-1 L_d u on one line of element e along axis d (nodes off + a * stride of
// the element, values x): the element's own block L^0 (even-odd form when the block
// is centro-symmetric), plus the neighbour blocks L^-, L^+ from the adjacent lines
// in global u.
// The tables of axis d, selected with compile-time indices (a runtime index into
// the kernel-parameter arrays would copy them to local memory).
template <typename T>
struct ApplyAxis {
  const T* L0;
  const int* sym;
  const T* cpl;
  int m;              // element index along the axis
  int ned;            // elements along the axis
  long long estride;  // element stride of the axis
};
template <typename T>
__device__ __forceinline__ ApplyAxis<T> apply_axis(const LevelDims& dm, const ApplyTables<T>& at,
                                                   const int (&me)[3], int d) {
  ApplyAxis<T> a;
  a.L0 = d == 0 ? at.L0[0] : (d == 1 ? at.L0[1] : at.L0[2]);
  a.sym = d == 0 ? at.sym[0] : (d == 1 ? at.sym[1] : at.sym[2]);
  a.cpl = d == 0 ? at.cpl[0] : (d == 1 ? at.cpl[1] : at.cpl[2]);
  a.m = d == 0 ? me[0] : (d == 1 ? me[1] : me[2]);
  a.ned = d == 0 ? dm.ne[0] : (d == 1 ? dm.ne[1] : dm.ne[2]);
  a.estride = (d == 0) ? 1 : (d == 1 ? (long long)dm.ne[0] : (long long)dm.ne[0] * dm.ne[1]);
  return a;
}

template <typename T, int NP, int NODES, typename TIO>
__device__ __forceinline__ void apply_line(const ApplyTables<T>& at, const ApplyAxis<T>& ax,
                                           const TIO* __restrict__ u, long long e, int off, int stride,
                                           const T (&x)[NP], T (&y)[NP]) {
  constexpr int P = NP - 1;
  constexpr int H = NP / 2, NE = NP - H, NO = H;
  constexpr int PNP = apad<T>(NP);
  if constexpr (sizeof(T) == 8) {
    // FP64 and double-float: the neighbour end terms first (their loads in flight during
    // the element's own block); mirrored coupling rows folded into the even-odd
    // accumulation (the tables flag them).  fp32 (below) keeps the order of the
    // contraction first and unfolded tables: holding the end terms across the block
    // spilled its 48-register budget.
    const T* L0 = ax.L0 + (size_t)ax.m * NP * PNP;
    // neighbour blocks L^-, L^+ (rank <= 3, already scaled by M_d^-1)
    const T* c = ax.cpl + (size_t)ax.m * (2 * PNP + 8);
    const long long estride = ax.estride;
    const int ned = ax.ned;
    // end value and end derivative (row Drow of the differentiation matrix) of the
    // neighbour line un.  Double-float apply of an FP64 vector: the dot product runs
    // in FP64 and only its result and the end value are split into two fp32 words
    // (splitting all NP values and accumulating in double-float took about half of
    // that kernel's issue slots; the FP64 pipe is otherwise idle there)
    auto end_terms = [&](const TIO* un, const T* Drow, const double* Drow_d, int iend, T& uend, T& dend) {
      if constexpr (std::is_same<T, dfloat>::value && std::is_same<TIO, double>::value) {
        double s = 0.0, v = 0.0;
  #pragma unroll
        for (int a = 0; a < NP; ++a) {
          const double val = __ldg(un + a * stride);
          s = ::fma(__ldg(Drow_d + a), val, s);
          if (a == iend) v = val;
        }
        uend = T(v);
        dend = T(s);
      } else {
        T s = T(0), v = T(0);
  #pragma unroll
        for (int a = 0; a < NP; ++a) {
          T val = T(__ldg(un + a * stride));
          s = madd(ldg(Drow + a), val, s);
          if (a == iend) v = val;
        }
        uend = v;
        dend = s;
      }
    };
    const bool hasL = ldg(c + 2 * PNP + 2) != T(0), hasR = ldg(c + 2 * PNP + 5) != T(0);
    T uP = T(0), dP = T(0), u0 = T(0), d0 = T(0);

    {
      if (hasL) {                                // neighbour m-1
        const long long en = (ax.m > 0) ? e - estride : e + (long long)(ned - 1) * estride;
        end_terms(u + en * NODES + off, at.DP, at.DPd, P, uP, dP);
      }
      if (hasR) {                                // neighbour m+1
        const long long en = (ax.m < ned - 1) ? e + estride : e - (long long)(ned - 1) * estride;
        end_terms(u + en * NODES + off, at.D0, at.D0d, 0, u0, d0);
      }
    }
    // folded coupling (both neighbours, mirrored rows c_R[P - i] = c_L[i]): c_L u_P + c_R u_0
    // = even part x (u_P + u_0) + odd part x (u_P - u_0)
    const bool csym = ldg(c + 2 * PNP + 6) != T(0);
    if (__ldg(ax.sym + ax.m)) {
      // even-odd split of the centro-symmetric block (folded, transposed rows)
      constexpr int PE = apad<T>(NE), PO = apad<T>(NO > 0 ? NO : 1);
      T xp[NE], xm[NO > 0 ? NO : 1];
  #pragma unroll
      for (int a = 0; a < H; ++a) {
        xp[a] = x[a] + x[P - a];
        xm[a] = x[a] - x[P - a];
      }
      if (NE > H) xp[NE - 1] = x[H];
      T ae[NE], ao[NO > 0 ? NO : 1];
  #pragma unroll
      for (int i = 0; i < NE; ++i) ae[i] = T(0);
  #pragma unroll
      for (int i = 0; i < NO; ++i) ao[i] = T(0);
  #pragma unroll
      for (int a = 0; a < NE; ++a) apply_axpy<T, NE>(ae, L0 + a * PE, xp[a]);
      if constexpr (NO > 0) {
  #pragma unroll
        for (int a = 0; a < NO; ++a)
          apply_axpy<T, NO>(reinterpret_cast<T(&)[NO]>(ao), L0 + NE * PE + a * PO, xm[a]);
      }
      if (csym) {
        apply_axpy<T, NE>(ae, c, uP + u0);
        if constexpr (NO > 0) apply_axpy<T, NO>(reinterpret_cast<T(&)[NO]>(ao), c + PNP, uP - u0);
      }
  #pragma unroll
      for (int i = 0; i < H; ++i) {
        y[i] = ae[i] + ao[i];
        y[P - i] = ae[i] - ao[i];
      }
      if (NE > H) y[H] = ae[H];
    } else {
  #pragma unroll
      for (int i = 0; i < NP; ++i) y[i] = T(0);
  #pragma unroll
      for (int a = 0; a < NP; ++a) apply_axpy<T, NP>(y, L0 + a * PNP, x[a]);
    }
    if (!csym) {
      if (hasL) apply_axpy<T, NP>(y, c, uP);
      if (hasR) apply_axpy<T, NP>(y, c + PNP, u0);
    }
    if (hasL) y[0] += ldg(c + 2 * PNP + 0) * dP - ldg(c + 2 * PNP + 1) * uP;
    if (hasR) y[P] = y[P] - (ldg(c + 2 * PNP + 3) * d0 + ldg(c + 2 * PNP + 4) * u0);
  } else {
    const T* L0 = ax.L0 + (size_t)ax.m * NP * PNP;
    if (__ldg(ax.sym + ax.m)) {
      // even-odd split of the centro-symmetric block (folded, transposed rows)
      constexpr int PE = apad<T>(NE), PO = apad<T>(NO > 0 ? NO : 1);
      T xp[NE], xm[NO > 0 ? NO : 1];
  #pragma unroll
      for (int a = 0; a < H; ++a) {
        xp[a] = x[a] + x[P - a];
        xm[a] = x[a] - x[P - a];
      }
      if (NE > H) xp[NE - 1] = x[H];
      T ae[NE], ao[NO > 0 ? NO : 1];
  #pragma unroll
      for (int i = 0; i < NE; ++i) ae[i] = T(0);
  #pragma unroll
      for (int i = 0; i < NO; ++i) ao[i] = T(0);
  #pragma unroll
      for (int a = 0; a < NE; ++a) apply_axpy<T, NE>(ae, L0 + a * PE, xp[a]);
      if constexpr (NO > 0) {
  #pragma unroll
        for (int a = 0; a < NO; ++a)
          apply_axpy<T, NO>(reinterpret_cast<T(&)[NO]>(ao), L0 + NE * PE + a * PO, xm[a]);
      }
  #pragma unroll
      for (int i = 0; i < H; ++i) {
        y[i] = ae[i] + ao[i];
        y[P - i] = ae[i] - ao[i];
      }
      if (NE > H) y[H] = ae[H];
    } else {
  #pragma unroll
      for (int i = 0; i < NP; ++i) y[i] = T(0);
  #pragma unroll
      for (int a = 0; a < NP; ++a) apply_axpy<T, NP>(y, L0 + a * PNP, x[a]);
    }
    // neighbour blocks L^-, L^+ (rank <= 3, already scaled by M_d^-1)
    const T* c = ax.cpl + (size_t)ax.m * (2 * PNP + 8);
    const long long estride = ax.estride;
    const int ned = ax.ned;
    // end value and end derivative (row Drow of the differentiation matrix) of the
    // neighbour line un.  Double-float apply of an FP64 vector: the dot product runs
    // in FP64 and only its result and the end value are split into two fp32 words
    // (splitting all NP values and accumulating in double-float took about half of
    // that kernel's issue slots; the FP64 pipe is otherwise idle there)
    auto end_terms = [&](const TIO* un, const T* Drow, const double* Drow_d, int iend, T& uend, T& dend) {
      if constexpr (std::is_same<T, dfloat>::value && std::is_same<TIO, double>::value) {
        double s = 0.0, v = 0.0;
  #pragma unroll
        for (int a = 0; a < NP; ++a) {
          const double val = __ldg(un + a * stride);
          s = ::fma(__ldg(Drow_d + a), val, s);
          if (a == iend) v = val;
        }
        uend = T(v);
        dend = T(s);
      } else {
        T s = T(0), v = T(0);
  #pragma unroll
        for (int a = 0; a < NP; ++a) {
          T val = T(__ldg(un + a * stride));
          s = madd(ldg(Drow + a), val, s);
          if (a == iend) v = val;
        }
        uend = v;
        dend = s;
      }
    };
    if (ldg(c + 2 * PNP + 2) != T(0)) {          // neighbour m-1 exists
      long long en = (ax.m > 0) ? e - estride : e + (long long)(ned - 1) * estride;
      T uP, dP;
      end_terms(u + en * NODES + off, at.DP, at.DPd, P, uP, dP);
      apply_axpy<T, NP>(y, c, uP);
      y[0] += ldg(c + 2 * PNP + 0) * dP - ldg(c + 2 * PNP + 1) * uP;
    }
    if (ldg(c + 2 * PNP + 5) != T(0)) {          // neighbour m+1 exists
      long long en = (ax.m < ned - 1) ? e + estride : e - (long long)(ned - 1) * estride;
      T u0, d0;
      end_terms(u + en * NODES + off, at.D0, at.D0d, 0, u0, d0);
      apply_axpy<T, NP>(y, c + PNP, u0);
      y[P] = y[P] - (ldg(c + 2 * PNP + 3) * d0 + ldg(c + 2 * PNP + 4) * u0);
    }
  }
}

template <int DIM, int NP>
struct ApplyShape {
  static constexpr int LINES = (DIM == 3) ? NP * NP : NP;
  static constexpr int NODES = (DIM == 3) ? NP * NP * NP : NP * NP;
  static constexpr int EPB = (128 / LINES) > 0 ? (128 / LINES) : 1;
  static constexpr int THREADS = ((EPB * LINES + 31) / 32) * 32;
  // CTAs per SM the register budget must allow (8-byte types): two for the 3-D
  // P = 16 kernel (320 threads), whose double-float form would otherwise take 114
  // registers and run one CTA per SM
  static constexpr int MINB8 = (DIM == 3 && NP == 17) ? 2 : 0;
  // fp32 P = 16: four CTAs per SM (51 registers) to hide the neighbour-line loads
  static constexpr int MINB4 = (DIM == 3 && NP == 17) ? 4 : 0;
};

// T: arithmetic and table type; TIO: type of u, f, v in global memory.
// NPC > 0 (with RESIDUAL): the residual is not stored but restricted at once,
// fc = (J (x) J (x) J)^T (f - A u) element by element (Sec. 3.2; J folded as in
// FoldedJ), in the operation order of the separate restriction kernel.
template <typename T, int DIM, int NP, bool RESIDUAL, typename TIO = T, int NPC = 0>
__global__ void __launch_bounds__(ApplyShape<DIM, NP>::THREADS,
                                  sizeof(T) == 8 ? ApplyShape<DIM, NP>::MINB8 : ApplyShape<DIM, NP>::MINB4)
apply_kernel(LevelDims dm, ApplyTables<T> at, const TIO* __restrict__ u, const TIO* __restrict__ f,
             TIO* __restrict__ v, FoldedJ<T, NP, NPC> J = FoldedJ<T, NP, NPC>{}, TIO* __restrict__ fc = nullptr,
             const int* __restrict__ unz = nullptr) {
  static_assert(NPC == 0 || (RESIDUAL && NPC < NP), "fused restriction: residual, coarser order");
  using S = ApplyShape<DIM, NP>;
  constexpr int P = NP - 1;
  extern __shared__ __align__(16) unsigned char apply_smem[];
  T* su = reinterpret_cast<T*>(apply_smem);
  T* acc = su + S::EPB * S::NODES;
  const int tid = threadIdx.x;
  const long long e0 = (long long)blockIdx.x * S::EPB;
  const long long nodes_blk = (long long)S::EPB * S::NODES;
  const long long total = dm.nelem * S::NODES;
  if constexpr (NPC == 0) {
    // u identically zero (flag from any_nonzero_kernel): A u = 0, so v = f (or 0)
    if (unz && __ldg(unz) == 0) {
      for (int t = tid; t < nodes_blk; t += blockDim.x) {
        const long long g = e0 * S::NODES + t;
        if (g < total) v[g] = RESIDUAL ? f[g] : TIO(0);
      }
      return;
    }
  }
  // element coordinates of the block's elements (one 64-bit division set per element)
  __shared__ int s_me[S::EPB][3];
  if (tid < S::EPB) {
    const long long ee = e0 + tid;
    s_me[tid][0] = (int)(ee % dm.ne[0]);
    s_me[tid][1] = (int)((ee / dm.ne[0]) % dm.ne[1]);
    s_me[tid][2] = (int)(ee / ((long long)dm.ne[0] * dm.ne[1]));
  }
  for (int t = tid; t < nodes_blk; t += blockDim.x) {
    long long g = e0 * S::NODES + t;
    su[t] = g < total ? T(u[g]) : T(0);
  }
  __syncthreads();
  const int el = tid / S::LINES;
  const int line = tid % S::LINES;
  const long long e = e0 + el;
  const bool active = (el < S::EPB) && (e < dm.nelem);
  int me[3] = {0, 0, 0};
  if (active) {
    me[0] = s_me[el][0];
    me[1] = s_me[el][1];
    me[2] = s_me[el][2];
  }
  T* sel = su + el * S::NODES;
  T* ael = acc + el * S::NODES;
  constexpr int H = NP / 2, NE = NP - H, NO = H;
  // axes unrolled (line offsets and strides become compile-time constants) for the
  // fp32 and FP64 kernels, except FP64 at P = 16, whose register cap would then spill;
  // the double-float kernel was measured faster without (instruction-cache pressure)
  constexpr int UNR = (std::is_same<T, dfloat>::value || (sizeof(T) == 8 && NP == 17)) ? 1 : DIM;
#pragma unroll UNR
  for (int d = 0; d < DIM; ++d) {
    if (active) {
      int off, stride;
      if (DIM == 3) {
        if (d == 0) { off = line * NP; stride = 1; }
        else if (d == 1) { off = (line / NP) * NP * NP + line % NP; stride = NP; }
        else { off = line; stride = NP * NP; }
      } else {
        if (d == 0) { off = line * NP; stride = 1; }
        else { off = line; stride = NP; }
      }
      T x[NP], y[NP];
#pragma unroll
      for (int a = 0; a < NP; ++a) x[a] = sel[off + a * stride];
      apply_line<T, NP, S::NODES, TIO>(at, apply_axis(dm, at, me, d), u, e, off, stride, x, y);
#pragma unroll
      for (int i = 0; i < NP; ++i) {
        if (d == 0) ael[off + i * stride] = y[i];
        else ael[off + i * stride] += y[i];
      }
    }
    __syncthreads();
  }
  // v = (M_z (x) M_y (x) M_x) * (sum over axes of M_d^-1 L_d u)
  for (int t = tid; t < nodes_blk; t += blockDim.x) {
    long long g = e0 * S::NODES + t;
    if (g >= total) {
      if constexpr (NPC > 0) acc[t] = T(0);
      continue;
    }
    const int le = t / S::NODES;
    const int nd = t - le * S::NODES;
    const int i = nd % NP, j = (nd / NP) % NP;
    const int mx = s_me[le][0], my = s_me[le][1];
    T m = ldg(at.M[0] + (size_t)mx * NP + i) * ldg(at.M[1] + (size_t)my * NP + j);
    if (DIM == 3) {
      const int k = nd / (NP * NP);
      const int mz = s_me[le][2];
      m = m * ldg(at.M[2] + (size_t)mz * NP + k);
    }
    const T val = m * acc[t];
    if constexpr (NPC > 0) acc[t] = T(f[g]) - val;
    else v[g] = RESIDUAL ? TIO(T(f[g]) - val) : TIO(val);
  }
  if constexpr (NPC > 0) {
    // restriction of the element residuals (in acc): x, y and z passes with J^T,
    // one thread per line of a pass (even-odd folded, coefficients in parameters)
    constexpr int NZF = (DIM == 3) ? NP : 1;
    constexpr int B1 = NPC * NP * NZF, B2 = NPC * NPC * NZF;
    __syncthreads();
    T* b1 = su;                                  // staged u is no longer needed
    #pragma unroll 1
    for (int t = tid; t < S::EPB * NP * NZF; t += blockDim.x) {      // x: lines (y, z)
      const int le = t / (NP * NZF), rest = t - le * (NP * NZF);
      const T* rr = acc + le * S::NODES + rest * NP;
      T x[NP];
#pragma unroll
      for (int a = 0; a < NP; ++a) x[a] = rr[a];
      T* dst = b1 + le * B1 + rest * NPC;
      fold_restrict<T, NP, NPC>(J, x, [&](int o, T v) { dst[o] = v; });
    }
    __syncthreads();
    T* b2 = acc;
    #pragma unroll 1
    for (int t = tid; t < S::EPB * NPC * NZF; t += blockDim.x) {     // y: lines (x', z)
      const int le = t / (NPC * NZF), tt = t - le * (NPC * NZF);
      const int i = tt % NPC, c = tt / NPC;
      T x[NP];
#pragma unroll
      for (int a = 0; a < NP; ++a) x[a] = b1[le * B1 + (c * NP + a) * NPC + i];
      if (DIM == 2) {
        if (e0 + le < dm.nelem) {
          TIO* dst = fc + (e0 + le) * B2 + i;
          fold_restrict<T, NP, NPC>(J, x, [&](int o, T v) { dst[o * NPC] = TIO(v); });
        }
      } else {
        T* dst = b2 + le * B2 + c * NPC * NPC + i;
        fold_restrict<T, NP, NPC>(J, x, [&](int o, T v) { dst[o * NPC] = v; });
      }
    }
    if (DIM == 3) {
      __syncthreads();
      constexpr int NC3 = NPC * NPC * NPC;
      #pragma unroll 1
      for (int t = tid; t < S::EPB * NPC * NPC; t += blockDim.x) {   // z: lines (x', y')
        const int le = t / (NPC * NPC), ij = t - le * (NPC * NPC);
        T x[NP];
#pragma unroll
        for (int a = 0; a < NP; ++a) x[a] = b2[le * B2 + a * NPC * NPC + ij];
        if (e0 + le < dm.nelem) {
          TIO* dst = fc + (e0 + le) * NC3 + ij;
          fold_restrict<T, NP, NPC>(J, x, [&](int o, T v) { dst[o * NPC * NPC] = TIO(v); });
        }
      }
    }
  }
}

// 3-D elements too large to stage in shared memory (P = 32: 33^3 nodes): one
// launch per axis d and one thread per (element, line).  The partial sums over
// the axes are kept in v between the launches (the same additions, in the same
// order, as the staged kernel's accumulator); the launch of the last axis applies
// the masses and forms v = A u or f - A u.
template <typename T, int NP, bool RESIDUAL, typename TIO>
// CTAs per SM: fp32 5 (96 registers), 8-byte types 3 (the double-float line needs 214 registers uncapped)
__global__ void __launch_bounds__(128, sizeof(T) == 4 ? 5 : 3)
apply_axis_kernel(LevelDims dm, ApplyTables<T> at, const TIO* __restrict__ u,
                  const TIO* __restrict__ f, TIO* __restrict__ v, int d, const int* __restrict__ unz) {
  constexpr int LINES = NP * NP, NODES = NP * NP * NP;
  const long long gid = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (gid >= dm.nelem * LINES) return;
  const long long e = gid / LINES;
  const int line = (int)(gid - e * LINES);
  if (unz && __ldg(unz) == 0) {
    // u identically zero: v = f (or 0), written by the last axis's launch, line by line
    if (d == 2) {
#pragma unroll 1
      for (int i = 0; i < NP; ++i) {
        const long long g = e * NODES + line + (long long)i * NP * NP;
        v[g] = RESIDUAL ? f[g] : TIO(0);
      }
    }
    return;
  }
  const int me[3] = {(int)(e % dm.ne[0]), (int)((e / dm.ne[0]) % dm.ne[1]),
                     (int)(e / ((long long)dm.ne[0] * dm.ne[1]))};
  int off, stride;
  if (d == 0) { off = line * NP; stride = 1; }
  else if (d == 1) { off = (line / NP) * NP * NP + line % NP; stride = NP; }
  else { off = line; stride = NP * NP; }
  const TIO* ue = u + e * NODES;
  TIO* ve = v + e * NODES;
  T x[NP], y[NP];
#pragma unroll
  for (int a = 0; a < NP; ++a) x[a] = T(ue[off + a * stride]);
  apply_line<T, NP, NODES, TIO>(at, apply_axis(dm, at, me, d), u, e, off, stride, x, y);
  if (d == 0) {
#pragma unroll
    for (int i = 0; i < NP; ++i) ve[off + i * stride] = TIO(y[i]);
  } else if (d == 1) {
#pragma unroll
    for (int i = 0; i < NP; ++i) ve[off + i * stride] = TIO(T(ve[off + i * stride]) + y[i]);
  } else {
#pragma unroll 1
    for (int i = 0; i < NP; ++i) {
      const int nd = off + i * stride;
      const int ii = nd % NP, jj = (nd / NP) % NP, kk = nd / (NP * NP);
      T m = ldg(at.M[0] + (size_t)me[0] * NP + ii) * ldg(at.M[1] + (size_t)me[1] * NP + jj);
      m = m * ldg(at.M[2] + (size_t)me[2] * NP + kk);
      const T val = m * (T(ve[nd]) + y[i]);
      ve[nd] = RESIDUAL ? TIO(T(f[e * NODES + nd]) - val) : TIO(val);
    }
  }
}

template <typename T, int NP, typename TIO>
static int apply_dispatch_axes(const LevelDims& dm, const ApplyTables<T>& at, const TIO* u, const TIO* f,
                               TIO* v, cudaStream_t s, const int* unz = nullptr) {
  const long long threads = dm.nelem * NP * NP;
  const long long blocks = (threads + 127) / 128;
  for (int d = 0; d < 3; ++d) {
    count_launch();
    if (f) apply_axis_kernel<T, NP, true, TIO><<<(unsigned)blocks, 128, 0, s>>>(dm, at, u, f, v, d, unz);
    else apply_axis_kernel<T, NP, false, TIO><<<(unsigned)blocks, 128, 0, s>>>(dm, at, u, f, v, d, unz);
  }
  return cudaGetLastError() == cudaSuccess ? PMG_OK : PMG_ECUDA;
}

template <typename T, int DIM, int NP, typename TIO = T>
static int apply_dispatch(const LevelDims& dm, const ApplyTables<T>& at, const TIO* u, const TIO* f,
                          TIO* v, cudaStream_t s, const int* unz = nullptr) {
  using S = ApplyShape<DIM, NP>;
  long long blocks = (dm.nelem + S::EPB - 1) / S::EPB;
  const size_t smem = 2 * sizeof(T) * S::EPB * S::NODES;
  if (f) {
    if (!set_smem(apply_kernel<T, DIM, NP, true, TIO>, smem)) return PMG_ECUDA;
    count_launch();
    apply_kernel<T, DIM, NP, true, TIO><<<(unsigned)blocks, S::THREADS, smem, s>>>(
        dm, at, u, f, v, FoldedJ<T, NP, 0>{}, nullptr, unz);
  } else {
    if (!set_smem(apply_kernel<T, DIM, NP, false, TIO>, smem)) return PMG_ECUDA;
    count_launch();
    apply_kernel<T, DIM, NP, false, TIO><<<(unsigned)blocks, S::THREADS, smem, s>>>(
        dm, at, u, f, v, FoldedJ<T, NP, 0>{}, nullptr, unz);
  }
  return cudaGetLastError() == cudaSuccess ? PMG_OK : PMG_ECUDA;
}

// v-less residual + restriction: fc = I^T (f - A u) for the staged kernel's shapes;
// PMG_EINVAL where no fused kernel exists (the caller then runs the two kernels).
template <typename T, int DIM, int NP, int NPC>
static int residual_restrict_dispatch(const LevelDims& dm, const ApplyTables<T>& at, const T* u, const T* f,
                                      const double* Jh, T* fc, cudaStream_t s) {
  const FoldedJ<T, NP, NPC> J = fold_interpolation<T, NP, NPC>(Jh);
  using S = ApplyShape<DIM, NP>;
  long long blocks = (dm.nelem + S::EPB - 1) / S::EPB;
  const size_t smem = 2 * sizeof(T) * S::EPB * S::NODES;
  if (!set_smem(apply_kernel<T, DIM, NP, true, T, NPC>, smem)) return PMG_ECUDA;
  count_launch();
  apply_kernel<T, DIM, NP, true, T, NPC><<<(unsigned)blocks, S::THREADS, smem, s>>>(dm, at, u, f, nullptr, J, fc);
  return cudaGetLastError() == cudaSuccess ? PMG_OK : PMG_ECUDA;
}

}  // namespace pmg
