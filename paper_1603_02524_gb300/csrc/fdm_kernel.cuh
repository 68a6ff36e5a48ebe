// Weighted additive Schwarz patch solve by fast diagonalisation (Sec. 3.1).
//
// One CTA per subdomain.  The kernel serves both the element-centred (EA) and
// the face-centred (FA) families: every patch is a tensor product of three
// contiguous global 1-D index ranges (one per axis, wrapped on periodic axes,
// truncated at Dirichlet walls), and every axis carries its own eigen-table of
// L_{s,d} S = M_{s,d} S Lambda:
//
//   gather   r_s = R_s r                          (0 outside the domain)
//   forward  t = (S_c^T (x) S_b^T (x) S_a^T) r_s   three in-place line passes
//   scale    t /= lambda_a + lambda_b + lambda_c
//   backward t = (W_c (x) W_b (x) W_a) t,  W_q = diag(w_q) S_q (omega folded into W_a)
//   scatter  u += t                               (atomic: patches overlap)
//
// Positions outside the domain carry a decoupled identity in the eigen-table
// and weight 0, so the tensor algebra needs no special cases.
//
// Even-odd split: when the 1-D patch problem of an axis is centro-symmetric
// (every interior patch of a uniform grid), its eigenvectors are symmetric or
// antisymmetric.  The host then stores them folded (symmetric modes first), and
// a line pass works on the half-sums v_a + v_{n-1-a} and half-differences
// v_a - v_{n-1-a}, which roughly halves the multiply-adds of that pass.
#pragma once

#include "pmg_internal.h"

namespace pmg {

constexpr long long kInvalidOffset = -(1LL << 60);

// 16-byte vector of T (shared-memory table rows are padded to a multiple of it).
template <typename T> struct Vec16;
template <> struct Vec16<float> {
  using type = float4;
  static constexpr int W = 4;
  __device__ static float get(const float4& v, int k) { return k == 0 ? v.x : k == 1 ? v.y : k == 2 ? v.z : v.w; }
};
template <> struct Vec16<double> {
  using type = double2;
  static constexpr int W = 2;
  __device__ static double get(const double2& v, int k) { return k == 0 ? v.x : v.y; }
};
template <typename T>
__host__ __device__ constexpr int padded(int n) { return (n + Vec16<T>::W - 1) / Vec16<T>::W * Vec16<T>::W; }

// acc[0..N) += row[0..N) * x, row 16-byte aligned and padded.
template <typename T, int N>
__device__ __forceinline__ void axpy_row(T* acc, const T* row, T x) {
  using V = Vec16<T>;
  const typename V::type* r = reinterpret_cast<const typename V::type*>(row);
#pragma unroll
  for (int c = 0; c < padded<T>(N) / V::W; ++c) {
    const typename V::type s = r[c];
#pragma unroll
    for (int k = 0; k < V::W; ++k)
      if (c * V::W + k < N) acc[c * V::W + k] = fma(V::get(s, k), x, acc[c * V::W + k]);
  }
}

// Transform of one line held in registers.  General form: out_i = sum_a M[a][i] v_a,
// M row-major with padded rows (forward: M = S, node-major; backward: M = W^T,
// mode-major, so the same form applies W), all N partial sums in registers (long
// lines, N > 32, use dot products instead).  Even-odd form on a centro-symmetric
// axis: M holds the symmetric block (NE rows, padded) then the antisymmetric block
// (NO rows, padded), NE = N - N/2, NO = N/2; forward: rows = nodes 0..NE-1 / 0..NO-1
// of S, output modes symmetric first (positions 0..NE-1) then antisymmetric;
// backward: rows = modes of W^T, output nodes.
template <typename T, int N, bool FORWARD>
__device__ __forceinline__ void line_transform(bool sym, const T* M, const T (&v)[N], T (&out)[N]) {
  constexpr int NP_ = padded<T>(N);
  if (N > 1 && N <= 32 && sym) {
    constexpr int H = N / 2, NE = N - H, NO = H;
    constexpr int PE = padded<T>(NE), PO = padded<T>(NO > 0 ? NO : 1);
    const T* Me = M;
    const T* Mo = M + NE * PE;
    T ae[NE], ao[NO > 0 ? NO : 1];
#pragma unroll
    for (int i = 0; i < NE; ++i) ae[i] = T(0);
#pragma unroll
    for (int i = 0; i < NO; ++i) ao[i] = T(0);
    if (FORWARD) {
#pragma unroll
      for (int a = 0; a < H; ++a) {
        axpy_row<T, NE>(ae, Me + a * PE, v[a] + v[N - 1 - a]);
        axpy_row<T, NO>(ao, Mo + a * PO, v[a] - v[N - 1 - a]);
      }
      if (NE > H) axpy_row<T, NE>(ae, Me + H * PE, v[H]);
#pragma unroll
      for (int i = 0; i < NE; ++i) out[i] = ae[i];
#pragma unroll
      for (int i = 0; i < NO; ++i) out[NE + i] = ao[i];
    } else {
#pragma unroll
      for (int i = 0; i < NE; ++i) axpy_row<T, NE>(ae, Me + i * PE, v[i]);
#pragma unroll
      for (int i = 0; i < NO; ++i) axpy_row<T, NO>(ao, Mo + i * PO, v[NE + i]);
#pragma unroll
      for (int a = 0; a < H; ++a) {
        out[a] = ae[a] + ao[a];
        out[N - 1 - a] = ae[a] - ao[a];
      }
      if (NE > H) out[H] = ae[H];
    }
  } else if constexpr (N <= 32) {
#pragma unroll
    for (int i = 0; i < N; ++i) out[i] = T(0);
#pragma unroll
    for (int a = 0; a < N; ++a) axpy_row<T, N>(out, M + a * NP_, v[a]);
  } else {
#pragma unroll 1
    for (int i = 0; i < N; ++i) {
      T s = T(0);
#pragma unroll
      for (int a = 0; a < N; ++a) s = fma(M[a * NP_ + i], v[a], s);
      out[i] = s;
    }
  }
}

// 1 / s: hardware single-precision approximate reciprocal (rcp.approx, relative
// error about 2^-23); in double refined by Newton's iteration x <- x + x (1 - s x),
// each step squaring the relative error (2^-22 -> 2^-44 -> below double rounding).
// The double <-> float moves are bit-level (dfloat.cuh): on GB300 a cvt between
// double and float costs as much as an FP64 multiply-add.
__device__ __forceinline__ float rcp_approx(float s) {
  float r;
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(s));
  return r;
}
__device__ __forceinline__ double recip(double s) {
  double x = widen(rcp_approx(split_double(s).hi));
  double e = fma(-s, x, 1.0);
  x = fma(x, e, x);
  e = fma(-s, x, 1.0);
  return fma(x, e, x);
}
__device__ __forceinline__ float recip(float s) { return rcp_approx(s); }

// One in-place pass over all lines of an axis: line l starts at
// (l % lo_count) * lo_stride + (l / lo_count) * hi_stride, nodes `stride` apart.
// SCALE (the last forward pass): output i of line l is multiplied by
// 1 / (lsum(l) + lq[i]), the inverse eigenvalue sum of the fast diagonalisation.
// SCALE = 2: the inverse eigenvalue sums come from a table (lq + lsum(l) + i * istride).
template <typename T, int N, bool FORWARD, int SCALE = 0, typename LS = int>
__device__ __forceinline__ void axis_pass(bool sym, T* buf, const T* M, int nlines, int lo_stride,
                                          int lo_count, int hi_stride, int stride,
                                          const T* lq = nullptr, LS lsum = LS(), int istride = 0) {
  if constexpr (N > 32) {
    // Long lines (P = 32 patches, 43 and 64 nodes): all N inputs in registers, the
    // outputs in chunks of CH = 8 accumulated from 16-byte segments of the table rows (a
    // quarter or half as many shared-memory loads as multiply-adds) and stored at once;
    // in place, since the whole line is read first.  The vector reads stay inside a
    // row's padding (NP_ is a multiple of the vector width).
    using V = Vec16<T>;
    constexpr int NP_ = padded<T>(N);
    constexpr int CH = 8;
    constexpr int H = N / 2, NE = N - H, NO = H;
    constexpr int PE = padded<T>(NE), PO = padded<T>(NO);
    for (int l = threadIdx.x; l < nlines; l += blockDim.x) {
      const int base = (l % lo_count) * lo_stride + (l / lo_count) * hi_stride;
      T v[N];
#pragma unroll
      for (int a = 0; a < N; ++a) v[a] = buf[base + a * stride];
      T s0 = T(0);
      const T* tb = nullptr;
      if constexpr (SCALE == 1) s0 = lsum(l);
      if constexpr (SCALE == 2) tb = lq + lsum(l);
      auto put = [&](int i, T o) {
        if constexpr (SCALE == 1) o *= recip(s0 + lq[i]);
        if constexpr (SCALE == 2) o *= __ldg(tb + i * istride);
        buf[base + i * stride] = o;
      };
      if (sym) {
        // centro-symmetric line, tables in even-odd form (the symmetric block of NE
        // rows, then the antisymmetric block of NO rows); halves of at most 32 values
        const T* Me = M;
        const T* Mo = M + NE * PE;
        if (FORWARD) {
          // half-sums and half-differences of the nodes, modes out symmetric first
#pragma unroll
          for (int a = 0; a < H; ++a) {
            const T p = v[a] + v[N - 1 - a], m = v[a] - v[N - 1 - a];
            v[a] = p;
            v[N - 1 - a] = m;
          }
#pragma unroll 1
          for (int i0 = 0; i0 < N; i0 += CH) {
            // chunk of symmetric (i < NE) or antisymmetric (i >= NE) modes
            const bool even = i0 < NE;
            const int j0 = even ? i0 : i0 - NE;
            T acc[CH];
#pragma unroll
            for (int k = 0; k < CH; ++k) acc[k] = T(0);
            if (even) {
#pragma unroll
              for (int a = 0; a < NE; ++a) {
                const typename V::type* row = reinterpret_cast<const typename V::type*>(Me + a * PE + j0);
#pragma unroll
                for (int c = 0; c < CH / V::W; ++c)
                  if (j0 + c * V::W < NE) {
                    const typename V::type w = row[c];
#pragma unroll
                    for (int k = 0; k < V::W; ++k) acc[c * V::W + k] = fma(V::get(w, k), v[a], acc[c * V::W + k]);
                  }
              }
            } else {
#pragma unroll
              for (int a = 0; a < NO; ++a) {
                const typename V::type* row = reinterpret_cast<const typename V::type*>(Mo + a * PO + j0);
#pragma unroll
                for (int c = 0; c < CH / V::W; ++c)
                  if (j0 + c * V::W < NO) {
                    const typename V::type w = row[c];
#pragma unroll
                    for (int k = 0; k < V::W; ++k)
                      acc[c * V::W + k] = fma(V::get(w, k), v[N - 1 - a], acc[c * V::W + k]);
                  }
              }
            }
            const int nn = even ? NE : NO;
#pragma unroll
            for (int k = 0; k < CH; ++k)
              if (j0 + k < nn) put((even ? 0 : NE) + j0 + k, acc[k]);
            if (even && i0 + CH >= NE) i0 = NE - CH;    // the next chunk starts the odd modes
          }
        } else {
          // modes in (symmetric 0..NE-1, antisymmetric NE..N-1), nodes out a and N-1-a
#pragma unroll 1
          for (int a0 = 0; a0 < NE; a0 += CH) {
            T ae[CH], ao[CH];
#pragma unroll
            for (int k = 0; k < CH; ++k) ae[k] = ao[k] = T(0);
#pragma unroll
            for (int i = 0; i < NE; ++i) {
              const typename V::type* row = reinterpret_cast<const typename V::type*>(Me + i * PE + a0);
#pragma unroll
              for (int c = 0; c < CH / V::W; ++c)
                if (a0 + c * V::W < NE) {
                  const typename V::type w = row[c];
#pragma unroll
                  for (int k = 0; k < V::W; ++k) ae[c * V::W + k] = fma(V::get(w, k), v[i], ae[c * V::W + k]);
                }
            }
#pragma unroll
            for (int i = 0; i < NO; ++i) {
              const typename V::type* row = reinterpret_cast<const typename V::type*>(Mo + i * PO + a0);
#pragma unroll
              for (int c = 0; c < CH / V::W; ++c)
                if (a0 + c * V::W < NO) {
                  const typename V::type w = row[c];
#pragma unroll
                  for (int k = 0; k < V::W; ++k) ao[c * V::W + k] = fma(V::get(w, k), v[NE + i], ao[c * V::W + k]);
                }
            }
#pragma unroll
            for (int k = 0; k < CH; ++k) {
              const int a = a0 + k;
              if (a < H) {
                put(a, ae[k] + ao[k]);
                put(N - 1 - a, ae[k] - ao[k]);
              } else if (a < NE) {
                put(a, ae[k]);                       // the middle node (odd N)
              }
            }
          }
        }
        continue;
      }
#pragma unroll 1
      for (int i0 = 0; i0 < N; i0 += CH) {
        T acc[CH];
#pragma unroll
        for (int k = 0; k < CH; ++k) acc[k] = T(0);
#pragma unroll
        for (int a = 0; a < N; ++a) {
          const typename V::type* row = reinterpret_cast<const typename V::type*>(M + a * NP_ + i0);
#pragma unroll
          for (int c = 0; c < CH / V::W; ++c) {
            if (i0 + c * V::W < N) {
              const typename V::type w = row[c];
#pragma unroll
              for (int k = 0; k < V::W; ++k) acc[c * V::W + k] = fma(V::get(w, k), v[a], acc[c * V::W + k]);
            }
          }
        }
#pragma unroll
        for (int k = 0; k < CH; ++k)
          if (i0 + k < N) put(i0 + k, acc[k]);
      }
    }
    return;
  }
  for (int l = threadIdx.x; l < nlines; l += blockDim.x) {
    const int base = (l % lo_count) * lo_stride + (l / lo_count) * hi_stride;
    T v[N], out[N];
#pragma unroll
    for (int a = 0; a < N; ++a) v[a] = buf[base + a * stride];
    line_transform<T, N, FORWARD>(sym, M, v, out);
    if constexpr (SCALE == 1) {
      const T s0 = lsum(l);
#pragma unroll
      for (int i = 0; i < N; ++i) out[i] *= recip(s0 + lq[i]);
    } else if constexpr (SCALE == 2) {
      const T* tb = lq + lsum(l);
#pragma unroll
      for (int i = 0; i < N; ++i) out[i] *= __ldg(tb + i * istride);
    }
#pragma unroll
    for (int i = 0; i < N; ++i) buf[base + i * stride] = out[i];
  }
}

// Copy an n x n table (general, row-major) or its even-odd folded blocks from
// global memory into padded shared-memory rows.
template <typename T, int N>
__device__ __forceinline__ void load_table(T* dst, const T* src, bool sym) {
  constexpr int NP_ = padded<T>(N);
  constexpr int H = N / 2, NE = N - H, NO = H;
  constexpr int PE = padded<T>(NE), PO = padded<T>(NO > 0 ? NO : 1);
  if (sym && N > 1 && N <= 64) {
    for (int t = threadIdx.x; t < NE * NE; t += blockDim.x) dst[(t / NE) * PE + t % NE] = src[t];
    for (int t = threadIdx.x; t < NO * NO; t += blockDim.x)
      dst[NE * PE + (t / NO) * PO + t % NO] = src[NE * NE + t];
  } else {
    for (int t = threadIdx.x; t < N * N; t += blockDim.x) dst[(t / N) * NP_ + t % N] = src[t];
  }
}

// ---------------------------------------------------------------------------
// Tensor-core line passes (fp32 data): out[line][n] = sum_k in[line][k] M[k][n]
// as 16 x 8 x 8 tf32 MMAs with fp32 accumulation.  Each operand is split as
// x = hi + lo with hi, lo tf32 and the product taken as hi*hi + hi*lo + lo*hi
// (3xTF32), which keeps fp32-level accuracy.  M is the zero-padded table in
// shared memory (P8 x P8, P8 = N rounded up to 8).  A warp owns 16 lines at a
// time; it reads all N inputs of its lines before writing any output, so the
// pass is in place.
// ---------------------------------------------------------------------------
__device__ __forceinline__ unsigned to_tf32(float x) {
  unsigned r;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
  return r;
}

__device__ __forceinline__ void mma_tf32(float (&d)[4], const unsigned (&a)[4], unsigned b0, unsigned b1) {
  asm volatile(
      "mma.sync.aligned.m16n8k8.row.col.f32.tf32.tf32.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
      "{%0,%1,%2,%3};"
      : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

template <int N>
__device__ __forceinline__ void line_pass_mma(float* buf, const float* M, int nlines, int lo_stride,
                                              int lo_count, int hi_stride, int stride, bool split3) {
  constexpr int P8 = (N + 7) / 8 * 8, KT = P8 / 8, NT = P8 / 8;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
  const int g = lane >> 2, t = lane & 3;
  // B fragments of the whole table (b0: row k = 8 kt + t, b1: row k + 4; column n = 8 nt + g)
  unsigned bh[KT][NT][2], bl[KT][NT][2];
#pragma unroll
  for (int kt = 0; kt < KT; ++kt)
#pragma unroll
    for (int nt = 0; nt < NT; ++nt)
#pragma unroll
      for (int j = 0; j < 2; ++j) {
        const float b = M[(kt * 8 + t + 4 * j) * P8 + nt * 8 + g];
        bh[kt][nt][j] = to_tf32(b);
        bl[kt][nt][j] = split3 ? to_tf32(b - __uint_as_float(bh[kt][nt][j])) : 0u;
      }
  const int mtiles = (nlines + 15) / 16;
  for (int mt = warp; mt < mtiles; mt += nwarps) {
    const int l0 = mt * 16 + g, l1 = l0 + 8;
    const bool v0 = l0 < nlines, v1 = l1 < nlines;
    const int b0 = v0 ? (l0 % lo_count) * lo_stride + (l0 / lo_count) * hi_stride : 0;
    const int b1 = v1 ? (l1 % lo_count) * lo_stride + (l1 / lo_count) * hi_stride : 0;
    float acc[NT][4];
#pragma unroll
    for (int nt = 0; nt < NT; ++nt) acc[nt][0] = acc[nt][1] = acc[nt][2] = acc[nt][3] = 0.0f;
#pragma unroll
    for (int kt = 0; kt < KT; ++kt) {
      const int k0 = kt * 8 + t, k1 = k0 + 4;
      // A fragment: (row g, col t), (row g+8, col t), (row g, col t+4), (row g+8, col t+4)
      const float x[4] = {(v0 && k0 < N) ? buf[b0 + k0 * stride] : 0.0f,
                          (v1 && k0 < N) ? buf[b1 + k0 * stride] : 0.0f,
                          (v0 && k1 < N) ? buf[b0 + k1 * stride] : 0.0f,
                          (v1 && k1 < N) ? buf[b1 + k1 * stride] : 0.0f};
      unsigned ah[4], al[4];
#pragma unroll
      for (int i = 0; i < 4; ++i) {
        ah[i] = to_tf32(x[i]);
        al[i] = split3 ? to_tf32(x[i] - __uint_as_float(ah[i])) : 0u;
      }
      if (split3) {
#pragma unroll
        for (int nt = 0; nt < NT; ++nt) {
          mma_tf32(acc[nt], al, bh[kt][nt][0], bh[kt][nt][1]);
          mma_tf32(acc[nt], ah, bl[kt][nt][0], bl[kt][nt][1]);
          mma_tf32(acc[nt], ah, bh[kt][nt][0], bh[kt][nt][1]);
        }
      } else {
#pragma unroll
        for (int nt = 0; nt < NT; ++nt) mma_tf32(acc[nt], ah, bh[kt][nt][0], bh[kt][nt][1]);
      }
    }
    __syncwarp();
    // C fragment: (row g, cols 2t, 2t+1), (row g+8, cols 2t, 2t+1)
#pragma unroll
    for (int nt = 0; nt < NT; ++nt) {
      const int n0 = nt * 8 + 2 * t;
      if (v0 && n0 < N) buf[b0 + n0 * stride] = acc[nt][0];
      if (v0 && n0 + 1 < N) buf[b0 + (n0 + 1) * stride] = acc[nt][1];
      if (v1 && n0 < N) buf[b1 + n0 * stride] = acc[nt][2];
      if (v1 && n0 + 1 < N) buf[b1 + (n0 + 1) * stride] = acc[nt][3];
    }
    __syncwarp();
  }
}

// Zero-padded P8 x P8 copy of an n x n table for the tensor-core passes.
template <int N>
__device__ __forceinline__ void load_table_mma(float* dst, const float* src) {
  constexpr int P8 = (N + 7) / 8 * 8;
  for (int t = threadIdx.x; t < P8 * P8; t += blockDim.x) {
    const int r = t / P8, c = t % P8;
    dst[t] = (r < N && c < N) ? src[r * N + c] : 0.0f;
  }
}

template <typename T, bool TC>
__host__ __device__ constexpr int table_floats(int n) {
  return TC ? (n + 7) / 8 * 8 * ((n + 7) / 8 * 8) : n * padded<T>(n);
}



// Default CTA size: enough threads for the widest line pass (one line per
// thread), rounded to whole warps, at most 256.
template <int NA, int NB, int NC>
constexpr int fdm_threads() {
  constexpr int l0 = NB * NC, l1 = NA * NC, l2 = NA * NB;
  constexpr int m = l0 > l1 ? (l0 > l2 ? l0 : l2) : (l1 > l2 ? l1 : l2);
  constexpr int t = (m + 31) / 32 * 32;
  return t < 256 ? t : 256;
}

// One line pass along an axis: tensor cores (fp32, TC) or SIMT (general / even-odd).
template <typename T, int N, bool FORWARD, bool TC>
__device__ __forceinline__ void pass(bool sym, T* buf, const T* M, int nlines, int lo_stride, int lo_count,
                                     int hi_stride, int stride, bool split3 = true) {
  if constexpr (TC) {
    line_pass_mma<N>(buf, M, nlines, lo_stride, lo_count, hi_stride, stride, split3);
  } else {
    axis_pass<T, N, FORWARD>(sym, buf, M, nlines, lo_stride, lo_count, hi_stride, stride);
  }
}

template <typename T, int N, bool TC>
__device__ __forceinline__ void tload(T* dst, const T* src, bool sym) {
  if constexpr (TC) load_table_mma<N>(dst, src);
  else load_table<T, N>(dst, src, sym);
}

// The patch solve proper on a staged patch: three forward line passes (the last
// one scaled by the inverse eigenvalue sums), three backward passes, and the
// weighted corrections added to u (atomically: patches overlap).
template <typename T, int NA, int NB, int NC, bool TC>
__device__ __forceinline__ void patch_compute(T* buf, T* const (&Sq)[3], T* const (&Wq)[3], const T* la,
                                              const T* lb, const T* lc, const bool (&sym)[3],
                                              const long long* off, const long long* rowoff,
                                              T* __restrict__ u, bool split3 = true,
                                              const T* invp = nullptr) {
  constexpr int NN = NA * NB * NC;
  // forward transforms, then the scaling by 1 / (lambda_a + lambda_b + lambda_c)
  // (SIMT: folded into the last forward pass)
  pass<T, NA, true, TC>(sym[0], buf, Sq[0], NB * NC, NA, NB * NC, 0, 1, split3);
  __syncthreads();
  if constexpr (TC) {
    pass<T, NB, true, TC>(sym[1], buf, Sq[1], NA * NC, 1, NA, NA * NB, NA, split3);
    __syncthreads();
    if (NC > 1) {
      pass<T, NC, true, TC>(sym[2], buf, Sq[2], NA * NB, 1, NA * NB, 0, NA * NB, split3);
      __syncthreads();
    }
    for (int t = threadIdx.x; t < NN; t += blockDim.x) {
      const int a = t % NA, b = (t / NA) % NB, c = t / (NA * NB);
      buf[t] *= recip(la[a] + lb[b] + lc[c]);
    }
  } else if constexpr (NC > 1) {
    axis_pass<T, NB, true>(sym[1], buf, Sq[1], NA * NC, 1, NA, NA * NB, NA);
    __syncthreads();
    // line l = (a, b) = (l % NA, l / NA), outputs along c
    if (invp)
      axis_pass<T, NC, true, 2>(sym[2], buf, Sq[2], NA * NB, 1, NA * NB, 0, NA * NB, invp,
                                [](int l) { return l; }, NA * NB);
    else
      axis_pass<T, NC, true, 1>(sym[2], buf, Sq[2], NA * NB, 1, NA * NB, 0, NA * NB, lc,
                                [&](int l) { return la[l % NA] + lb[l / NA]; });
  } else {
    // 2-D: line l = (a, c) = (l % NA, l / NA), outputs along b
    if (invp)
      axis_pass<T, NB, true, 2>(sym[1], buf, Sq[1], NA * NC, 1, NA, NA * NB, NA, invp,
                                [](int l) { return l % NA + (l / NA) * NA * NB; }, NA);
    else
      axis_pass<T, NB, true, 1>(sym[1], buf, Sq[1], NA * NC, 1, NA, NA * NB, NA, lb,
                                [&](int l) { return la[l % NA] + lc[l / NA]; });
  }
  __syncthreads();
  if (NC > 1) {
    pass<T, NC, false, TC>(sym[2], buf, Wq[2], NA * NB, 1, NA * NB, 0, NA * NB, split3);
    __syncthreads();
  }
  pass<T, NB, false, TC>(sym[1], buf, Wq[1], NA * NC, 1, NA, NA * NB, NA, split3);
  __syncthreads();
  pass<T, NA, false, TC>(sym[0], buf, Wq[0], NB * NC, NA, NB * NC, 0, 1, split3);
  __syncthreads();

  for (int t = threadIdx.x; t < NN; t += blockDim.x) {
    const int row = t / NA, a = t - row * NA;
    const long long o = off[a] + rowoff[row];
    if (o >= 0) atomicAdd(u + o, buf[t]);
  }
}

// Largest CTA of a shape: kFdmMaxThreads (registers capped at 128 per thread), or
// 256 for FP64 patches with 32-node axes, whose lines need more registers.
template <typename T, int NA, int NB, int NC>
constexpr int fdm_max_threads() {
  return (sizeof(T) == 8 && (NA >= 32 || NB >= 32 || NC >= 32)) ? 256 : kFdmMaxThreads;
}

template <typename T, int NA, int NB, int NC, bool TC>
__global__ void __launch_bounds__(fdm_max_threads<T, NA, NB, NC>())
fdm_kernel(LevelDims dm, FdmFamily<T> fam, const T* __restrict__ r, T* __restrict__ u) {
  static_assert(!TC || (sizeof(T) == 4 && NA <= 32 && NB <= 32 && NC <= 32 && NC > 1),
                "tensor-core passes: fp32, 3-D, at most 32 nodes per axis");
  constexpr int NN = NA * NB * NC;
  extern __shared__ __align__(16) unsigned char fdm_smem[];
  long long* off = reinterpret_cast<long long*>(fdm_smem);        // NA + NB + NC
  long long* rowoff = off + (NA + NB + NC + 1) / 2 * 2;             // NB * NC row offsets
  T* buf = reinterpret_cast<T*>(rowoff + (NB * NC + 1) / 2 * 2);
  T* Sq[3];
  T* Wq[3];
  Sq[0] = buf + padded<T>(NN);
  Wq[0] = Sq[0] + table_floats<T, TC>(NA);
  Sq[1] = Wq[0] + table_floats<T, TC>(NA);
  Wq[1] = Sq[1] + table_floats<T, TC>(NB);
  Sq[2] = Wq[1] + table_floats<T, TC>(NB);
  Wq[2] = Sq[2] + table_floats<T, TC>(NC);
  T* la = Wq[2] + table_floats<T, TC>(NC);
  T* lb = la + NA;
  T* lc = lb + NB;

  const int ca = fam.ax[0].count, cb = fam.ax[1].count;
  const int pid = blockIdx.x;
  const int pidx[3] = {pid % ca, (pid / ca) % cb, pid / (ca * cb)};
  const int nq[3] = {NA, NB, NC};
  T* lq[3] = {la, lb, lc};
  bool sym[3];
  const long long nodes_el = (long long)dm.NP * dm.NP * dm.NPz;
  const long long estride[3] = {nodes_el, nodes_el * dm.ne[0], nodes_el * dm.ne[0] * dm.ne[1]};
  const long long nstride[3] = {1, dm.NP, (long long)dm.NP * dm.NP};
  long long* offq[3] = {off, off + NA, off + NA + NB};

#pragma unroll
  for (int q = 0; q < 3; ++q) {
    const FdmAxis<T>& ax = fam.ax[q];
    const int n = nq[q];
    const size_t p = pidx[q];
    sym[q] = ax.sym[p] != 0;
    if (q == 0) {
      tload<T, NA, TC>(Sq[0], ax.S + p * n * n, sym[0]);
      tload<T, NA, TC>(Wq[0], ax.W + p * n * n, sym[0]);
    } else if (q == 1) {
      tload<T, NB, TC>(Sq[1], ax.S + p * n * n, sym[1]);
      tload<T, NB, TC>(Wq[1], ax.W + p * n * n, sym[1]);
    } else {
      tload<T, NC, TC>(Sq[2], ax.S + p * n * n, sym[2]);
      tload<T, NC, TC>(Wq[2], ax.W + p * n * n, sym[2]);
    }
    if (threadIdx.x < n) {
      const int a = threadIdx.x;
      lq[q][a] = ax.lam[p * n + a];
      // element-major offset contribution of local index a, or "invalid"
      const int ph = ax.phys;
      const int npp = (ph == 2) ? dm.NPz : dm.NP;
      int G = patch_start(ax, (int)p, npp) + a;
      long long o;
      if (ax.periodic) {
        G %= ax.N;
        if (G < 0) G += ax.N;
        o = (long long)(G / npp) * estride[ph] + (G % npp) * nstride[ph];
      } else if (G < 0 || G >= ax.N) {
        o = kInvalidOffset;
      } else {
        o = (long long)(G / npp) * estride[ph] + (G % npp) * nstride[ph];
      }
      offq[q][a] = o;
    }
  }
  __syncthreads();
  // offset of each row (b, c) of the patch buffer (negative: outside the grid)
  for (int rr = threadIdx.x; rr < NB * NC; rr += blockDim.x)
    rowoff[rr] = off[NA + rr % NB] + off[NA + NB + rr / NB];
  __syncthreads();

  for (int t = threadIdx.x; t < NN; t += blockDim.x) {
    const int row = t / NA, a = t - row * NA;
    const long long o = off[a] + rowoff[row];
    buf[t] = o >= 0 ? r[o] : T(0);
  }
  __syncthreads();

  const T* invp = nullptr;      // precomputed inverse eigenvalue sums of this patch's combination
  if (fam.inv) {
    const int combo = (fam.uid[2][pidx[2]] * fam.ucount[1] + fam.uid[1][pidx[1]]) * fam.ucount[0] +
                      fam.uid[0][pidx[0]];
    invp = fam.inv + (size_t)combo * NN;
  }
  patch_compute<T, NA, NB, NC, TC>(buf, Sq, Wq, la, lb, lc, sym, off, rowoff, u, fam.tc != 2, invp);
}

// ---------------------------------------------------------------------------
// Pipelined form (fp32 SIMT, shapes whose two stages fit twice per SM): a
// persistent CTA walks over patches p, p + gridDim.x, ...; while it computes
// one patch, the gather of the next patch (residual values, eigen-tables,
// eigenvalues) is already in flight as cp.async copies into the other stage,
// so the long-latency loads of one patch overlap the line passes of another.
// ---------------------------------------------------------------------------
template <int BYTES>
__device__ __forceinline__ void cp_async(void* dst, const void* src, bool valid) {
  const unsigned d = (unsigned)__cvta_generic_to_shared(dst);
  asm volatile("cp.async.ca.shared.global [%0], [%1], %2, %3;\n" ::"r"(d), "l"(src), "n"(BYTES),
               "r"(valid ? BYTES : 0)
               : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory"); }

// table copy of load_table as asynchronous element copies (row padding left unset:
// the line passes never read it)
template <typename T, int N>
__device__ __forceinline__ void load_table_async(T* dst, const T* src, bool sym) {
  constexpr int NP_ = padded<T>(N);
  constexpr int H = N / 2, NE = N - H, NO = H;
  constexpr int PE = padded<T>(NE), PO = padded<T>(NO > 0 ? NO : 1);
  if (sym && N > 1 && N <= 64) {
    for (int t = threadIdx.x; t < NE * NE; t += blockDim.x)
      cp_async<sizeof(T)>(dst + (t / NE) * PE + t % NE, src + t, true);
    for (int t = threadIdx.x; t < NO * NO; t += blockDim.x)
      cp_async<sizeof(T)>(dst + NE * PE + (t / NO) * PO + t % NO, src + NE * NE + t, true);
  } else {
    for (int t = threadIdx.x; t < N * N; t += blockDim.x)
      cp_async<sizeof(T)>(dst + (t / N) * NP_ + t % N, src + t, true);
  }
}

// one stage: offsets, row offsets, symmetry flags, patch buffer, six tables, eigenvalues
template <typename T, int NA, int NB, int NC>
struct PipeStage {
  static constexpr int NN = NA * NB * NC;
  static constexpr size_t OFF = 0;
  static constexpr size_t ROW = OFF + 8 * (size_t)((NA + NB + NC + 1) / 2 * 2);
  static constexpr size_t SYM = ROW + 8 * (size_t)((NB * NC + 1) / 2 * 2);
  static constexpr size_t BUF = SYM + 16;
  static constexpr size_t TBL = BUF + sizeof(T) * (size_t)padded<T>(NN);
  static constexpr size_t LAM = TBL + sizeof(T) * 2 * (size_t)(table_floats<T, false>(NA) +
                                                               table_floats<T, false>(NB) +
                                                               table_floats<T, false>(NC));
  static constexpr size_t END = LAM + sizeof(T) * (size_t)((NA + NB + NC + 3) / 4 * 4);
  static constexpr size_t BYTES = (END + 15) / 16 * 16;
};

// The pipelined form exists for fp32 SIMT shapes whose two stages fit one CTA;
// by default it runs where two such CTAs fit an SM, and the autotuner may choose
// either form (FdmFamily::variant).
template <typename T, int NA, int NB, int NC, bool TC>
constexpr bool fdm_pipelined() {
  return !TC && sizeof(T) == 4 && 2 * PipeStage<T, NA, NB, NC>::BYTES <= 226 * 1024;
}
template <typename T, int NA, int NB, int NC>
constexpr bool fdm_pipelined_default() {
  return 2 * PipeStage<T, NA, NB, NC>::BYTES <= 100 * 1024;
}

// Offsets of patch pid (plain stores, then two barriers), then its gather and
// tables as one cp.async group.  Every thread of the CTA calls it.
template <typename T, int NA, int NB, int NC>
__device__ __forceinline__ void pipe_prepare(const LevelDims& dm, const FdmFamily<T>& fam,
                                             const T* __restrict__ r, unsigned char* st, int pid) {
  using PS = PipeStage<T, NA, NB, NC>;
  long long* off = reinterpret_cast<long long*>(st + PS::OFF);
  long long* rowoff = reinterpret_cast<long long*>(st + PS::ROW);
  int* sym = reinterpret_cast<int*>(st + PS::SYM);
  T* buf = reinterpret_cast<T*>(st + PS::BUF);
  T* tb = reinterpret_cast<T*>(st + PS::TBL);
  T* lam = reinterpret_cast<T*>(st + PS::LAM);
  const int ca = fam.ax[0].count, cb = fam.ax[1].count;
  const int pidx[3] = {pid % ca, (pid / ca) % cb, pid / (ca * cb)};
  const int nq[3] = {NA, NB, NC};
  const int base[3] = {0, NA, NA + NB};
  const long long nodes_el = (long long)dm.NP * dm.NP * dm.NPz;
  const long long estride[3] = {nodes_el, nodes_el * dm.ne[0], nodes_el * dm.ne[0] * dm.ne[1]};
  const long long nstride[3] = {1, dm.NP, (long long)dm.NP * dm.NP};
  if (threadIdx.x < 3) sym[threadIdx.x] = fam.ax[threadIdx.x].sym[pidx[threadIdx.x]] != 0;
#pragma unroll
  for (int q = 0; q < 3; ++q) {
    const FdmAxis<T>& ax = fam.ax[q];
    const int n = nq[q];
    if (threadIdx.x < n) {
      const int a = threadIdx.x;
      const size_t p = pidx[q];
      cp_async<sizeof(T)>(lam + base[q] + a, ax.lam + p * n + a, true);
      const int ph = ax.phys;
      const int npp = (ph == 2) ? dm.NPz : dm.NP;
      int G = patch_start(ax, (int)p, npp) + a;
      long long o;
      if (ax.periodic) {
        G %= ax.N;
        if (G < 0) G += ax.N;
        o = (long long)(G / npp) * estride[ph] + (G % npp) * nstride[ph];
      } else if (G < 0 || G >= ax.N) {
        o = kInvalidOffset;
      } else {
        o = (long long)(G / npp) * estride[ph] + (G % npp) * nstride[ph];
      }
      off[base[q] + a] = o;
    }
  }
  __syncthreads();
  for (int rr = threadIdx.x; rr < NB * NC; rr += blockDim.x)
    rowoff[rr] = off[NA + rr % NB] + off[NA + NB + rr / NB];
  __syncthreads();
  for (int t = threadIdx.x; t < PS::NN; t += blockDim.x) {
    const int row = t / NA, a = t - row * NA;
    const long long o = off[a] + rowoff[row];
    cp_async<sizeof(T)>(buf + t, o >= 0 ? r + o : r, o >= 0);
  }
  T* S0 = tb;
  T* W0 = S0 + table_floats<T, false>(NA);
  T* S1 = W0 + table_floats<T, false>(NA);
  T* W1 = S1 + table_floats<T, false>(NB);
  T* S2 = W1 + table_floats<T, false>(NB);
  T* W2 = S2 + table_floats<T, false>(NC);
  {
    const size_t p0 = pidx[0], p1 = pidx[1], p2 = pidx[2];
    load_table_async<T, NA>(S0, fam.ax[0].S + p0 * NA * NA, sym[0]);
    load_table_async<T, NA>(W0, fam.ax[0].W + p0 * NA * NA, sym[0]);
    load_table_async<T, NB>(S1, fam.ax[1].S + p1 * NB * NB, sym[1]);
    load_table_async<T, NB>(W1, fam.ax[1].W + p1 * NB * NB, sym[1]);
    load_table_async<T, NC>(S2, fam.ax[2].S + p2 * NC * NC, sym[2]);
    load_table_async<T, NC>(W2, fam.ax[2].W + p2 * NC * NC, sym[2]);
  }
  cp_async_commit();
}

template <typename T, int NA, int NB, int NC>
__global__ void __launch_bounds__(fdm_max_threads<T, NA, NB, NC>())
fdm_kernel_pipe(LevelDims dm, FdmFamily<T> fam, const T* __restrict__ r, T* __restrict__ u) {
  using PS = PipeStage<T, NA, NB, NC>;
  extern __shared__ __align__(16) unsigned char fdm_smem[];
  const int count = fam.count_total;
  int p = blockIdx.x;
  if (p >= count) return;
  pipe_prepare<T, NA, NB, NC>(dm, fam, r, fdm_smem, p);
  int s = 0;
  for (; p < count; p += gridDim.x) {
    const int pn = p + gridDim.x;
    if (pn < count) pipe_prepare<T, NA, NB, NC>(dm, fam, r, fdm_smem + (s ^ 1) * PS::BYTES, pn);
    else cp_async_commit();
    cp_async_wait<1>();
    __syncthreads();
    unsigned char* st = fdm_smem + s * PS::BYTES;
    T* tb = reinterpret_cast<T*>(st + PS::TBL);
    T* const Sq[3] = {tb, tb + 2 * table_floats<T, false>(NA),
                      tb + 2 * (table_floats<T, false>(NA) + table_floats<T, false>(NB))};
    T* const Wq[3] = {Sq[0] + table_floats<T, false>(NA), Sq[1] + table_floats<T, false>(NB),
                      Sq[2] + table_floats<T, false>(NC)};
    const T* lam = reinterpret_cast<const T*>(st + PS::LAM);
    const int* sy = reinterpret_cast<const int*>(st + PS::SYM);
    const bool sym[3] = {sy[0] != 0, sy[1] != 0, sy[2] != 0};
    patch_compute<T, NA, NB, NC, false>(reinterpret_cast<T*>(st + PS::BUF), Sq, Wq, lam, lam + NA,
                                        lam + NA + NB, sym, reinterpret_cast<const long long*>(st + PS::OFF),
                                        reinterpret_cast<const long long*>(st + PS::ROW), u);
    __syncthreads();
    s ^= 1;
  }
}

// ---------------------------------------------------------------------------
// Patches too large for shared memory (3-D, P = 32: n = 43, and the face patches
// 64 x 43 x 43): persistent CTAs keep their patch buffer in a global scratch
// array (one buffer per CTA, reused patch after patch; it stays in L2 while the
// CTA works on it) and only the offsets, tables and eigenvalues in shared memory.
// ---------------------------------------------------------------------------
template <typename T, int NA, int NB, int NC>
constexpr size_t fdm_gbuf_smem_bytes() {
  return sizeof(long long) * ((NA + NB + NC + 1) / 2 * 2 + (NB * NC + 1) / 2 * 2) +
         sizeof(T) * (2 * (size_t)(table_floats<T, false>(NA) + table_floats<T, false>(NB) +
                                   table_floats<T, false>(NC)) + NA + NB + NC);
}

template <typename T, int NA, int NB, int NC>
__global__ void __launch_bounds__(256)
fdm_kernel_gbuf(LevelDims dm, FdmFamily<T> fam, const T* __restrict__ r, T* __restrict__ u) {
  constexpr int NN = NA * NB * NC;
  extern __shared__ __align__(16) unsigned char fdm_smem[];
  long long* off = reinterpret_cast<long long*>(fdm_smem);
  long long* rowoff = off + (NA + NB + NC + 1) / 2 * 2;
  T* tb = reinterpret_cast<T*>(rowoff + (NB * NC + 1) / 2 * 2);
  T* const Sq[3] = {tb, tb + 2 * table_floats<T, false>(NA),
                    tb + 2 * (table_floats<T, false>(NA) + table_floats<T, false>(NB))};
  T* const Wq[3] = {Sq[0] + table_floats<T, false>(NA), Sq[1] + table_floats<T, false>(NB),
                    Sq[2] + table_floats<T, false>(NC)};
  T* la = Sq[2] + 2 * table_floats<T, false>(NC);
  T* lb = la + NA;
  T* lc = lb + NB;
  T* buf = fam.scratch + (long long)blockIdx.x * fam.scratch_stride;
  const int ca = fam.ax[0].count, cb = fam.ax[1].count;
  const int nq[3] = {NA, NB, NC};
  T* lq[3] = {la, lb, lc};
  long long* offq[3] = {off, off + NA, off + NA + NB};
  const long long nodes_el = (long long)dm.NP * dm.NP * dm.NPz;
  const long long estride[3] = {nodes_el, nodes_el * dm.ne[0], nodes_el * dm.ne[0] * dm.ne[1]};
  const long long nstride[3] = {1, dm.NP, (long long)dm.NP * dm.NP};
  for (int pid = blockIdx.x; pid < fam.count_total; pid += gridDim.x) {
    const int pidx[3] = {pid % ca, (pid / ca) % cb, pid / (ca * cb)};
    bool sym[3];
#pragma unroll
    for (int q = 0; q < 3; ++q) {
      const FdmAxis<T>& ax = fam.ax[q];
      const int n = nq[q];
      const size_t p = pidx[q];
      sym[q] = ax.sym[p] != 0;
      if (q == 0) {
        load_table<T, NA>(Sq[0], ax.S + p * n * n, sym[0]);
        load_table<T, NA>(Wq[0], ax.W + p * n * n, sym[0]);
      } else if (q == 1) {
        load_table<T, NB>(Sq[1], ax.S + p * n * n, sym[1]);
        load_table<T, NB>(Wq[1], ax.W + p * n * n, sym[1]);
      } else {
        load_table<T, NC>(Sq[2], ax.S + p * n * n, sym[2]);
        load_table<T, NC>(Wq[2], ax.W + p * n * n, sym[2]);
      }
      for (int a = threadIdx.x; a < n; a += blockDim.x) {
        lq[q][a] = ax.lam[p * n + a];
        const int ph = ax.phys;
        const int npp = (ph == 2) ? dm.NPz : dm.NP;
        int G = patch_start(ax, (int)p, npp) + a;
        long long o;
        if (ax.periodic) {
          G %= ax.N;
          if (G < 0) G += ax.N;
          o = (long long)(G / npp) * estride[ph] + (G % npp) * nstride[ph];
        } else if (G < 0 || G >= ax.N) {
          o = kInvalidOffset;
        } else {
          o = (long long)(G / npp) * estride[ph] + (G % npp) * nstride[ph];
        }
        offq[q][a] = o;
      }
    }
    __syncthreads();
    for (int rr = threadIdx.x; rr < NB * NC; rr += blockDim.x)
      rowoff[rr] = off[NA + rr % NB] + off[NA + NB + rr / NB];
    __syncthreads();
    for (int t = threadIdx.x; t < NN; t += blockDim.x) {
      const int row = t / NA, a = t - row * NA;
      const long long o = off[a] + rowoff[row];
      buf[t] = o >= 0 ? r[o] : T(0);
    }
    __syncthreads();
    patch_compute<T, NA, NB, NC, false>(buf, Sq, Wq, la, lb, lc, sym, off, rowoff, u);
    __syncthreads();
  }
}

// ---------------------------------------------------------------------------
// The same large patches in slabs: the forward passes along a and b act within each
// c-plane, so they run in shared memory a few planes (a slab of CS) at a time; the
// planes go to the CTA's scratch buffer, the c-lines are transformed there (forward
// with the eigenvalue scaling, then backward), and the backward b and a passes run
// slab by slab in shared memory again before the weighted scatter.  The scratch
// buffer is written once and read once around the c passes instead of around all
// six passes.  Plane rows are padded to NA + 1 values (odd), so that the a-lines of
// consecutive threads fall into distinct shared-memory banks.
// ---------------------------------------------------------------------------
template <typename T, int NA, int NB, int NC>
struct SlabShape {
  static constexpr int NAP = NA % 2 == 0 ? NA + 1 : NA;  // odd row stride
  static constexpr int MAXT = sizeof(T) == 8 ? 256 : 512;  // long lines in registers: 255 / 128 per thread
  static constexpr int PL = NB * NAP;                       // floats of one padded plane
  static constexpr size_t FIXED = sizeof(long long) * ((NA + NB + NC + 1) / 2 * 2 + (NB * NC + 1) / 2 * 2) +
                                  sizeof(T) * (2 * (size_t)(table_floats<T, false>(NA) + table_floats<T, false>(NB) +
                                                            table_floats<T, false>(NC)) + NA + NB + NC);
  static constexpr size_t BUDGET = 227 * 1024;
  static constexpr int CS_FIT = FIXED < BUDGET ? (int)((BUDGET - FIXED) / (sizeof(T) * PL)) : 0;
  static constexpr int CS = CS_FIT > 8 ? 8 : CS_FIT;       // planes per slab
  static constexpr size_t BYTES = FIXED + sizeof(T) * (size_t)CS * PL;
};

template <typename T, int NA, int NB, int NC>
__global__ void __launch_bounds__(SlabShape<T, NA, NB, NC>::MAXT)
fdm_kernel_slab(LevelDims dm, FdmFamily<T> fam, const T* __restrict__ r, T* __restrict__ u) {
  using SS = SlabShape<T, NA, NB, NC>;
  constexpr int NAP = SS::NAP, CS = SS::CS, PL = SS::PL;
  extern __shared__ __align__(16) unsigned char fdm_smem[];
  long long* off = reinterpret_cast<long long*>(fdm_smem);
  long long* rowoff = off + (NA + NB + NC + 1) / 2 * 2;
  T* tb = reinterpret_cast<T*>(rowoff + (NB * NC + 1) / 2 * 2);
  T* const Sq[3] = {tb, tb + 2 * table_floats<T, false>(NA),
                    tb + 2 * (table_floats<T, false>(NA) + table_floats<T, false>(NB))};
  T* const Wq[3] = {Sq[0] + table_floats<T, false>(NA), Sq[1] + table_floats<T, false>(NB),
                    Sq[2] + table_floats<T, false>(NC)};
  T* la = Sq[2] + 2 * table_floats<T, false>(NC);
  T* lb = la + NA;
  T* lc = lb + NB;
  T* sb = lc + NC;                                          // CS padded planes [k][b][a]
  T* buf = fam.scratch + (long long)blockIdx.x * fam.scratch_stride;   // [c][b][a]
  const int ca = fam.ax[0].count, cb = fam.ax[1].count;
  const int nq[3] = {NA, NB, NC};
  T* lq[3] = {la, lb, lc};
  long long* offq[3] = {off, off + NA, off + NA + NB};
  const long long nodes_el = (long long)dm.NP * dm.NP * dm.NPz;
  const long long estride[3] = {nodes_el, nodes_el * dm.ne[0], nodes_el * dm.ne[0] * dm.ne[1]};
  const long long nstride[3] = {1, dm.NP, (long long)dm.NP * dm.NP};
  for (int pid = blockIdx.x; pid < fam.count_total; pid += gridDim.x) {
    const int pidx[3] = {pid % ca, (pid / ca) % cb, pid / (ca * cb)};
    bool sym[3];
#pragma unroll
    for (int q = 0; q < 3; ++q) {
      const FdmAxis<T>& ax = fam.ax[q];
      const int n = nq[q];
      const size_t p = pidx[q];
      sym[q] = ax.sym[p] != 0;
      if (q == 0) {
        load_table<T, NA>(Sq[0], ax.S + p * n * n, sym[0]);
        load_table<T, NA>(Wq[0], ax.W + p * n * n, sym[0]);
      } else if (q == 1) {
        load_table<T, NB>(Sq[1], ax.S + p * n * n, sym[1]);
        load_table<T, NB>(Wq[1], ax.W + p * n * n, sym[1]);
      } else {
        load_table<T, NC>(Sq[2], ax.S + p * n * n, sym[2]);
        load_table<T, NC>(Wq[2], ax.W + p * n * n, sym[2]);
      }
      for (int a = threadIdx.x; a < n; a += blockDim.x) {
        lq[q][a] = ax.lam[p * n + a];
        const int ph = ax.phys;
        const int npp = (ph == 2) ? dm.NPz : dm.NP;
        int G = patch_start(ax, (int)p, npp) + a;
        long long o;
        if (ax.periodic) {
          G %= ax.N;
          if (G < 0) G += ax.N;
          o = (long long)(G / npp) * estride[ph] + (G % npp) * nstride[ph];
        } else if (G < 0 || G >= ax.N) {
          o = kInvalidOffset;
        } else {
          o = (long long)(G / npp) * estride[ph] + (G % npp) * nstride[ph];
        }
        offq[q][a] = o;
      }
    }
    __syncthreads();
    for (int rr = threadIdx.x; rr < NB * NC; rr += blockDim.x)
      rowoff[rr] = off[NA + rr % NB] + off[NA + NB + rr / NB];
    __syncthreads();
    // forward a and b, slab by slab
    for (int c0 = 0; c0 < NC; c0 += CS) {
      const int cs = NC - c0 < CS ? NC - c0 : CS;
      for (int t = threadIdx.x; t < cs * NB * NA; t += blockDim.x) {
        const int row = t / NA, a = t - row * NA;              // row = b + NB k
        const long long o = off[a] + rowoff[c0 * NB + row];
        sb[row * NAP + a] = o >= 0 ? r[o] : T(0);
      }
      __syncthreads();
      axis_pass<T, NA, true>(sym[0], sb, Sq[0], NB * cs, NAP, NB * cs, 0, 1);
      __syncthreads();
      axis_pass<T, NB, true>(sym[1], sb, Sq[1], NA * cs, 1, NA, PL, NAP);
      __syncthreads();
      for (int t = threadIdx.x; t < cs * NB * NA; t += blockDim.x) {
        const int row = t / NA, a = t - row * NA;
        buf[(long long)c0 * NB * NA + t] = sb[row * NAP + a];
      }
      __syncthreads();
    }
    // c: forward with the scaling by 1 / (lambda_a + lambda_b + lambda_c), backward
    axis_pass<T, NC, true, 1>(sym[2], buf, Sq[2], NA * NB, 1, NA * NB, 0, NA * NB, lc,
                              [&](int l) { return la[l % NA] + lb[l / NA]; });
    __syncthreads();
    axis_pass<T, NC, false>(sym[2], buf, Wq[2], NA * NB, 1, NA * NB, 0, NA * NB);
    __syncthreads();
    // backward b and a, slab by slab, and the weighted corrections added to u
    for (int c0 = 0; c0 < NC; c0 += CS) {
      const int cs = NC - c0 < CS ? NC - c0 : CS;
      for (int t = threadIdx.x; t < cs * NB * NA; t += blockDim.x) {
        const int row = t / NA, a = t - row * NA;
        sb[row * NAP + a] = buf[(long long)c0 * NB * NA + t];
      }
      __syncthreads();
      axis_pass<T, NB, false>(sym[1], sb, Wq[1], NA * cs, 1, NA, PL, NAP);
      __syncthreads();
      axis_pass<T, NA, false>(sym[0], sb, Wq[0], NB * cs, NAP, NB * cs, 0, 1);
      __syncthreads();
      for (int t = threadIdx.x; t < cs * NB * NA; t += blockDim.x) {
        const int row = t / NA, a = t - row * NA;
        const long long o = off[a] + rowoff[c0 * NB + row];
        if (o >= 0) atomicAdd(u + o, sb[row * NAP + a]);
      }
      __syncthreads();
    }
  }
}

template <typename T, int NA, int NB, int NC, bool TC>
constexpr size_t fdm_smem_bytes() {
  return sizeof(long long) * ((NA + NB + NC + 1) / 2 * 2 + (NB * NC + 1) / 2 * 2) +
         sizeof(T) * ((size_t)padded<T>(NA * NB * NC) +
                      2 * (table_floats<T, TC>(NA) + table_floats<T, TC>(NB) + table_floats<T, TC>(NC)) +
                      NA + NB + NC);
}

template <typename T, int NA, int NB, int NC, bool TC = false>
int fdm_launch(const LevelDims& dm, const FdmFamily<T>& fam, const T* r, T* u, cudaStream_t s) {
  bool pipe = false;
  if constexpr (fdm_pipelined<T, NA, NB, NC, TC>())
    pipe = fam.variant < 0 ? fdm_pipelined_default<T, NA, NB, NC>() : fam.variant == 1;
  if constexpr (fdm_pipelined<T, NA, NB, NC, TC>()) if (pipe) {
    constexpr size_t smem2 = 2 * PipeStage<T, NA, NB, NC>::BYTES;
    constexpr int maxt = fdm_max_threads<T, NA, NB, NC>();
    struct Shape {
      int nsm;
      int per_sm[maxt / 32 + 1];
    };
    static PerDevice<Shape> shapes;
    int threads = (fam.threads >= 32 && fam.threads % 32 == 0) ? fam.threads : fdm_threads<NA, NB, NC>();
    if (threads > maxt) threads = maxt;
    int occ = 0, nsm = 0;
    const int rc = shapes.with(
        [](Shape& sh, int dev) {
          if (smem2 > 48 * 1024 &&
              cudaFuncSetAttribute(fdm_kernel_pipe<T, NA, NB, NC>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                   (int)smem2) != cudaSuccess)
            return (int)PMG_ECUDA;
          if (cudaDeviceGetAttribute(&sh.nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
            return (int)PMG_ECUDA;
          for (int& v : sh.per_sm) v = 0;
          return (int)PMG_OK;
        },
        [&](Shape& sh) {
          int& o = sh.per_sm[threads / 32];
          if (o <= 0 && cudaOccupancyMaxActiveBlocksPerMultiprocessor(&o, fdm_kernel_pipe<T, NA, NB, NC>, threads,
                                                                      smem2) != cudaSuccess)
            return (int)PMG_ECUDA;
          occ = o;
          nsm = sh.nsm;
          return (int)PMG_OK;
        });
    if (rc != PMG_OK) return rc;
    if (fam.count_total <= 0) return PMG_OK;
    long long grid = (long long)(occ > 0 ? occ : 1) * nsm;
    if (grid > fam.count_total) grid = fam.count_total;
    count_launch();
    fdm_kernel_pipe<T, NA, NB, NC><<<(unsigned)grid, threads, smem2, s>>>(dm, fam, r, u);
    return cudaGetLastError() == cudaSuccess ? PMG_OK : PMG_ECUDA;
  }
  if constexpr (fdm_smem_bytes<T, NA, NB, NC, TC>() > 227 * 1024) {
    static_assert(!TC, "tensor-core passes need the patch in shared memory");
    constexpr size_t smem_g = fdm_gbuf_smem_bytes<T, NA, NB, NC>();
    static_assert(smem_g <= 227 * 1024, "patch tables do not fit in shared memory");
    if (!fam.scratch || fam.scratch_ctas <= 0 || fam.scratch_stride < (long long)NA * NB * NC)
      return PMG_EINVAL;
    if (smem_g > 48 * 1024 &&
        cudaFuncSetAttribute(fdm_kernel_gbuf<T, NA, NB, NC>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)smem_g) != cudaSuccess)
      return PMG_ECUDA;
    if (fam.count_total <= 0) return PMG_OK;
    const int grid = fam.count_total < fam.scratch_ctas ? fam.count_total : fam.scratch_ctas;
    using SS = SlabShape<T, NA, NB, NC>;
    // slab form (3-D) or scratch form: the tuner times both (variant 1 / 0); untuned,
    // the slab form for fp32 face patches (FA P = 32: 13.8 -> 11.1 ms per family sweep
    // of 8^3 elements with four right-hand sides), the scratch form otherwise (fp32 EA
    // 4.3 against 4.9 ms, FP64 FA 110 against 123 ms)
    const bool slab = fam.variant < 0 ? (sizeof(T) == 4 && NA != NB) : fam.variant == 1;
    if constexpr (NC > 1 && SS::CS >= 1) if (slab) {
      // CTA size from the tuner, up to SS::MAXT
      if (SS::BYTES > 48 * 1024 &&
          cudaFuncSetAttribute(fdm_kernel_slab<T, NA, NB, NC>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                               (int)SS::BYTES) != cudaSuccess)
        return PMG_ECUDA;
      int threads = (fam.threads >= 32 && fam.threads % 32 == 0) ? fam.threads : SS::MAXT;
      if (threads > SS::MAXT) threads = SS::MAXT;
      count_launch();
      fdm_kernel_slab<T, NA, NB, NC><<<grid, threads, SS::BYTES, s>>>(dm, fam, r, u);
      return cudaGetLastError() == cudaSuccess ? PMG_OK : PMG_ECUDA;
    }
    int threads = (fam.threads >= 32 && fam.threads % 32 == 0) ? fam.threads : 256;
    if (threads > 256) threads = 256;
    count_launch();
    fdm_kernel_gbuf<T, NA, NB, NC><<<grid, threads, smem_g, s>>>(dm, fam, r, u);
    return cudaGetLastError() == cudaSuccess ? PMG_OK : PMG_ECUDA;
  } else {
  constexpr size_t smem = fdm_smem_bytes<T, NA, NB, NC, TC>();
  static_assert(smem <= 227 * 1024, "patch does not fit in shared memory");
  if (smem > 48 * 1024 &&
      cudaFuncSetAttribute(fdm_kernel<T, NA, NB, NC, TC>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           (int)smem) != cudaSuccess)
    return PMG_ECUDA;
  if (fam.count_total <= 0) return PMG_OK;
  constexpr int maxt = fdm_max_threads<T, NA, NB, NC>();
  int threads = (fam.threads >= 32 && fam.threads % 32 == 0) ? fam.threads : fdm_threads<NA, NB, NC>();
  if (threads > maxt) threads = maxt;
  count_launch();
  fdm_kernel<T, NA, NB, NC, TC><<<fam.count_total, threads, smem, s>>>(dm, fam, r, u);
  return cudaGetLastError() == cudaSuccess ? PMG_OK : PMG_ECUDA;
  }
}

}  // namespace pmg
