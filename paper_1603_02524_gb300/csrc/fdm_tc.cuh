// Schwarz patch solve (Sec. 3.1) with the six line passes of the fast
// diagonalisation as tf32 matrix products on the fifth-generation tensor cores
// (tcgen05: operands in shared memory, accumulators in tensor memory).
//
// A line pass along axis q of a patch with n_q nodes on that axis is the
// product D = A B^T: A holds one row per line (the M = product of the other two
// patch extents lines; K = n_q inputs), B the n_q x n_q table (row j = output j),
// D one row per line with its n_q outputs.  M is cut into tiles of 128 rows, K
// into steps of 8; the accumulator of tile t occupies tensor-memory columns
// [t N_pad, (t + 1) N_pad).  Between passes the accumulators are read back
// (one row per thread) and written into shared memory as the next pass's A, in
// the row order that pass needs; the third forward pass's read-back applies the
// inverse eigenvalue sums, the last backward pass's read-back goes to a plain
// staging array from which the weighted corrections are added to u (atomically,
// patches overlap) with coalesced accesses.
//
// Row orders (m) and K indices of the six A operands, for a patch (a, b, c)
// of extents (NA, NB, NC); primes mark transformed (mode) indices, XP is X
// rounded up to a multiple of 8 (rows with an index beyond its extent are
// padding whose accumulators are never read):
//   pass 0  forward a   m = b + NBP c,    k = a
//   pass 1  forward b   m = c + NCP a',   k = b
//   pass 2  forward c   m = b + NBP a',   k = c      (outputs scaled)
//   pass 3  backward c  m = b' + NBP a',  k = c'
//   pass 4  backward b  m = a' + NAP c,   k = b'
//   pass 5  backward a  m = b + NBP c,    k = a'
// For patches whose padded extents are all 24 (PERM: 17 to 23 nodes per axis) the
// line indices c of A1, a' of A2/A3 (and of A4, composed) and c of A5 are permuted
// within blocks of 8 (tc_sig, tc_tau), so that the two patch lines a 32-row warp
// covers store into disjoint shared-memory banks.
// With the padded strides, the shared-memory offset of output j of a row is the
// thread's base offset plus a compile-time step.  Each pass's read-back writes,
// for a fixed output, consecutive K indices from consecutive threads (except
// pass 2, whose outputs are the next K index); with core matrices 144 bytes
// apart along K those stores fall into distinct shared-memory banks.
//
// Precision: tf32 products (10-bit operand mantissas) with fp32 accumulation;
// the tables are rounded to tf32 on the host; the gathered residual and the fp32
// operands stored between passes are truncated to tf32 by the tensor core (relative
// error below 2^-10 each; rounding them first cost two integer operations per value
// and changed neither the iteration counts nor the smoother's error bound).
// The preconditioner is applied inside a flexible CG whose residual, operator
// and inner products stay FP64.
#pragma once

#include "fdm_kernel.cuh"
#include "umma.cuh"

namespace pmg {

// Geometry of the tensor-core patch kernel for a patch of extents NA x NB x NC.
template <int NA, int NB, int NC>
struct TcGeom {
  static constexpr int NN = NA * NB * NC;
  __host__ __device__ static constexpr int kp(int n) { return (n + 7) / 8 * 8; }      // K padded to whole MMA steps
  __host__ __device__ static constexpr int npd(int n) { return (n + 15) / 16 * 16; }  // N of an M = 128 MMA
  __host__ __device__ static constexpr int mt(int m) { return (m + 127) / 128; }      // row tiles
  // fastest row index of every operand padded to a multiple of 8, so that a row
  // step of the slow index is a whole number of 8-row core-matrix groups
  static constexpr int NAP = (NA + 7) / 8 * 8, NBP = (NB + 7) / 8 * 8, NCP = (NC + 7) / 8 * 8;
  // Row permutations (PERM, all extents padded to 24): a warp's 32 rows span two
  // patch lines, whose read-back stores would share banks in the next operand; the
  // next operand's rows are permuted (tc_sig, tc_tau below) so that the second line
  // lands on the banks the first leaves free.
  static constexpr bool PERM = NAP == 24 && NBP == 24 && NCP == 24;
  static constexpr int M0 = NBP * NC;   // pass 0:      rows b + NBP c
  static constexpr int M5 = PERM ? NBP * NCP : NBP * NC;   // pass 5: rows b + NBP tau(c)
  static constexpr int M1 = NCP * NA;   // pass 1:      rows sig(c) + NCP a'
  static constexpr int M2 = PERM ? NBP * NAP : NBP * NA;   // passes 2, 3: rows b + NBP tau(a')
  static constexpr int M4 = NAP * NC;   // pass 4:      rows sig(tau(a')) + NAP c
  static constexpr uint32_t LBO = 144;                            // A: core matrices along K
  __host__ __device__ static constexpr uint32_t sbo(int n) { return (uint32_t)(kp(n) / 4) * LBO; }
  __host__ __device__ static constexpr uint32_t abytes(int n, int m) { return (uint32_t)mt(m) * 16u * sbo(n); }
  __host__ __device__ static constexpr uint32_t mx(uint32_t x, uint32_t y) { return x > y ? x : y; }
  static constexpr int FS = (NA + 3) / 4 * 4 % 8 == 0 ? (NA + 3) / 4 * 4 + 4 : (NA + 3) / 4 * 4;  // staging row stride
  static constexpr uint32_t ABYTES =
      (mx(mx(mx(mx(abytes(NA, M0), abytes(NA, M5)), abytes(NB, M1)), mx(abytes(NC, M2), abytes(NB, M4))),
          4u * NB * NC * FS) + 1023) /
      1024 * 1024;
  // B tables: dense K-major (core matrices 128 bytes apart along K)
  __host__ __device__ static constexpr uint32_t tsbo(int n) { return (uint32_t)(kp(n) / 4) * 128u; }
  __host__ __device__ static constexpr uint32_t tbytes(int n) { return (uint32_t)npd(n) * (uint32_t)kp(n) * 4u; }
  static constexpr uint32_t T_OFF = ABYTES;                       // S_a, W_a, S_b, W_b, S_c, W_c
  __host__ __device__ static constexpr uint32_t tab_off(int i) {
    return T_OFF + (i >= 1 ? tbytes(NA) : 0) + (i >= 2 ? tbytes(NA) : 0) + (i >= 3 ? tbytes(NB) : 0) +
           (i >= 4 ? tbytes(NB) : 0) + (i >= 5 ? tbytes(NC) : 0);
  }
  static constexpr uint32_t OFF_OFF = tab_off(5) + tbytes(NC);
  static constexpr int NOFF = (NA + NB + NC + 1) / 2 * 2;
  static constexpr uint32_t LAM_OFF = OFF_OFF + 8u * NOFF;
  // mbarrier of the MMA completions (+0), tensor-memory address slot (+8), and a
  // second mbarrier that nothing ever completes (+16): the stalled-wait test hook
  static constexpr uint32_t BAR_OFF = (LAM_OFF + 4u * (NA + NB + NC) + 15) / 16 * 16;
  static constexpr uint32_t BYTES = BAR_OFF + 32;
  __host__ __device__ static constexpr uint32_t cols(int n, int m) { return (uint32_t)mt(m) * (uint32_t)npd(n); }
  static constexpr uint32_t COLS_USED =
      mx(mx(mx(cols(NA, M0), cols(NA, M5)), cols(NB, M1)), mx(cols(NC, M2), cols(NB, M4)));
  static constexpr uint32_t TCOLS = COLS_USED <= 32 ? 32 : COLS_USED <= 64 ? 64 : COLS_USED <= 128 ? 128 : 256;
  static_assert(COLS_USED <= 256, "accumulators exceed the tensor-memory budget of one CTA");
  static_assert(NA <= 32 && NB <= 32 && NC <= 32 && NC > 1, "tensor-core patch kernel: 3-D, n <= 32");
};

// Table of the patch (forward S or backward W^T, n x n, entry [k][j] = input k,
// output j; uploaded already rounded to tf32) as the K-major B operand:
// asynchronous element copies (the zero pads of the npd(n) x kp(n) operand are
// written once per CTA).
template <int NA, int NB, int NC, int N>
__device__ __forceinline__ int tc_boff(int i) {
  using G = TcGeom<NA, NB, NC>;
  const int k = i / N, j = i - k * N;
  return (j >> 3) * (int)(G::tsbo(N) / 4) + (k >> 2) * 32 + (j & 7) * 4 + (k & 3);
}
template <int NA, int NB, int NC, int N>
__device__ __forceinline__ void tc_table_async(float* B, const float* __restrict__ src) {
  for (int i = threadIdx.x; i < N * N; i += blockDim.x) cp_async<4>(B + tc_boff<NA, NB, NC, N>(i), src + i, true);
}
// The row permutations of PERM shapes, on [0, 24) and mapping each block of 8 to
// itself.  tc_sig moves consecutive line indices to rows whose bank offsets differ by
// 24 words (4 x 6 mod 32) within each block of 4; tc_tau reverses the last three of
// each block of 4, so that consecutive line indices land 3 rows (24 words mod 32) apart;
// tc_tau is its own inverse.
__device__ __forceinline__ int tc_sig(int c) {
  const int k = c >> 2, q = k & 1, g = k >> 1, i = c & 3;
  return 8 * g + ((q + 6 * i - 6 * g + 48) & 7);
}
__device__ __forceinline__ int tc_sig_inv(int r) {
  const int g = r >> 3, s = r & 7, q = s & 1;
  return 4 * (2 * g + q) + ((3 * ((s - q) >> 1) + g) & 3);
}
__device__ __forceinline__ int tc_tau(int a) { return (a & ~3) | ((3 * (a & 3)) & 3); }

// Store accumulator row m (registers r, outputs j = 0..) of pass PASS as the next
// pass's operand (or, after the last pass, into the staging rows); rows beyond the
// patch extents are padding and are dropped.
template <int NA, int NB, int NC, int PASS, int NPD>
__device__ __forceinline__ void tc_store_row(float* A, int m, const uint32_t (&r)[NPD], const float* la,
                                             const float* lb, const float* lc) {
  using G = TcGeom<NA, NB, NC>;
  auto d = [&](int j) { return __uint_as_float(r[j]); };
  // offsets of the next operand: a thread-dependent base plus, for output j, a
  // compile-time step (rows a multiple of 8 apart, or a fixed position in K)
  if constexpr (PASS == 0) {                   // m = b + NBP c -> A1[sig(c) + NCP a'][b]
    constexpr int S = (int)G::sbo(NB) / 4;
    const int b = m % G::NBP, c = m / G::NBP;
    if (b >= NB || c >= NC) return;
    const int cr = G::PERM ? tc_sig(c) : c;
    const int base = (cr >> 3) * S + (cr & 7) * 4 + (b >> 2) * 36 + (b & 3);
#pragma unroll
    for (int j = 0; j < NA; ++j) A[base + j * (G::NCP / 8) * S] = d(j);
  } else if constexpr (PASS == 1) {            // m = sig(c) + NCP a' -> A2[b' + NBP tau(a')][c]
    constexpr int S = (int)G::sbo(NC) / 4;
    const int c = G::PERM ? tc_sig_inv(m % G::NCP) : m % G::NCP, a = m / G::NCP;
    if (c >= NC || a >= NA) return;
    const int base = (G::PERM ? tc_tau(a) : a) * (G::NBP / 8) * S + (c >> 2) * 36 + (c & 3);
#pragma unroll
    for (int j = 0; j < NB; ++j) A[base + (j >> 3) * S + (j & 7) * 4] = d(j);
  } else if constexpr (PASS == 2) {            // m = b' + NBP tau(a') -> A3[m][c'] / (la + lb + lc)
    constexpr int S = (int)G::sbo(NC) / 4;
    const int b = m % G::NBP, a = G::PERM ? tc_tau(m / G::NBP) : m / G::NBP;
    if (b >= NB || a >= NA) return;
    const float s0 = la[a] + lb[b];
    float4* dst = reinterpret_cast<float4*>(A + (m >> 3) * S + (m & 7) * 4);   // 4 K values: 16 bytes
#pragma unroll
    for (int g = 0; g < (NC + 3) / 4; ++g) {
      float v[4];
#pragma unroll
      for (int k = 0; k < 4; ++k) v[k] = (4 * g + k < NC) ? d(4 * g + k) * recip(s0 + lc[4 * g + k]) : 0.0f;
      dst[g * 9] = make_float4(v[0], v[1], v[2], v[3]);                        // groups 144 bytes apart
    }
  } else if constexpr (PASS == 3) {            // m = b' + NBP tau(a') -> A4[sig(tau(a')) + NAP c][b']
    constexpr int S = (int)G::sbo(NB) / 4;
    const int b = m % G::NBP, u = m / G::NBP, a = G::PERM ? tc_tau(u) : u;
    if (b >= NB || a >= NA) return;
    const int ar = G::PERM ? tc_sig(u) : a;    // sig(tau(a')) = sig(u)
    const int base = (ar >> 3) * S + (ar & 7) * 4 + (b >> 2) * 36 + (b & 3);
#pragma unroll
    for (int j = 0; j < NC; ++j) A[base + j * (G::NAP / 8) * S] = d(j);
  } else if constexpr (PASS == 4) {            // m = sig(tau(a')) + NAP c -> A5[b + NBP tau(c)][a']
    constexpr int S = (int)G::sbo(NA) / 4;
    const int a = G::PERM ? tc_tau(tc_sig_inv(m % G::NAP)) : m % G::NAP, c = m / G::NAP;
    if (a >= NA || c >= NC) return;
    const int base = (G::PERM ? tc_tau(c) : c) * (G::NBP / 8) * S + (a >> 2) * 36 + (a & 3);
#pragma unroll
    for (int j = 0; j < NB; ++j) A[base + (j >> 3) * S + (j & 7) * 4] = d(j);
  } else {                                     // m = b + NBP tau(c) -> staging row b + NB c
    const int b = m % G::NBP, c = G::PERM ? tc_tau(m / G::NBP) : m / G::NBP;
    if (b >= NB || c >= NC) return;
    float4* st = reinterpret_cast<float4*>(A + (b + NB * c) * G::FS);
#pragma unroll
    for (int g = 0; g < (NA + 3) / 4; ++g)
      st[g] = make_float4(d(4 * g), 4 * g + 1 < NA ? d(4 * g + 1) : 0.0f, 4 * g + 2 < NA ? d(4 * g + 2) : 0.0f,
                          4 * g + 3 < NA ? d(4 * g + 3) : 0.0f);
  }
}

// One line pass: MMAs of all row tiles (one thread), wait, read-back into the
// next operand.  Returns false (uniformly) if the MMAs did not complete in time.
// stall_ns != 0 (test hook): the threads wait instead on `never`, an mbarrier that
// nothing completes, and give up after stall_ns; the MMAs stay in flight on mbar.
template <int NA, int NB, int NC, int PASS>
__device__ __forceinline__ bool tc_pass(float* A, const float* B, uint64_t* mbar, uint32_t& phase, uint32_t tmem,
                                        const float* la, const float* lb, const float* lc, uint64_t* never,
                                        uint32_t stall_ns) {
  using G = TcGeom<NA, NB, NC>;
  constexpr int q = (PASS == 0 || PASS == 5) ? 0 : (PASS == 1 || PASS == 4) ? 1 : 2;
  constexpr int n = q == 0 ? NA : q == 1 ? NB : NC;
  constexpr int M = PASS == 0 ? G::M0 : PASS == 5 ? G::M5 : PASS == 1 ? G::M1 : PASS == 4 ? G::M4 : G::M2;
  constexpr int KS = G::kp(n) / 8, NPD = G::npd(n), MT = G::mt(M);
  constexpr uint32_t SB = G::sbo(n);
  constexpr uint32_t idesc = umma::idesc_tf32(128, NPD);
  // generic-proxy stores of A (and of the tables) -> visible to the tensor core;
  // earlier tensor-memory reads complete before the accumulators are overwritten
  umma::fence_async_smem();
  umma::fence_before_sync();
  __syncthreads();
  if (threadIdx.x == 0) {
    umma::fence_after_sync();
    // descriptors of the first tile and K step; later ones advance the start
    // address field (bytes / 16; operands lie below 256 KB, so no carry)
    const uint64_t ad = umma::smem_desc(umma::smem_u32(A), G::LBO, SB);
    const uint64_t bd = umma::smem_desc(umma::smem_u32(B), 128, G::tsbo(n));
#pragma unroll
    for (int t = 0; t < MT; ++t)
#pragma unroll
      for (int ks = 0; ks < KS; ++ks)
        umma::mma_tf32(tmem + (uint32_t)(t * NPD), ad + (uint64_t)((t * 16 * SB + ks * 2 * G::LBO) >> 4),
                       bd + (uint64_t)((ks * 256) >> 4), idesc, ks > 0);
    umma::mma_commit(mbar);
  }
  const bool ok = stall_ns ? umma::mbar_wait(never, 0, stall_ns) : umma::mbar_wait(mbar, phase, 1000000000ull);
  phase ^= 1u;
  if (__syncthreads_or(!ok)) return false;
  umma::fence_after_sync();

  // read-back: warp w reads lanes 32 (w % 4) .. of tiles w / 4, w / 4 + nw / 4, ...;
  // the tensor-memory load of the warp's next tile is in flight while it stores this one
  const int warp = threadIdx.x >> 5, quarter = warp & 3;
  const int nw4 = blockDim.x >> 7;
  auto valid = [&](int t) { return t < MT && t * 128 + 32 * quarter < M; };
  auto taddr = [&](int t) { return tmem + ((uint32_t)(32 * quarter) << 16) + (uint32_t)(t * NPD); };
  uint32_t ra[NPD];
  for (int t = warp >> 2; valid(t); t += nw4) {
    umma::tmem_ld_nowait<NPD>(taddr(t), ra);
    umma::tmem_wait_ld<NPD>(ra);
    tc_store_row<NA, NB, NC, PASS>(A, t * 128 + 32 * quarter + (threadIdx.x & 31), ra, la, lb, lc);
  }
  return true;
}

// Persistent CTAs (blockDim a multiple of 128, at most 512) walk over the patches of a family.
// *timeouts counts CTAs that gave up waiting for their MMAs (they stop early); such a
// CTA also sets the family's device status word (fam.status, the hierarchy's) to
// PMG_ETIMEOUT if it holds no other status.
template <int NA, int NB, int NC>
__global__ void __launch_bounds__(512)
fdm_kernel_tc(LevelDims dm, FdmFamily<float> fam, const float* __restrict__ r, float* __restrict__ u,
              unsigned int* timeouts) {
  using G = TcGeom<NA, NB, NC>;
  extern __shared__ __align__(1024) unsigned char tc_smem[];
  float* A = reinterpret_cast<float*>(tc_smem);
  float* Tb[6];
#pragma unroll
  for (int i = 0; i < 6; ++i) Tb[i] = reinterpret_cast<float*>(tc_smem + G::tab_off(i));
  long long* off = reinterpret_cast<long long*>(tc_smem + G::OFF_OFF);
  float* la = reinterpret_cast<float*>(tc_smem + G::LAM_OFF);
  float* lb = la + NA;
  float* lc = lb + NB;
  uint64_t* mbar = reinterpret_cast<uint64_t*>(tc_smem + G::BAR_OFF);
  uint32_t* slot = reinterpret_cast<uint32_t*>(tc_smem + G::BAR_OFF + 8);
  uint64_t* never = reinterpret_cast<uint64_t*>(tc_smem + G::BAR_OFF + 16);
  const uint32_t stall_ns = fam.stall_ns;
  const int tid = threadIdx.x;

  // operand pads must hold finite values (their products with the zero table pads vanish)
  for (int i = tid; i < (int)(G::OFF_OFF / 4); i += blockDim.x) A[i] = 0.0f;
  if (tid == 0) {
    umma::mbar_init(mbar, 1);
    umma::mbar_init(never, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (tid < 32) {
    umma::tmem_alloc(slot, G::TCOLS);
    umma::tmem_relinquish();
  }
  umma::fence_before_sync();
  __syncthreads();
  umma::fence_after_sync();
  const uint32_t tmem = *slot;
  uint32_t phase = 0;

  const int ca = fam.ax[0].count, cb = fam.ax[1].count;
  const int nq[3] = {NA, NB, NC};
  float* lq[3] = {la, lb, lc};
  long long* offq[3] = {off, off + NA, off + NA + NB};
  const long long nodes_el = (long long)dm.NP * dm.NP * dm.NPz;
  const long long estride[3] = {nodes_el, nodes_el * dm.ne[0], nodes_el * dm.ne[0] * dm.ne[1]};
  const long long nstride[3] = {1, dm.NP, (long long)dm.NP * dm.NP};
  bool ok = true;
  // contiguous chunk of patches per CTA: consecutive patches share their b and c
  // positions (and often a), whose tables, eigenvalues and offsets are kept
  const int chunk = (fam.count_total + gridDim.x - 1) / gridDim.x;
  const int pbeg = blockIdx.x * chunk;
  const int pend = min(fam.count_total, pbeg + chunk);
  int prev[3] = {-1, -1, -1}, prevtab[3] = {-1, -1, -1};
  for (int pid = pbeg; pid < pend && ok; ++pid) {
    const int pidx[3] = {pid % ca, (pid / ca) % cb, pid / (ca * cb)};
    const bool fresh[3] = {pidx[0] != prev[0], pidx[1] != prev[1], pidx[2] != prev[2]};
#pragma unroll
    for (int q = 0; q < 3; ++q) {
      if (!fresh[q]) continue;
      const FdmAxis<float>& ax = fam.ax[q];
      const int n = nq[q];
      const size_t p = pidx[q];
      // tables and eigenvalues only when they differ from the ones in shared memory
      const int tab = ax.tabid ? __ldg(ax.tabid + p) : (int)p;
      const bool newtab = tab != prevtab[q];
      prevtab[q] = tab;
      if (newtab) {
        if (q == 0) {
          tc_table_async<NA, NB, NC, NA>(Tb[0], ax.S + p * NA * NA);
          tc_table_async<NA, NB, NC, NA>(Tb[1], ax.W + p * NA * NA);
        } else if (q == 1) {
          tc_table_async<NA, NB, NC, NB>(Tb[2], ax.S + p * NB * NB);
          tc_table_async<NA, NB, NC, NB>(Tb[3], ax.W + p * NB * NB);
        } else {
          tc_table_async<NA, NB, NC, NC>(Tb[4], ax.S + p * NC * NC);
          tc_table_async<NA, NB, NC, NC>(Tb[5], ax.W + p * NC * NC);
        }
      }
      for (int a = tid; a < n; a += blockDim.x) {
        if (newtab) cp_async<4>(lq[q] + a, ax.lam + p * n + a, true);
        const int ph = ax.phys;
        const int npp = (ph == 2) ? dm.NPz : dm.NP;
        int Gi = patch_start(ax, (int)p, npp) + a;
        long long o;
        if (ax.periodic) {
          Gi %= ax.N;
          if (Gi < 0) Gi += ax.N;
          o = (long long)(Gi / npp) * estride[ph] + (Gi % npp) * nstride[ph];
        } else if (Gi < 0 || Gi >= ax.N) {
          o = kInvalidOffset;
        } else {
          o = (long long)(Gi / npp) * estride[ph] + (Gi % npp) * nstride[ph];
        }
        offq[q][a] = o;
      }
    }
    __syncthreads();
    // gather into the first operand (row b + NBP c, K index a) as asynchronous copies,
    // zero-filled outside the grid: each thread takes one (a, c) line and walks b (the
    // row's offset in the operand is then a compile-time step, the global offset one
    // broadcast load); lanes hold consecutive a, so a warp's copies are contiguous
    {
      constexpr int S = (int)G::sbo(NA) / 4;
      for (int pr = tid; pr < NA * NC; pr += blockDim.x) {
        const int a = pr % NA, c = pr / NA;
        const long long oac = off[a] + off[NA + NB + c];
        const int dac = c * (G::NBP / 8) * S + (a >> 2) * 36 + (a & 3);
#pragma unroll
        for (int b = 0; b < NB; ++b) {
          const long long o = oac + off[NA + b];
          cp_async<4>(A + dac + (b >> 3) * S + (b & 7) * 4, o >= 0 ? r + o : r, o >= 0);
        }
      }
    }
    cp_async_commit();
    cp_async_wait<0>();
    prev[0] = pidx[0];
    prev[1] = pidx[1];
    prev[2] = pidx[2];
    ok = tc_pass<NA, NB, NC, 0>(A, Tb[0], mbar, phase, tmem, la, lb, lc, never, stall_ns) &&
         tc_pass<NA, NB, NC, 1>(A, Tb[2], mbar, phase, tmem, la, lb, lc, never, stall_ns) &&
         tc_pass<NA, NB, NC, 2>(A, Tb[4], mbar, phase, tmem, la, lb, lc, never, stall_ns) &&
         tc_pass<NA, NB, NC, 3>(A, Tb[5], mbar, phase, tmem, la, lb, lc, never, stall_ns) &&
         tc_pass<NA, NB, NC, 4>(A, Tb[3], mbar, phase, tmem, la, lb, lc, never, stall_ns) &&
         tc_pass<NA, NB, NC, 5>(A, Tb[1], mbar, phase, tmem, la, lb, lc, never, stall_ns);
    if (!ok) break;
    __syncthreads();
    // scatter: the weighted corrections (staging row b + NB c, column a) added to u,
    // again one (a, c) line per thread walking b
    for (int pr = tid; pr < NA * NC; pr += blockDim.x) {
      const int a = pr % NA, c = pr / NA;
      const long long oac = off[a] + off[NA + NB + c];
      const float* st = A + (NB * c) * G::FS + a;
#pragma unroll
      for (int b = 0; b < NB; ++b) {
        const long long o = oac + off[NA + b];
        const float v = st[b * G::FS];
        if (o >= 0) atomicAdd(u + o, v);
      }
    }
    __syncthreads();                             // staging, offsets and tables are rewritten next
  }
  if (!ok) {
    if (tid == 0) {
      atomicAdd(timeouts, 1u);
      if (fam.status) atomicCAS(fam.status, 0, (int)PMG_ETIMEOUT);
    }
    // the MMAs may still be running: give them a bounded time before the release
    umma::mbar_wait(mbar, phase ^ 1u, 1000000000ull);
  }
  umma::fence_before_sync();
  __syncthreads();
  if (tid < 32) umma::tmem_dealloc(tmem, G::TCOLS);
}

// Launch: persistent grid of (resident CTAs per SM, limited by shared memory and
// by tensor memory) x SMs.  fam.threads (128, 256, 384 or 512) selects the CTA size.
template <int NA, int NB, int NC>
int fdm_launch_tc(const LevelDims& dm, const FdmFamily<float>& fam, const float* r, float* u,
                  unsigned int* timeouts, cudaStream_t s) {
  using G = TcGeom<NA, NB, NC>;
  constexpr size_t smem = G::BYTES;
  static_assert(smem <= 227 * 1024, "tensor-core patch kernel: shared memory");
  struct Shape {
    int nsm, smem_sm, smem_rsv, regs_sm, thr_sm, blk_sm, numRegs;
    int occ[5];
  };
  static PerDevice<Shape> shapes;
  const int threads = fam.threads >= 128 && fam.threads <= 512 && fam.threads % 128 == 0
                          ? fam.threads
                          : (G::NN >= 4096 ? 256 : 128);
  int o = 1, nsm = 0;
  const int rc = shapes.with(
      [](Shape& sh, int dev) {
        cudaFuncAttributes fa{};
        if (smem > 48 * 1024 &&
            cudaFuncSetAttribute(fdm_kernel_tc<NA, NB, NC>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)smem) != cudaSuccess)
          return (int)PMG_ECUDA;
        if (cudaFuncSetAttribute(fdm_kernel_tc<NA, NB, NC>, cudaFuncAttributePreferredSharedMemoryCarveout,
                                 (int)cudaSharedmemCarveoutMaxShared) != cudaSuccess ||
            cudaDeviceGetAttribute(&sh.nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
            cudaDeviceGetAttribute(&sh.smem_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev) != cudaSuccess ||
            cudaDeviceGetAttribute(&sh.smem_rsv, cudaDevAttrReservedSharedMemoryPerBlock, dev) != cudaSuccess ||
            cudaDeviceGetAttribute(&sh.regs_sm, cudaDevAttrMaxRegistersPerMultiprocessor, dev) != cudaSuccess ||
            cudaDeviceGetAttribute(&sh.thr_sm, cudaDevAttrMaxThreadsPerMultiProcessor, dev) != cudaSuccess ||
            cudaDeviceGetAttribute(&sh.blk_sm, cudaDevAttrMaxBlocksPerMultiprocessor, dev) != cudaSuccess ||
            cudaFuncGetAttributes(&fa, fdm_kernel_tc<NA, NB, NC>) != cudaSuccess)
          return (int)PMG_ECUDA;
        sh.numRegs = fa.numRegs;
        for (int& v : sh.occ) v = 0;
        return (int)PMG_OK;
      },
      [&](Shape& sh) {
        // resident CTAs per SM: shared memory, registers (whole warps, 256-register
        // granules), threads, blocks, and the 512 tensor-memory columns
        int& oc = sh.occ[threads / 128];
        if (oc <= 0) {
          const int by_smem = sh.smem_sm / ((int)smem + sh.smem_rsv);
          const int regs_warp = (sh.numRegs * 32 + 255) / 256 * 256;
          const int by_regs = sh.regs_sm / (regs_warp * (threads / 32));
          int v = by_smem < by_regs ? by_smem : by_regs;
          if (v > sh.thr_sm / threads) v = sh.thr_sm / threads;
          if (v > sh.blk_sm) v = sh.blk_sm;
          if (v > 512 / (int)G::TCOLS) v = 512 / (int)G::TCOLS;
          oc = v < 1 ? 1 : v;
        }
        o = oc;
        nsm = sh.nsm;
        return (int)PMG_OK;
      });
  if (rc != PMG_OK) return rc;
  if (fam.count_total <= 0) return PMG_OK;
  long long grid = (long long)o * nsm;
  if (grid > fam.count_total) grid = fam.count_total;
  count_launch();
  fdm_kernel_tc<NA, NB, NC><<<(unsigned)grid, threads, smem, s>>>(dm, fam, r, u, timeouts);
  return cudaGetLastError() == cudaSuccess ? PMG_OK : PMG_ECUDA;
}

}  // namespace pmg
