// Instantiations of the Schwarz patch kernel with tensor-core line passes: fp32,
// 3-D patch shapes (EA: n^3; FA: 2P x n_t^2), all axes at most 32 nodes.
//   tc = 2 (one tf32 product per multiply-add): tcgen05 MMAs with accumulators in
//          tensor memory (fdm_tc.cuh)
//   tc = 1 (3xTF32 products, fp32-level accuracy): warp-level mma.sync passes
#include "fdm_tc.cuh"

namespace pmg {

// CTAs of the tcgen05 kernel that gave up waiting for their MMAs (stays 0).
__device__ unsigned int g_tc_timeouts;

// Device address of g_tc_timeouts on the current device (looked up once per device).
unsigned int* tc_timeouts_ptr() {
  static PerDevice<unsigned int*> addr;
  unsigned int* p = nullptr;
  addr.with(
      [](unsigned int*& a, int) {
        return cudaGetSymbolAddress(reinterpret_cast<void**>(&a), g_tc_timeouts) == cudaSuccess && a
                   ? (int)PMG_OK
                   : (int)PMG_ECUDA;
      },
      [&](unsigned int*& a) {
        p = a;
        return (int)PMG_OK;
      });
  return p;
}

int fdm_dispatch_f3tc(const LevelDims& dm, const FdmFamily<float>& fam, const float* r, float* u,
                      cudaStream_t s) {
  const int na = fam.ax[0].n, nb = fam.ax[1].n, nc = fam.ax[2].n;
  if (fam.tc == 2) {
    unsigned int* to = tc_timeouts_ptr();
    if (!to) return PMG_ECUDA;
#define C(A, B, CC) \
  if (na == A && nb == B && nc == CC) return fdm_launch_tc<A, B, CC>(dm, fam, r, u, to, s);
    C(3, 3, 3) C(5, 5, 5) C(7, 7, 7) C(9, 9, 9) C(13, 13, 13) C(17, 17, 17) C(23, 23, 23)
    C(4, 3, 3) C(4, 5, 5) C(8, 5, 5) C(8, 7, 7) C(8, 9, 9) C(16, 9, 9) C(16, 13, 13)
    C(32, 17, 17) C(32, 23, 23)
#undef C
    return PMG_EINVAL;
  }
#define C(A, B, CC) \
  if (na == A && nb == B && nc == CC) return fdm_launch<float, A, B, CC, true>(dm, fam, r, u, s);
  C(3, 3, 3) C(5, 5, 5) C(7, 7, 7) C(9, 9, 9) C(13, 13, 13) C(17, 17, 17) C(23, 23, 23)
  C(4, 3, 3) C(4, 5, 5) C(8, 5, 5) C(8, 7, 7) C(8, 9, 9) C(16, 9, 9) C(16, 13, 13)
  C(32, 17, 17) C(32, 23, 23)
#undef C
  return PMG_EINVAL;
}

// Read and reset the timeout count (host; synchronises the device).
int tc_timeouts_take(unsigned int* out) {
  unsigned int* p = tc_timeouts_ptr();
  if (!p) return PMG_ECUDA;
  unsigned int v = 0;
  if (cudaMemcpy(&v, p, sizeof(v), cudaMemcpyDeviceToHost) != cudaSuccess ||
      cudaMemset(p, 0, sizeof(v)) != cudaSuccess)
    return PMG_ECUDA;
  *out = v;
  return PMG_OK;
}

}  // namespace pmg
