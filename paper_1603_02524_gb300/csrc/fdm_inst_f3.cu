// Instantiations of the Schwarz patch kernel: float, 3-D patch shapes
// (EA: n^3; FA: 2P x n_t^2), n = N_P + 2 N_o over the supported orders.
#include "fdm_kernel.cuh"

namespace pmg {

int fdm_dispatch_f3tc(const LevelDims& dm, const FdmFamily<float>& fam, const float* r, float* u,
                      cudaStream_t s);

int fdm_dispatch_f3(const LevelDims& dm, const FdmFamily<float>& fam, const float* r, float* u,
                     cudaStream_t s) {
  if (fam.tc) {                    // tensor-core line passes (tables unfolded)
    const int st = fdm_dispatch_f3tc(dm, fam, r, u, s);
    if (st != PMG_EINVAL) return st;
  }
  const int na = fam.ax[0].n, nb = fam.ax[1].n, nc = fam.ax[2].n;
#define C(A, B, CC) \
  if (na == A && nb == B && nc == CC) return fdm_launch<float, A, B, CC>(dm, fam, r, u, s);
  C(3, 3, 3) C(5, 5, 5) C(7, 7, 7) C(9, 9, 9) C(13, 13, 13) C(17, 17, 17) C(23, 23, 23)
  C(4, 3, 3) C(4, 5, 5) C(8, 5, 5) C(8, 7, 7) C(8, 9, 9) C(16, 9, 9) C(16, 13, 13)
  C(32, 17, 17) C(32, 23, 23)
  C(33, 33, 33) C(43, 43, 43) C(64, 33, 33) C(64, 43, 43)    // P = 32: patch buffers in global scratch
#undef C
  return PMG_EINVAL;
}

}  // namespace pmg
