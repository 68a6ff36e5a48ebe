// Instantiations of the Schwarz patch kernel: double, 2-D patch shapes
// (EA: n^2; FA: 2P x n_t^1), n = N_P + 2 N_o over the supported orders.
#include "fdm_kernel.cuh"

namespace pmg {

int fdm_dispatch_d2(const LevelDims& dm, const FdmFamily<double>& fam, const double* r, double* u,
                     cudaStream_t s) {
  const int na = fam.ax[0].n, nb = fam.ax[1].n, nc = fam.ax[2].n;
#define C(A, B, CC) \
  if (na == A && nb == B && nc == CC) return fdm_launch<double, A, B, CC>(dm, fam, r, u, s);
  C(3, 3, 1) C(5, 5, 1) C(7, 7, 1) C(9, 9, 1) C(13, 13, 1) C(17, 17, 1) C(23, 23, 1)
  C(33, 33, 1) C(43, 43, 1)
  C(4, 3, 1) C(4, 5, 1) C(8, 5, 1) C(8, 7, 1) C(8, 9, 1) C(16, 9, 1) C(16, 13, 1)
  C(32, 17, 1) C(32, 23, 1) C(64, 33, 1) C(64, 43, 1)
#undef C
  return PMG_EINVAL;
}

}  // namespace pmg
