// The outer CG's operator apply in double-float arithmetic (fp64 vectors in and
// out, two fp32 words per value inside): the same sum-factorised kernel as the
// FP64 apply, instantiated for the dfloat type of dfloat.cuh.
#include "apply_kernel.cuh"
#include "dfloat.cuh"

namespace pmg {

int launch_apply_df(const LevelDims& dm, const ApplyTables<dfloat>& at, const double* u,
                    const double* f, double* v, cudaStream_t s, const int* unz) {
  if (dm.nelem == 0) return PMG_OK;
#define PMG_APPLY_CASE(DIMV, NPV) \
  if (dm.dim == DIMV && dm.NP == NPV) return apply_dispatch<dfloat, DIMV, NPV, double>(dm, at, u, f, v, s, unz);
  PMG_APPLY_CASE(3, 2) PMG_APPLY_CASE(3, 3) PMG_APPLY_CASE(3, 5) PMG_APPLY_CASE(3, 9)
  PMG_APPLY_CASE(3, 17)
  if (dm.dim == 3 && dm.NP == 33) return apply_dispatch_axes<dfloat, 33, double>(dm, at, u, f, v, s, unz);
  PMG_APPLY_CASE(2, 2) PMG_APPLY_CASE(2, 3) PMG_APPLY_CASE(2, 5) PMG_APPLY_CASE(2, 9)
  PMG_APPLY_CASE(2, 17) PMG_APPLY_CASE(2, 33)
#undef PMG_APPLY_CASE
  return PMG_EINVAL;
}

}  // namespace pmg
