// pmg_fma_probe: a fused multiply-add throughput probe of the FP64 or FP32 pipes,
// the denominator of the roofline fraction of the ALU-bound kernels (the FP64
// patch solves and operator apply, the fp32 SIMT patch solves).  Not part of the
// paper's method.
//
// Every thread runs kChains independent recurrences x <- x * a + b (a multiply-add
// each), kUnroll steps per loop trip so that the loop counter and branch take a
// small share of the issue slots.  With a = 1 - 2^-20 and b = 2^-20 the fixed point
// b / (1 - a) is 1, and every chain, started in [0.5, 0.65], rises monotonically
// towards it: no value overflows or becomes subnormal.  The sum is stored only if it
// is negative, which never happens; the compiler cannot prove that, so every
// multiply-add is executed.  The probe allocates nothing.
#include "pmg_internal.h"

namespace pmg {

constexpr int kChains = 16;
constexpr int kUnroll = 4;
constexpr int kProbeThreads = 256;

__device__ double g_probe_sink64;
__device__ float g_probe_sink32;

template <typename T>
__global__ void __launch_bounds__(kProbeThreads) fma_probe_kernel(int iters) {
  const T a = (T)(1.0 - 1.0 / 1048576.0), b = (T)(1.0 / 1048576.0);
  T x[kChains];
#pragma unroll
  for (int c = 0; c < kChains; ++c) x[c] = (T)(0.5 + 0.01 * (c + (threadIdx.x & 7)));
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int u = 0; u < kUnroll; ++u)
#pragma unroll
      for (int c = 0; c < kChains; ++c) x[c] = fma(x[c], a, b);
  }
  T s = 0;
#pragma unroll
  for (int c = 0; c < kChains; ++c) s += x[c];
  if (s < (T)0) {
    if constexpr (sizeof(T) == 8) g_probe_sink64 = s;
    else g_probe_sink32 = s;
  }
}

}  // namespace pmg

extern "C" int pmg_fma_probe(int fp64, int iters, void* stream, double* flops) {
  using namespace pmg;
  if (iters < 1 || !flops) return PMG_EINVAL;
  int dev = 0, nsm = 0, per_sm = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
    return PMG_ECUDA;
  cudaError_t e = fp64 ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fma_probe_kernel<double>,
                                                                       kProbeThreads, 0)
                       : cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fma_probe_kernel<float>,
                                                                       kProbeThreads, 0);
  if (e != cudaSuccess) return PMG_ECUDA;
  if (per_sm < 1) per_sm = 1;
  const int blocks = per_sm * nsm;
  count_launch();
  if (fp64) fma_probe_kernel<double><<<blocks, kProbeThreads, 0, (cudaStream_t)stream>>>(iters);
  else fma_probe_kernel<float><<<blocks, kProbeThreads, 0, (cudaStream_t)stream>>>(iters);
  if (cudaGetLastError() != cudaSuccess) return PMG_ECUDA;
  *flops = 2.0 * (double)blocks * kProbeThreads * kChains * kUnroll * (double)iters;
  return PMG_OK;
}
