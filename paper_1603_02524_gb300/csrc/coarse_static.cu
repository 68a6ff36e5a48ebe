// pmg_coarse_solve_static: the exact coarse solve of pmg_coarse_solve with its two
// scratch vectors taken from a fixed device array instead of hierarchy workspace.
//
// For callers that cannot call cudaMalloc when they solve: code that lives inside a
// host framework whose own allocator owns all device memory and forbids side
// allocations, or a caller that reserved its memory up front and must not grow it
// mid-run.  The call itself allocates nothing: no cudaMalloc, no cudaFree, no
// allocating library routine.
//
// Limit: the coarse (P = 1) problem may have at most kCoarseStaticMaxDof = 262 144
// unknowns (32^3 elements in 3-D).  The array, 2 x 262 144 doubles = 4 MiB, is part
// of the library image: every GPU that loads the library holds it until the process
// exits.
#include <mutex>
#include <string>

#include "pmg_internal.h"

namespace pmg {

constexpr long long kCoarseStaticMaxDof = 262144;

// The two ping-pong vectors of the coarse fast diagonalisation.  Host code must
// never pass this name to a kernel: on the host it is only a stand-in for the
// device symbol.  The device address comes from cudaGetSymbolAddress below.
static __device__ __align__(256) double g_coarse_scratch[2 * kCoarseStaticMaxDof];

// Device address of g_coarse_scratch on the current device, looked up once per
// device (the first call on a device does the lookup; it should come before any
// stream capture, since cudaGetSymbolAddress may initialise the module).
static int coarse_scratch_address(double** out, std::string& err) {
  constexpr int kMaxDevices = 64;
  static std::mutex mu;
  static double* addr[kMaxDevices] = {};
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) {
    err = std::string("cudaGetDevice: ") + cudaGetErrorString(e);
    return PMG_ECUDA;
  }
  if (dev < 0 || dev >= kMaxDevices) {
    err = "device ordinal out of range for the static coarse scratch";
    return PMG_EINVAL;
  }
  std::lock_guard<std::mutex> lock(mu);
  if (!addr[dev]) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_coarse_scratch);
    if (e != cudaSuccess || !p) {
      err = std::string("cudaGetSymbolAddress(g_coarse_scratch): ") + cudaGetErrorString(e);
      return PMG_ECUDA;
    }
    addr[dev] = static_cast<double*>(p);
  }
  *out = addr[dev];
  return PMG_OK;
}

}  // namespace pmg

extern "C" int pmg_coarse_solve_static(pmg_hier hh, const double* f0, double* u0, void* stream) {
  using namespace pmg;
  Hier* h = reinterpret_cast<Hier*>(hh);
  if (!h || !f0 || !u0) return PMG_EINVAL;
  const long long n = h->dims[0].ndof;
  if (n > kCoarseStaticMaxDof) {
    h->err = "pmg_coarse_solve_static: the coarse problem has " + std::to_string(n) +
             " unknowns; the static scratch holds at most " + std::to_string(kCoarseStaticMaxDof);
    return PMG_EINVAL;
  }
  double* scratch = nullptr;
  int rc = coarse_scratch_address(&scratch, h->err);
  if (rc != PMG_OK) return rc;
  // Every pass of the coarse solve writes all n entries of its output vector before
  // the next pass reads it, so the stale contents left by an earlier call never need
  // clearing.
  CoarseFdm c = h->coarse;
  c.tmp[0] = scratch;
  c.tmp[1] = scratch + kCoarseStaticMaxDof;
  rc = launch_coarse_fdm(h->dims[0], c, f0, u0, (cudaStream_t)stream);
  if (rc != PMG_OK) {
    // take the launch error out of the runtime's sticky slot, so that a later call
    // does not report it as its own
    const cudaError_t e = cudaGetLastError();
    h->err = std::string("pmg_coarse_solve_static: kernel launch failed: ") + cudaGetErrorString(e);
  }
  return rc;
}
