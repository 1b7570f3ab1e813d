// noalloc.cu -- one diffusion step for callers that cannot allocate device memory.
//
// The regular path keeps its scratch (the per-block FP64 partial sums of the mass total) in memory
// that bdm_create allocates.  Some callers cannot allocate at all: a host application that owns
// every byte of device memory through its own pool, code that runs while another framework is
// capturing a CUDA graph on the same device, or latency-critical loops where the implicit
// synchronisation of cudaMalloc/cudaFree is not acceptable.  bdm_diffusion_step_noalloc serves them:
// the caller passes the input and output grids (and an optional mass slot) in memory it already
// owns, and the scratch lives in a fixed-size array in the library's own device image.
//
// That array is shared by every call on a device and keeps the last call's contents; two calls
// that overlap on the GPU (different streams, no ordering between them) race on it.  Every block
// writes its own partial before the mass kernel reads it, so nothing needs clearing between calls.
#include <cuda_runtime.h>

#include <cmath>
#include <mutex>

#include "bdm.h"
#include "common.cuh"

namespace bdm {
// Largest number of FTCS blocks (32 x 8 x 16 voxels each) one call may use: 65,536 FP64 partials,
// 512 KB of device memory held by every GPU that loads the library, until the process exits.
constexpr int kNoAllocMaxPartials = 65536;
static __device__ __align__(256) double g_noalloc_partials[kNoAllocMaxPartials];
}  // namespace bdm

namespace {
constexpr int kMaxDevices = 64;
std::mutex g_setup_mu;
void* g_partials_ptr[kMaxDevices] = {};

// Device address of the static scratch array for the current device; looked up once per device (in
// its primary context, which is what the runtime API makes current) and kept for the life of the
// process.  The address is not valid after cudaDeviceReset or in another context.
cudaError_t scratch_address(void** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lock(g_setup_mu);
  if (!g_partials_ptr[dev]) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, bdm::g_noalloc_partials);
    if (e != cudaSuccess) return e;
    g_partials_ptr[dev] = p;
  }
  *out = g_partials_ptr[dev];
  return cudaSuccess;
}
}  // namespace

extern "C" int bdm_diffusion_step_noalloc(const float* u, float* out, const int32_t grid_n[3],
                                          double diffusion_coeff, double dt_diffusion,
                                          double voxel, double decay, double* mass,
                                          void* stream) {
  if (!u || !out || !grid_n || u == out) return BDM_EINVAL;
  for (int a = 0; a < 3; ++a)
    if (grid_n[a] <= 0) return BDM_EINVAL;
  if (!(voxel > 0.0) || !(diffusion_coeff >= 0.0) || !(dt_diffusion >= 0.0) || !(decay >= 0.0))
    return BDM_EINVAL;
  const double lam = (diffusion_coeff * dt_diffusion) / (voxel * voxel);
  if (lam > 1.0 / 6.0 || decay * dt_diffusion > 1.0) return BDM_EINVAL;
  const int dims[3] = {grid_n[0], grid_n[1], grid_n[2]};
  // block count in 64-bit arithmetic (no wrap-around for huge extents), within the launch limits
  if (!bdm::ftcs_launchable(dims) || bdm::ftcs_partials_needed(dims) > bdm::kNoAllocMaxPartials)
    return BDM_EINVAL;
  void* partials = nullptr;
  if (scratch_address(&partials) != cudaSuccess) {
    cudaGetLastError();
    return BDM_ECUDA;
  }
  bdm::launch_ftcs_mass_to((cudaStream_t)stream, u, out, dims, (float)lam,
                           (float)(decay * dt_diffusion), (double*)partials, mass);
  return cudaGetLastError() == cudaSuccess ? BDM_OK : BDM_ECUDA;
}
