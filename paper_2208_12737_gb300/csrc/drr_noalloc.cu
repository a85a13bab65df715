// Pose gradient from a stored Jacobian for callers that must not allocate
// device memory (drr_pose_grad_noalloc in include/drr.h).
//
// Some callers cannot call cudaMalloc / cudaMallocAsync at all: a host
// application that reserves its whole device-memory footprint at start-up and
// forbids later allocations (e.g. a guidance loop that must never fail or stall
// on the allocator mid-procedure), or a plugin whose host framework owns every
// device allocation.  drr_render_backward takes its per-block partial sums from
// the stream-ordered pool; this variant keeps them in a fixed array of device
// memory that lives in this library instead.
#include <cuda_runtime.h>

#include <mutex>

#include "drr.h"
#include "drr_internal.cuh"

namespace {

// 1 MiB of partial sums: B * ceil(H*W / 2048) * 6 floats must fit.
constexpr size_t kScratchFloats = size_t(1) << 18;
constexpr int kMaxDevices = 64;

// Every GPU that loads the library holds this array until the process exits.
__device__ __align__(256) float g_pose_grad_scratch[kScratchFloats];

std::mutex g_scratch_mu;
float* g_scratch_addr[kMaxDevices] = {};

// Device address of the array on the current device.  In host code the array's
// name is only a host-side stand-in, so the address is looked up once per
// device (with that device current) and cached.
drr_status scratch_address(float** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return drr::cuda_error(e, "cudaGetDevice");
  if (dev < 0 || dev >= kMaxDevices) return drr::set_error(DRR_ERR_INVALID, "device ordinal %d not supported", dev);
  std::lock_guard<std::mutex> lk(g_scratch_mu);
  if (!g_scratch_addr[dev]) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_pose_grad_scratch);
    if (e != cudaSuccess) return drr::cuda_error(e, "cudaGetSymbolAddress(pose-gradient scratch)");
    g_scratch_addr[dev] = static_cast<float*>(p);
  }
  *out = g_scratch_addr[dev];
  return DRR_OK;
}

}  // namespace

extern "C" drr_status drr_pose_grad_noalloc(const drr_detector* det, int32_t B, const float* grad_drr_dev,
                                            const float* jac_dev, float* grad_pose_dev, void* cuda_stream) {
  drr::DetDev dd;
  if (drr_status s = drr::check_detector(det, &dd)) return s;
  if (B <= 0 || B > 65535) return drr::set_error(DRR_ERR_INVALID, "B must be in [1, 65535]");
  if (!grad_drr_dev || !jac_dev || !grad_pose_dev) return drr::set_error(DRR_ERR_INVALID, "NULL pointer");
  const int nblk = drr::pose_grad_blocks(dd, true);
  const size_t need = size_t(B) * nblk * 6;
  if (need > kScratchFloats)
    return drr::set_error(DRR_ERR_INVALID,
                          "B * ceil(H*W/2048) * 6 = %zu partial sums exceed the fixed scratch of %zu; "
                          "split the batch or use drr_render_backward",
                          need, kScratchFloats);
  float* scratch = nullptr;
  if (drr_status s = scratch_address(&scratch)) return s;
  cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
  // Every partial sum is written before it is read, so nothing needs clearing.
  cudaError_t e = drr::launch_jac_reduce(dd, B, grad_drr_dev, jac_dev, scratch, st);
  if (e == cudaSuccess) e = drr::launch_pose_grad_finalize(scratch, B, nblk, grad_pose_dev, st);
  if (e != cudaSuccess) return drr::cuda_error(e, "drr_pose_grad_noalloc launch");
  drr::count_launches(2);
  return DRR_OK;
}
