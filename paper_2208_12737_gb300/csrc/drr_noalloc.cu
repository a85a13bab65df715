// Pose gradient from a stored Jacobian for callers that must not allocate
// device memory (drr_pose_grad_noalloc in include/drr.h).
//
// Some callers cannot call cudaMalloc / cudaMallocAsync at all: a host
// application that reserves its whole device-memory footprint at start-up and
// forbids later allocations (e.g. a guidance loop that must never fail or stall
// on the allocator mid-procedure), or a plugin whose host framework owns every
// device allocation.  The stored-Jacobian reduction keeps all of its partial
// sums on chip (one thread-block cluster per pose, distributed shared memory),
// so this entry point is the same single launch as drr_render_backward's
// stored-Jacobian path, without the volume handle and without any allocation.
#include <cuda_runtime.h>

#include "drr.h"
#include "drr_internal.cuh"

extern "C" drr_status drr_pose_grad_noalloc(const drr_detector* det, int32_t B, const float* grad_drr_dev,
                                            const float* jac_dev, float* grad_pose_dev, void* cuda_stream) {
  drr::DetDev dd;
  if (drr_status s = drr::check_detector(det, &dd)) return s;
  if (B <= 0 || B > 65535) return drr::set_error(DRR_ERR_INVALID, "B must be in [1, 65535]");
  if (!grad_drr_dev || !jac_dev || !grad_pose_dev) return drr::set_error(DRR_ERR_INVALID, "NULL pointer");
  // (a pointer query, no allocation)
  const int dev = drr::current_device();
  if (drr_status s = drr::device_view(grad_drr_dev, dev, true, "grad_drr", &grad_drr_dev)) return s;
  if (drr_status s = drr::device_view(jac_dev, dev, true, "jac", &jac_dev)) return s;
  if (drr_status s = drr::device_view(grad_pose_dev, dev, true, "grad_pose", &grad_pose_dev)) return s;
  cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
  cudaError_t e = drr::launch_pose_grad_from_jacobian(dd, B, grad_drr_dev, jac_dev, grad_pose_dev, st);
  if (e != cudaSuccess) return drr::cuda_error(e, "drr_pose_grad_noalloc launch");
  drr::count_launches(1);
  return DRR_OK;
}
