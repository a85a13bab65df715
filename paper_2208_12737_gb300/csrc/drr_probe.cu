// Read-bandwidth probe: the denominator of the gather roofline.  The walk's
// voxel gathers are served from L2 (the volume stays resident), so their
// ceiling is the rate at which all SMs can read an L2-resident buffer; this
// kernel measures it by streaming such a buffer with 16-byte loads.  No
// counterpart in the paper: it exists to put the gather rate in context.
#include <cuda_runtime.h>

#include "drr.h"
#include "drr_internal.cuh"

namespace {

__global__ void __launch_bounds__(256) l2_read_kernel(const float4* __restrict__ buf, size_t n4, int reps,
                                                      float* __restrict__ sink) {
  float acc = 0.f;
  const size_t stride = static_cast<size_t>(gridDim.x) * blockDim.x;
  for (int r = 0; r < reps; ++r) {
    for (size_t i = static_cast<size_t>(blockIdx.x) * blockDim.x + threadIdx.x; i < n4; i += stride) {
      const float4 v = __ldcg(buf + i);  // cached in L2 only: every pass is an L2 read
      acc += (v.x + v.y) + (v.z + v.w);
    }
  }
  if (acc == 1.2345678e-30f) sink[0] = acc;  // keeps the loads; never taken for the probe's zero buffer
}

}  // namespace

extern "C" drr_status drr_probe_l2_read(const void* buf_dev, size_t bytes, int32_t reps, float* sink_dev,
                                        void* cuda_stream) {
  if (!buf_dev || !sink_dev || bytes < 16 || reps <= 0) return drr::set_error(DRR_ERR_INVALID, "bad probe arguments");
  if (reinterpret_cast<uintptr_t>(buf_dev) % 16 != 0) return drr::set_error(DRR_ERR_INVALID, "buffer not 16-byte aligned");
  int dev = drr::current_device(), sms = 0;
  if (drr_status s = drr::device_view(buf_dev, dev, false, "buf", &buf_dev)) return s;  // an L2 probe: device memory
  if (drr_status s = drr::device_view(sink_dev, dev, true, "sink", &sink_dev)) return s;
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const int grid = (sms > 0 ? sms : 1) * 8;
  l2_read_kernel<<<grid, 256, 0, static_cast<cudaStream_t>(cuda_stream)>>>(static_cast<const float4*>(buf_dev),
                                                                           bytes / 16, reps, sink_dev);
  const cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return drr::cuda_error(e, "probe launch");
  drr::count_launches(1);
  return DRR_OK;
}
