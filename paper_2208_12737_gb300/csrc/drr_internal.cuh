// Internal types shared by the libdrr kernels and the C-ABI layer.
// Nothing here is part of the public ABI (include/drr.h is).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <atomic>

#include "drr.h"

namespace drr {

// Pixel tiling of the ray kernels: the work unit is a warp tile of
// kWarpTileW x kWarpTileH pixels (8 x 4 by default), so that a warp's 32 rays
// are spatial neighbours and their voxel gathers share cache lines; warps of
// 256-thread blocks claim tiles from a counter.
#ifndef DRR_WARP_TILE_W
#define DRR_WARP_TILE_W 8
#endif
constexpr int kThreads = 256;
constexpr int kWarpTileW = DRR_WARP_TILE_W;
constexpr int kWarpTileH = 32 / kWarpTileW;
static_assert(kWarpTileW >= 4 && kWarpTileW <= 32 && 32 % kWarpTileW == 0, "warp tile width");
// The back-projection walks 4 x 8 pixel tiles instead: its atomic adds are
// merged down the tile's columns, and longer columns merge more (rays a pixel
// apart along h often cross the same voxel).
#ifndef DRR_BP_TILE_W
#define DRR_BP_TILE_W 4
#endif
constexpr int kBpTileW = DRR_BP_TILE_W;
static_assert(kBpTileW >= 1 && kBpTileW <= 32 && 32 % kBpTileW == 0, "back-projection tile width");

// Tile counters of the walk kernels, kept in the geometry buffer right after the
// last pose's PoseGeom and zeroed by the pose-setup kernel.
constexpr int kLaunchCounters = 4;

enum StorageType : int { kF32 = 0, kBF16 = 1, kF16 = 2 };

// Per-pose ray geometry (Sec. 2.4), written by the pose-setup kernel.
// Positions and directions are in voxel-index units of the volume:
// u = (x - b) / delta per axis, so voxel i spans [i, i+1).
struct PoseGeom {
  double u0[3];   // source position u(s)
  double un[3];   // n_a - u0[a] (distance of the far face, voxel units)
  double g00[3];  // direction (p - s) / delta at pixel (h=0, w=0)
  double gw[3];   // change of the direction per detector column
  double gh[3];   // change of the direction per detector row
  float u0f[3];   // FP32 copies of u0, un for the coarse clip
  float unf[3];
  // Chain-rule terms for the pose Jacobian, world units (mm), j = angle index:
  float Om[3][3];  // omega_j: dR/d eta_j R^T x = omega_j x x (the angle's angular velocity)
  float t[3];      // the pose translation
  float Q[3][3];   // dR/d eta_j * (p_c(0,0) - s_c)
  float Wv[3][3];  // dR/d eta_j * (0, dw, 0)
  float Hv[3][3];  // dR/d eta_j * (0, 0, dh)
  // Chain-rule terms for the detector parameters: the columns of R (R e_x,
  // R e_y, R e_z), and the detector centre indices (H-1)/2, (W-1)/2.
  float Rc[3][3];
  float hc, wc;
};

// A device-resident volume as the kernels see it.
struct VolumeDev {
  const void* data;  // storage (padded: one zero voxel on each side of every axis)
  int n[3];          // logical voxel counts nx, ny, nz
  float delta[3];    // spacing (mm)
  int dtype;         // StorageType
  float out_scale;   // E multiplier undoing the storage scale (FP16)
  int stride[3];     // element strides of the padded layout along x, y, z
  int origin;        // element offset of voxel (0,0,0)
  int64_t elems;     // padded element count
};

struct DetDev {
  int H, W;
  float sdr, dh, dw;
};

// Warp tiles (kWarpTileW x kWarpTileH pixels) per pose: the work units of the walk kernels.
__host__ __device__ __forceinline__ int pose_tiles(const DetDev& det) {
  return ((det.W + kWarpTileW - 1) / kWarpTileW) * ((det.H + kWarpTileH - 1) / kWarpTileH);
}

// Warp tiles per pose of the back-projection.
__host__ __device__ __forceinline__ int bp_pose_tiles(const DetDev& det) {
  return ((det.W + kBpTileW - 1) / kBpTileW) * ((det.H + 32 / kBpTileW - 1) / (32 / kBpTileW));
}

// One admitted request as the serving kernels see it (device-resident table).
struct ServeRequest {
  VolumeDev vd;
  DetDev det;
  const float* poses;  // [B][6]
  const float* grad;   // [B][H][W] upstream gradient, or null for render-only requests
  float* out;          // [B][H][W]
  float* partials;     // [B][tiles per pose][6] (gradient requests)
  float* grad_pose;    // [B][6] (gradient requests)
  PoseGeom* geom;      // [B]
  int B;
  int tile_start;      // first warp tile of this request in the tick's global tile numbering
  int pose_start;      // first pose of this request in the tick's global pose numbering
  int pad_;
};

struct ServeHeader {
  int nreq;
  int total_tiles;
  int total_poses;
  int pad_;
};

// Per-request device status words of a serving tick (one unsigned int per
// request, after the request table).  The host uploads them as zero; a kernel
// that meets an inconsistency it can detect sets a bit instead of touching
// memory, and the host returns DRR_ERR_DEVICE for that request.
enum ServeStatusBits : unsigned int {
  kServeTileRange = 1u,  // a tile decoded to a pose index outside its request
  kServePoseRange = 2u,  // a tick pose index decoded outside its request
};

// Launchers (drr_kernels.cu).  All enqueue on `stream` and return the
// cudaGetLastError() of the launch.
cudaError_t launch_pose_setup(const float* poses, int B, const DetDev& det, const VolumeDev* vd, PoseGeom* out,
                              cudaStream_t stream);
cudaError_t launch_ray_setup(const float* poses, int B, const DetDev& det, float* rays, cudaStream_t stream);
// lanes: 1 = one lane per ray; 4 or 8 = the split walk (fused forward +
// Jacobian only), as render_split_lanes chooses for the launch.
cudaError_t launch_render(const VolumeDev& vd, const DetDev& det, const PoseGeom* pg, int B, float* out, float* jac,
                          cudaStream_t stream, int lanes = 1);
int render_split_lanes(const VolumeDev& vd, const DetDev& det, int B);
// Comparison baseline: the plain FP32 forward walk (out: [B][H][W]).
cudaError_t launch_render_plain_fp32(const VolumeDev& vd, const DetDev& det, const PoseGeom* pg, int B, float* out,
                                     cudaStream_t stream);
// Central-difference pose Jacobian from the 13 renders per pose of the plain
// FP32 comparison server (E13: [B][13][npix], render 0 at the pose, 1 + 2k and
// 2 + 2k at +h_k and -h_k of parameter k): out [B][npix] = render 0,
// jac [B][6][npix] = (E(+h_k) - E(-h_k)) / (2 h_k).
cudaError_t launch_plain_fd_finish(const float* E13, int B, int npix, float h_rot, float h_trans, float* out,
                                   float* jac, cudaStream_t stream);
// Negative ZNCC of B moving images against fixed images fixed_stride elements
// apart (0: one fixed image for all), and optionally d loss / d moving.
cudaError_t launch_zncc(const float* moving, const float* fixed, size_t fixed_stride, int B, int npix, float eps,
                        float* loss, float* grad, cudaStream_t stream);
// Pose gradient by re-tracing: one partial sum of g . J per warp tile
// (partials: B * pose_tiles(det) * 6 floats), then the fixed-order FP64
// finalize over nblk = pose_tiles(det) partials per pose.
cudaError_t launch_pose_grad_walk(const VolumeDev& vd, const DetDev& det, const PoseGeom* pg, int B,
                                  const float* grad_drr, float* partials, cudaStream_t stream);
cudaError_t launch_pose_grad_finalize(const float* partials, int B, int nblk, float* grad_pose, cudaStream_t stream);
// Pose gradient from a stored Jacobian [B][6][H][W]: one launch, no scratch
// memory (one thread-block cluster per pose), grad_pose [B][6] overwritten.
cudaError_t launch_pose_grad_from_jacobian(const DetDev& det, int B, const float* grad_drr, const float* jac,
                                           float* grad_pose, cudaStream_t stream);
// dL/d(sdr, dh, dw) per pose by a re-walk: partials must hold
// B * pose_tiles(det) * 3 floats; grad_geometry is [B][3].
cudaError_t launch_geometry_grad(const VolumeDev& vd, const DetDev& det, const PoseGeom* pg, int B,
                                 const float* grad_drr, float* partials, float* grad_geometry, cudaStream_t stream);
cudaError_t launch_count_segments(const VolumeDev& vd, const DetDev& det, const PoseGeom* pg, int B, int* counts,
                                  cudaStream_t stream);
cudaError_t launch_backproject(const VolumeDev& vd, const DetDev& det, const PoseGeom* pg, int B,
                               const float* grad_drr, float* grad_vol, cudaStream_t stream);
// Serving tick: pose setup over all poses of the tick, the persistent walk
// over all tiles (tiles claimed through *counter, which must be zero), and the
// fixed-order pose-gradient sums.  Grids are fixed so the three launches can be
// captured once in a CUDA graph; the counts are read from the device header.
int serve_walk_grid(int device);
cudaError_t launch_serve_tick(const ServeHeader* hdr, const ServeRequest* reqs, unsigned int* status, int* counter,
                              int max_poses, int walk_grid, cudaStream_t stream);
// Bounds-checked builds: the device fault word (0 in the product build, which
// has none), read and cleared; and whether this build checks.
cudaError_t read_and_clear_fault(unsigned int* bits);
bool bounds_checked();
// Volume ingest.
cudaError_t launch_abs_max(const void* src, int src_dtype, int64_t count, float mu_water, unsigned int* out_bits,
                           cudaStream_t stream);
cudaError_t launch_ingest(const void* src, int src_dtype, float mu_water, const VolumeDev& vd, void* dst,
                          float scale, cudaStream_t stream);

// ---- host-side helpers shared by the C-ABI files (drr_api.cu) -------------
drr_status set_error(drr_status st, const char* fmt, ...);
drr_status cuda_error(cudaError_t e, const char* what);
drr_status check_detector(const drr_detector* det, DetDev* out);
drr_status check_geometry(const VolumeDev& vd, const DetDev& det);
void configure_pool(int dev);
// The address under which the kernels may access buffer p on device dev:
// device (or managed) memory of dev as it is, or, where host_ok, mapped
// page-locked host memory; anything else is DRR_ERR_INVALID (drr_api.cu).
drr_status device_view(const void* p, int dev, bool host_ok, const char* what, const void** out);
template <typename T>
drr_status device_view(T* p, int dev, bool host_ok, const char* what, T** out) {
  const void* q = nullptr;
  if (drr_status s = device_view(static_cast<const void*>(p), dev, host_ok, what, &q)) return s;
  *out = static_cast<T*>(const_cast<void*>(q));
  return DRR_OK;
}
// The calling thread's current device (-1 if CUDA cannot say).
int current_device();
void count_launches(int n);  // kernel launches issued outside LaunchScope (serving ticks)

}  // namespace drr

// A device-resident volume (drr_volume_create).
struct drr_volume_s {
  void* storage = nullptr;
  size_t bytes = 0;
  int device = 0;
  int layout = DRR_LAYOUT_LINEAR_X;
  drr::VolumeDev vd{};
  std::atomic<int> refs{0};  // requests queued or running in servers
};
