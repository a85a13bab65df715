// libdrr C ABI (include/drr.h): argument checking, volume registry, scratch
// management and kernel launches.  No compute happens here.
#include <cuda_runtime.h>

#include <atomic>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <algorithm>
#include <cstring>
#include <mutex>
#include <string>
#include <vector>

#include "drr.h"
#include "drr_internal.cuh"

namespace {
thread_local std::string g_err;
}  // namespace

namespace drr {

drr_status set_error(drr_status st, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof(buf), fmt, ap);
  va_end(ap);
  g_err = buf;
  return st;
}

drr_status cuda_error(cudaError_t e, const char* what) {
  return set_error(e == cudaErrorMemoryAllocation ? DRR_ERR_OOM : DRR_ERR_CUDA, "%s: %s", what,
                   cudaGetErrorString(e));
}

}  // namespace drr

namespace {

using drr::check_detector;
using drr::check_geometry;
using drr::configure_pool;

#define DRR_CUDA(call, what)                  \
  do {                                        \
    cudaError_t e_ = (call);                  \
    if (e_ != cudaSuccess) return drr::cuda_error(e_, what); \
  } while (0)

}  // namespace

namespace drr {

// Stream-ordered scratch comes from the device's default memory pool; keep
// freed blocks cached in the pool instead of returning them to the driver.
std::once_flag g_pool_once[64];
void configure_pool(int dev) {
  if (dev < 0 || dev >= 64) return;
  std::call_once(g_pool_once[dev], [dev] {
    cudaMemPool_t pool;
    if (cudaDeviceGetDefaultMemPool(&pool, dev) == cudaSuccess) {
      uint64_t thr = UINT64_MAX;
      cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &thr);
    }
  });
}

// The address under which the kernels may access the buffer p of a call on
// the volume's device: device (or managed) memory of that device as it is, or,
// where host_ok, page-locked host memory mapped into the device's address
// space (the kernels then read or write it across the host link, and no
// staging copy is needed; under unified addressing the address is p itself).
// Anything else -- pageable host memory, another device's memory -- is
// DRR_ERR_INVALID here, before a kernel could fault on it.
drr_status device_view(const void* p, int dev, bool host_ok, const char* what, const void** out) {
  int cur = -1;
  if (cudaGetDevice(&cur) != cudaSuccess || cur != dev)
    return set_error(DRR_ERR_INVALID, "%s: the current device (%d) is not the volume's (%d)", what, cur, dev);
  cudaPointerAttributes a{};
  const cudaError_t e = cudaPointerGetAttributes(&a, p);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return set_error(DRR_ERR_INVALID, "%s: not an address CUDA knows (%s)", what, cudaGetErrorString(e));
  }
  if (a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged) {
    if (a.type == cudaMemoryTypeDevice && a.device != dev)
      return set_error(DRR_ERR_INVALID, "%s is on device %d, the volume on device %d", what, a.device, dev);
    *out = p;
    return DRR_OK;
  }
  if (a.type == cudaMemoryTypeHost) {
    if (!host_ok) return set_error(DRR_ERR_INVALID, "%s must be device memory", what);
    if (!a.devicePointer)
      return set_error(DRR_ERR_INVALID, "%s: page-locked host memory not mapped for device %d", what, dev);
    *out = a.devicePointer;
    return DRR_OK;
  }
  return set_error(DRR_ERR_INVALID, "%s: pageable host memory (pin it, or copy it to the device)", what);
}


int current_device() {
  int d = -1;
  if (cudaGetDevice(&d) != cudaSuccess) return -1;
  return d;
}

drr_status check_detector(const drr_detector* det, drr::DetDev* out) {
  if (!det) return drr::set_error(DRR_ERR_INVALID, "detector is NULL");
  if (det->height <= 0 || det->width <= 0) return drr::set_error(DRR_ERR_INVALID, "detector size must be positive");
  if (!(det->sdr_mm > 0.f) || !(det->delta_h_mm > 0.f) || !(det->delta_w_mm > 0.f) || !std::isfinite(det->sdr_mm) ||
      !std::isfinite(det->delta_h_mm) || !std::isfinite(det->delta_w_mm))
    return drr::set_error(DRR_ERR_INVALID, "detector distances must be positive and finite");
  if (static_cast<int64_t>(det->height) * det->width > (int64_t{1} << 30))
    return drr::set_error(DRR_ERR_INVALID, "detector has too many pixels");
  out->H = det->height;
  out->W = det->width;
  out->sdr = det->sdr_mm;
  out->dh = det->delta_h_mm;
  out->dw = det->delta_w_mm;
  return DRR_OK;
}

// The FP32 walk steps alpha by 1/|g| per plane; keep that step far above
// FP32 resolution (alpha <= 1): longest ray / smallest voxel < 2^20.
drr_status check_geometry(const drr::VolumeDev& vd, const drr::DetDev& det) {
  double hw = 0.5 * det.W * det.dw, hh = 0.5 * det.H * det.dh;
  double Lmax = std::sqrt(double(det.sdr) * det.sdr + hw * hw + hh * hh);
  double dmin = std::fmin(vd.delta[0], std::fmin(vd.delta[1], vd.delta[2]));
  if (Lmax / dmin >= double(1 << 20))
    return drr::set_error(DRR_ERR_INVALID, "ray length / voxel spacing too large (%.3g >= 2^20)", Lmax / dmin);
  return DRR_OK;
}

}  // namespace drr

namespace {

drr_status check_volume(drr_volume v) {
  if (!v || !v->storage) return drr::set_error(DRR_ERR_INVALID, "volume handle is NULL or destroyed");
  return DRR_OK;
}


template <typename T>
struct AsyncBuf {
  T* p = nullptr;
  cudaStream_t s = nullptr;
  ~AsyncBuf() {
    if (p) cudaFreeAsync(p, s);
  }
  cudaError_t alloc(size_t count, cudaStream_t stream) {
    s = stream;
    return cudaMallocAsync(reinterpret_cast<void**>(&p), count * sizeof(T), stream);
  }
};

// ---- kernel timing: CUDA events around each launch while enabled ----------
enum ProfKernel {
  kPoseSetup, kSiddonFwd, kSiddonFwdJac, kSiddonPoseGrad, kJacReduce, kFinalize, kBackproject, kCountSeg, kZncc,
  kSiddonGeoGrad, kPlainFp32, kSiddonFwdJacSplit, kNumProf
};
const char* const kProfNames[kNumProf] = {"pose_setup",        "siddon_fwd", "siddon_fwd_jac",     "siddon_pose_grad",
                                          "jac_reduce",        "pose_grad_finalize", "siddon_backproject",
                                          "count_segments",    "zncc",       "siddon_geometry_grad",
                                          "plain_fp32_fwd",    "siddon_fwd_jac_split"};
struct ProfRecord {
  int kernel;
  cudaEvent_t start, stop;
};
std::mutex g_prof_mu;
std::atomic<bool> g_prof_on{false};
std::vector<ProfRecord> g_prof_records;
std::vector<cudaEvent_t> g_event_pool;
std::atomic<int64_t> g_launches{0};

cudaEvent_t take_event() {
  if (!g_event_pool.empty()) {
    cudaEvent_t e = g_event_pool.back();
    g_event_pool.pop_back();
    return e;
  }
  cudaEvent_t e = nullptr;
  cudaEventCreate(&e);
  return e;
}

// Brackets exactly one kernel launch: counts it and, while profiling is on,
// records start/stop events on the launch stream.
struct LaunchScope {
  int kernel;
  cudaStream_t stream;
  cudaEvent_t start = nullptr;
  LaunchScope(int k, cudaStream_t s) : kernel(k), stream(s) {
    g_launches.fetch_add(1);
    if (g_prof_on.load()) {
      std::lock_guard<std::mutex> lk(g_prof_mu);
      start = take_event();
      if (start) cudaEventRecord(start, stream);
    }
  }
  ~LaunchScope() {
    if (!start) return;
    std::lock_guard<std::mutex> lk(g_prof_mu);
    cudaEvent_t stop = take_event();
    if (!stop) {
      g_event_pool.push_back(start);
      return;
    }
    cudaEventRecord(stop, stream);
    g_prof_records.push_back({kernel, start, stop});
  }
};

}  // namespace

void drr::count_launches(int n) { g_launches.fetch_add(n); }

namespace {

drr_status setup_geometry(drr_volume v, const drr::DetDev& dd, const float* poses_dev, int32_t B, cudaStream_t st,
                          AsyncBuf<drr::PoseGeom>& pg) {
  // one PoseGeom per pose plus one slot for the walk kernels' tile counters
  static_assert(sizeof(drr::PoseGeom) >= drr::kLaunchCounters * sizeof(unsigned int), "counter slot");
  if (int64_t(drr::pose_tiles(dd) > drr::bp_pose_tiles(dd) ? drr::pose_tiles(dd) : drr::bp_pose_tiles(dd)) * B >=
      (int64_t{1} << 31))
    return drr::set_error(DRR_ERR_INVALID, "too many rays in one call (B * pixels / 32 must stay below 2^31)");
  DRR_CUDA(pg.alloc(size_t(B) + 1, st), "cudaMallocAsync(pose geometry)");
  LaunchScope ls(kPoseSetup, st);
  DRR_CUDA(drr::launch_pose_setup(poses_dev, B, dd, &v->vd, pg.p, st), "pose_setup launch");
  return DRR_OK;
}

}  // namespace

extern "C" {

drr_status drr_profile_enable(int32_t on) {
  g_prof_on.store(on != 0);
  return DRR_OK;
}

drr_status drr_profile_reset(void) {
  std::lock_guard<std::mutex> lk(g_prof_mu);
  for (auto& r : g_prof_records) {
    cudaEventSynchronize(r.stop);
    g_event_pool.push_back(r.start);
    g_event_pool.push_back(r.stop);
  }
  g_prof_records.clear();
  return DRR_OK;
}

drr_status drr_profile_read(const char* kernel, double* total_ms, int64_t* launches) {
  if (!kernel || !total_ms || !launches) return drr::set_error(DRR_ERR_INVALID, "NULL argument");
  int k = -1;
  for (int i = 0; i < kNumProf; ++i)
    if (std::strcmp(kernel, kProfNames[i]) == 0) k = i;
  if (k < 0) return drr::set_error(DRR_ERR_INVALID, "unknown kernel name '%s'", kernel);
  std::lock_guard<std::mutex> lk(g_prof_mu);
  double ms = 0.0;
  int64_t n = 0;
  for (auto& r : g_prof_records) {
    if (r.kernel != k) continue;
    DRR_CUDA(cudaEventSynchronize(r.stop), "cudaEventSynchronize");
    float t = 0.f;
    DRR_CUDA(cudaEventElapsedTime(&t, r.start, r.stop), "cudaEventElapsedTime");
    ms += t;
    ++n;
  }
  *total_ms = ms;
  *launches = n;
  return DRR_OK;
}

int64_t drr_launch_count(void) { return g_launches.load(); }

const char* drr_last_error(void) { return g_err.c_str(); }

const char* drr_version(void) { return "libdrr 0.1 (sm_103a)"; }

drr_status drr_volume_create(const void* data, int32_t data_on_device, drr_dtype src_dtype, int32_t nx, int32_t ny,
                             int32_t nz, float dx_mm, float dy_mm, float dz_mm, const drr_volume_options* opt,
                             void* cuda_stream, drr_volume* out) {
  if (!out) return drr::set_error(DRR_ERR_INVALID, "out is NULL");
  *out = nullptr;
  if (!data) return drr::set_error(DRR_ERR_INVALID, "data is NULL");
  if (src_dtype != DRR_F32 && src_dtype != DRR_I16_HU)
    return drr::set_error(DRR_ERR_INVALID, "src_dtype must be DRR_F32 or DRR_I16_HU");
  if (nx <= 0 || ny <= 0 || nz <= 0) return drr::set_error(DRR_ERR_INVALID, "volume dims must be positive");
  if (!(dx_mm > 0.f && dy_mm > 0.f && dz_mm > 0.f) || !std::isfinite(dx_mm) || !std::isfinite(dy_mm) ||
      !std::isfinite(dz_mm))
    return drr::set_error(DRR_ERR_INVALID, "voxel spacing must be positive and finite");
  const int64_t padded = (int64_t(nx) + 2) * (int64_t(ny) + 2) * (int64_t(nz) + 2);
  if (padded >= (int64_t{1} << 31)) return drr::set_error(DRR_ERR_INVALID, "volume too large (padded voxels >= 2^31)");
  drr_dtype storage = DRR_F32;
  float mu_water = 0.02f;
  int layout = DRR_LAYOUT_LINEAR_X;
  if (opt) {
    storage = opt->storage;
    if (opt->hu_mu_water != 0.f) mu_water = opt->hu_mu_water;
    if (opt->layout < 0 || opt->layout > DRR_LAYOUT_LINEAR_Z)
      return drr::set_error(DRR_ERR_INVALID, "layout %d not supported (0 .. 3)", opt->layout);
    if (opt->layout != 0) layout = opt->layout;
  }
  if (storage != DRR_F32 && storage != DRR_BF16 && storage != DRR_F16)
    return drr::set_error(DRR_ERR_INVALID, "storage dtype must be DRR_F32, DRR_BF16 or DRR_F16");
  if (!(mu_water > 0.f) || !std::isfinite(mu_water)) return drr::set_error(DRR_ERR_INVALID, "hu_mu_water must be positive");

  cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
  int dev = 0;
  DRR_CUDA(cudaGetDevice(&dev), "cudaGetDevice");
  configure_pool(dev);
  const int64_t count = int64_t(nx) * ny * nz;
  const size_t src_bytes = size_t(count) * (src_dtype == DRR_I16_HU ? 2 : 4);

  const void* src = data;
  void* staged = nullptr;
  if (data_on_device) {
    if (drr_status s = drr::device_view(data, dev, true, "data", &src)) return s;
  } else {
    DRR_CUDA(cudaMallocAsync(&staged, src_bytes, st), "cudaMallocAsync(volume staging)");
    cudaError_t e = cudaMemcpyAsync(staged, data, src_bytes, cudaMemcpyHostToDevice, st);
    if (e != cudaSuccess) {
      cudaFreeAsync(staged, st);
      return drr::cuda_error(e, "cudaMemcpyAsync(volume upload)");
    }
    src = staged;
  }
  auto cleanup = [&] {
    if (staged) cudaFreeAsync(staged, st);
    cudaStreamSynchronize(st);
  };

  drr_volume v = new drr_volume_s();
  v->device = dev;
  drr::VolumeDev& vd = v->vd;
  vd.n[0] = nx;
  vd.n[1] = ny;
  vd.n[2] = nz;
  vd.delta[0] = dx_mm;
  vd.delta[1] = dy_mm;
  vd.delta[2] = dz_mm;
  vd.dtype = storage == DRR_F32 ? drr::kF32 : storage == DRR_BF16 ? drr::kBF16 : drr::kF16;
  {
    // padded linear storage, the layout's axis fastest, the other two in x, y, z order
    const int fast = layout - DRR_LAYOUT_LINEAR_X;
    const int order[3] = {fast, fast == 0 ? 1 : 0, fast == 2 ? 1 : 2};
    int stride = 1;
    for (int q = 0; q < 3; ++q) {
      vd.stride[order[q]] = stride;
      stride *= vd.n[order[q]] + 2;
    }
  }
  v->layout = layout;
  vd.origin = vd.stride[2] + vd.stride[1] + vd.stride[0];
  vd.elems = padded;
  vd.out_scale = 1.f;

  float scale = 1.f;
  cudaError_t e = cudaSuccess;
  if (vd.dtype == drr::kF16) {
    unsigned int* bits = nullptr;
    e = cudaMallocAsync(reinterpret_cast<void**>(&bits), sizeof(unsigned int), st);
    if (e == cudaSuccess) e = cudaMemsetAsync(bits, 0, sizeof(unsigned int), st);
    if (e == cudaSuccess) e = drr::launch_abs_max(src, src_dtype == DRR_I16_HU ? 3 : 0, count, mu_water, bits, st);
    unsigned int hbits = 0;
    if (e == cudaSuccess) e = cudaMemcpyAsync(&hbits, bits, sizeof(unsigned int), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (bits) cudaFreeAsync(bits, st);
    if (e != cudaSuccess) {
      cleanup();
      delete v;
      return drr::cuda_error(e, "volume max for FP16 scale");
    }
    float mx;
    std::memcpy(&mx, &hbits, 4);
    if (mx > 0.f && std::isfinite(mx)) {
      int ex = 0;
      std::frexp(double(mx), &ex);  // mx = m 2^ex, m in [0.5, 1)
      scale = float(std::ldexp(1.0, 14 - ex));
    }
    vd.out_scale = 1.f / scale;
  }
  const size_t elem = vd.dtype == drr::kF32 ? 4 : 2;
  v->bytes = size_t(padded) * elem;
  e = cudaMalloc(&v->storage, v->bytes);
  if (e != cudaSuccess) {
    cleanup();
    delete v;
    return drr::cuda_error(e, "cudaMalloc(volume storage)");
  }
  vd.data = v->storage;
  e = drr::launch_ingest(src, src_dtype == DRR_I16_HU ? 3 : 0, mu_water, vd, v->storage, scale, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  cleanup();
  if (e != cudaSuccess) {
    cudaFree(v->storage);
    delete v;
    return drr::cuda_error(e, "volume ingest");
  }
  *out = v;
  return DRR_OK;
}

drr_status drr_volume_destroy(drr_volume v) {
  if (!v) return DRR_OK;
  if (v->refs.load() > 0) return drr::set_error(DRR_ERR_BUSY, "volume is still referenced by %d server(s)", v->refs.load());
  if (v->storage) {
    int cur = 0;
    cudaGetDevice(&cur);
    if (cur != v->device) cudaSetDevice(v->device);
    cudaFree(v->storage);
    if (cur != v->device) cudaSetDevice(cur);
  }
  delete v;
  return DRR_OK;
}

drr_status drr_volume_info(drr_volume v, int32_t dims[3], float spacing[3], drr_dtype* storage, float* storage_scale,
                           size_t* device_bytes) {
  if (drr_status s = check_volume(v)) return s;
  for (int a = 0; a < 3; ++a) {
    if (dims) dims[a] = v->vd.n[a];
    if (spacing) spacing[a] = v->vd.delta[a];
  }
  if (storage) *storage = v->vd.dtype == drr::kF32 ? DRR_F32 : v->vd.dtype == drr::kBF16 ? DRR_BF16 : DRR_F16;
  if (storage_scale) *storage_scale = 1.f / v->vd.out_scale;
  if (device_bytes) *device_bytes = v->bytes;
  return DRR_OK;
}

drr_status drr_ray_setup(const drr_detector* det, const float* poses_dev, int32_t B, float* rays_out_dev,
                         void* cuda_stream) {
  drr::DetDev dd;
  if (drr_status s = check_detector(det, &dd)) return s;
  if (B <= 0) return drr::set_error(DRR_ERR_INVALID, "B must be positive");
  if (!poses_dev || !rays_out_dev) return drr::set_error(DRR_ERR_INVALID, "NULL pointer");
  const int dev = drr::current_device();
  if (drr_status s = drr::device_view(poses_dev, dev, true, "poses", &poses_dev)) return s;
  if (drr_status s = drr::device_view(rays_out_dev, dev, true, "rays_out", &rays_out_dev)) return s;
  LaunchScope ls(kPoseSetup, static_cast<cudaStream_t>(cuda_stream));
  DRR_CUDA(drr::launch_ray_setup(poses_dev, B, dd, rays_out_dev, static_cast<cudaStream_t>(cuda_stream)),
           "ray_setup launch");
  return DRR_OK;
}

drr_status drr_render(drr_volume v, const drr_detector* det, const float* poses_dev, int32_t B, float* drr_out_dev,
                      float* jac_out_dev, void* cuda_stream) {
  if (drr_status s = check_volume(v)) return s;
  drr::DetDev dd;
  if (drr_status s = check_detector(det, &dd)) return s;
  if (drr_status s = check_geometry(v->vd, dd)) return s;
  if (B <= 0) return drr::set_error(DRR_ERR_INVALID, "B must be positive");
  if (B > 65535) return drr::set_error(DRR_ERR_INVALID, "B must be <= 65535");
  if (!poses_dev || !drr_out_dev) return drr::set_error(DRR_ERR_INVALID, "NULL pointer");
  if (drr_status s = drr::device_view(poses_dev, v->device, true, "poses", &poses_dev)) return s;
  if (drr_status s = drr::device_view(drr_out_dev, v->device, true, "drr_out", &drr_out_dev)) return s;
  if (jac_out_dev) {
    if (drr_status s = drr::device_view(jac_out_dev, v->device, true, "jac_out", &jac_out_dev)) return s;
  }
  cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
  configure_pool(v->device);
  AsyncBuf<drr::PoseGeom> pg;
  if (drr_status s = setup_geometry(v, dd, poses_dev, B, st, pg)) return s;
  const int lanes = jac_out_dev ? drr::render_split_lanes(v->vd, dd, B) : 1;
  LaunchScope ls(jac_out_dev ? (lanes > 1 ? kSiddonFwdJacSplit : kSiddonFwdJac) : kSiddonFwd, st);
  DRR_CUDA(drr::launch_render(v->vd, dd, pg.p, B, drr_out_dev, jac_out_dev, st, lanes), "render launch");
  return DRR_OK;
}

drr_status drr_render_backward(drr_volume v, const drr_detector* det, const float* poses_dev, int32_t B,
                               const float* grad_drr_dev, const float* jac_dev, float* grad_pose_dev,
                               float* grad_volume_dev, void* cuda_stream) {
  if (drr_status s = check_volume(v)) return s;
  drr::DetDev dd;
  if (drr_status s = check_detector(det, &dd)) return s;
  if (drr_status s = check_geometry(v->vd, dd)) return s;
  if (B <= 0) return drr::set_error(DRR_ERR_INVALID, "B must be positive");
  if (B > 65535) return drr::set_error(DRR_ERR_INVALID, "B must be <= 65535");
  if (!poses_dev || !grad_drr_dev) return drr::set_error(DRR_ERR_INVALID, "NULL pointer");
  if (!grad_pose_dev && !grad_volume_dev)
    return drr::set_error(DRR_ERR_INVALID, "nothing to compute: grad_pose_dev and grad_volume_dev are both NULL");
  if (drr_status s = drr::device_view(poses_dev, v->device, true, "poses", &poses_dev)) return s;
  if (drr_status s = drr::device_view(grad_drr_dev, v->device, true, "grad_drr", &grad_drr_dev)) return s;
  if (jac_dev) {
    if (drr_status s = drr::device_view(jac_dev, v->device, true, "jac", &jac_dev)) return s;
  }
  if (grad_pose_dev) {
    if (drr_status s = drr::device_view(grad_pose_dev, v->device, true, "grad_pose", &grad_pose_dev)) return s;
  }
  if (grad_volume_dev) {  // atomics into host memory would cross the host link per add: device memory only
    if (drr_status s = drr::device_view(grad_volume_dev, v->device, false, "grad_volume", &grad_volume_dev)) return s;
  }
  cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
  configure_pool(v->device);
  AsyncBuf<drr::PoseGeom> pg;
  const bool need_geom = grad_volume_dev || (grad_pose_dev && !jac_dev);
  if (need_geom) {
    if (drr_status s = setup_geometry(v, dd, poses_dev, B, st, pg)) return s;
  }
  if (grad_pose_dev && jac_dev) {
    LaunchScope ls(kJacReduce, st);
    DRR_CUDA(drr::launch_pose_grad_from_jacobian(dd, B, grad_drr_dev, jac_dev, grad_pose_dev, st),
             "pose-gradient launch");
  } else if (grad_pose_dev) {
    const int nblk = drr::pose_tiles(dd);
    AsyncBuf<float> partials;
    DRR_CUDA(partials.alloc(size_t(B) * nblk * 6, st), "cudaMallocAsync(pose-gradient partials)");
    {
      LaunchScope ls(kSiddonPoseGrad, st);
      DRR_CUDA(drr::launch_pose_grad_walk(v->vd, dd, pg.p, B, grad_drr_dev, partials.p, st), "pose-gradient launch");
    }
    LaunchScope ls(kFinalize, st);
    DRR_CUDA(drr::launch_pose_grad_finalize(partials.p, B, nblk, grad_pose_dev, st), "pose-gradient finalize");
  }
  if (grad_volume_dev) {
    LaunchScope ls(kBackproject, st);
    DRR_CUDA(drr::launch_backproject(v->vd, dd, pg.p, B, grad_drr_dev, grad_volume_dev, st), "backproject launch");
  }
  return DRR_OK;
}

drr_status drr_count_segments(drr_volume v, const drr_detector* det, const float* poses_dev, int32_t B,
                              int32_t* segments_out_dev, void* cuda_stream) {
  if (drr_status s = check_volume(v)) return s;
  drr::DetDev dd;
  if (drr_status s = check_detector(det, &dd)) return s;
  if (drr_status s = check_geometry(v->vd, dd)) return s;
  if (B <= 0 || B > 65535) return drr::set_error(DRR_ERR_INVALID, "B must be in [1, 65535]");
  if (!poses_dev || !segments_out_dev) return drr::set_error(DRR_ERR_INVALID, "NULL pointer");
  if (drr_status s = drr::device_view(poses_dev, v->device, true, "poses", &poses_dev)) return s;
  if (drr_status s = drr::device_view(segments_out_dev, v->device, true, "segments_out", &segments_out_dev)) return s;
  cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
  configure_pool(v->device);
  AsyncBuf<drr::PoseGeom> pg;
  if (drr_status s = setup_geometry(v, dd, poses_dev, B, st, pg)) return s;
  LaunchScope ls(kCountSeg, st);
  DRR_CUDA(drr::launch_count_segments(v->vd, dd, pg.p, B, segments_out_dev, st), "count_segments launch");
  return DRR_OK;
}

drr_status drr_render_plain_fp32(drr_volume v, const drr_detector* det, const float* poses_dev, int32_t B,
                                 float* drr_out_dev, void* cuda_stream) {
  if (drr_status s = check_volume(v)) return s;
  drr::DetDev dd;
  if (drr_status s = check_detector(det, &dd)) return s;
  if (drr_status s = check_geometry(v->vd, dd)) return s;
  if (B <= 0 || B > 65535) return drr::set_error(DRR_ERR_INVALID, "B must be in [1, 65535]");
  if (!poses_dev || !drr_out_dev) return drr::set_error(DRR_ERR_INVALID, "NULL pointer");
  if (drr_status s = drr::device_view(poses_dev, v->device, true, "poses", &poses_dev)) return s;
  if (drr_status s = drr::device_view(drr_out_dev, v->device, true, "drr_out", &drr_out_dev)) return s;
  cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
  configure_pool(v->device);
  AsyncBuf<drr::PoseGeom> pg;
  if (drr_status s = setup_geometry(v, dd, poses_dev, B, st, pg)) return s;
  LaunchScope ls(kPlainFp32, st);
  DRR_CUDA(drr::launch_render_plain_fp32(v->vd, dd, pg.p, B, drr_out_dev, st), "plain FP32 render launch");
  return DRR_OK;
}

drr_status drr_geometry_grad(drr_volume v, const drr_detector* det, const float* poses_dev, int32_t B,
                             const float* grad_drr_dev, float* grad_geometry_dev, void* cuda_stream) {
  if (drr_status s = check_volume(v)) return s;
  drr::DetDev dd;
  if (drr_status s = check_detector(det, &dd)) return s;
  if (drr_status s = check_geometry(v->vd, dd)) return s;
  if (B <= 0 || B > 65535) return drr::set_error(DRR_ERR_INVALID, "B must be in [1, 65535]");
  if (!poses_dev || !grad_drr_dev || !grad_geometry_dev) return drr::set_error(DRR_ERR_INVALID, "NULL pointer");
  if (drr_status s = drr::device_view(poses_dev, v->device, true, "poses", &poses_dev)) return s;
  if (drr_status s = drr::device_view(grad_drr_dev, v->device, true, "grad_drr", &grad_drr_dev)) return s;
  if (drr_status s = drr::device_view(grad_geometry_dev, v->device, true, "grad_geometry", &grad_geometry_dev))
    return s;
  cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
  configure_pool(v->device);
  AsyncBuf<drr::PoseGeom> pg;
  if (drr_status s = setup_geometry(v, dd, poses_dev, B, st, pg)) return s;
  AsyncBuf<float> partials;
  DRR_CUDA(partials.alloc(size_t(B) * drr::pose_tiles(dd) * 3, st), "cudaMallocAsync(geometry-gradient partials)");
  LaunchScope ls(kSiddonGeoGrad, st);
  DRR_CUDA(drr::launch_geometry_grad(v->vd, dd, pg.p, B, grad_drr_dev, partials.p, grad_geometry_dev, st),
           "geometry-gradient launch");
  drr::count_launches(1);  // the finalize launch
  return DRR_OK;
}

drr_status drr_loss_landscape(drr_volume v, const drr_detector* det, const float* fixed_dev, const float* poses_dev,
                              int32_t N, float eps, float* loss_out_dev, int32_t chunk, void* cuda_stream) {
  if (drr_status s = check_volume(v)) return s;
  drr::DetDev dd;
  if (drr_status s = check_detector(det, &dd)) return s;
  if (drr_status s = check_geometry(v->vd, dd)) return s;
  if (N <= 0) return drr::set_error(DRR_ERR_INVALID, "N must be positive");
  if (chunk < 0) return drr::set_error(DRR_ERR_INVALID, "chunk must be >= 0");
  if (!(eps >= 0.f)) return drr::set_error(DRR_ERR_INVALID, "eps must be >= 0");
  if (!fixed_dev || !poses_dev || !loss_out_dev) return drr::set_error(DRR_ERR_INVALID, "NULL pointer");
  if (drr_status s = drr::device_view(fixed_dev, v->device, true, "fixed", &fixed_dev)) return s;
  if (drr_status s = drr::device_view(poses_dev, v->device, true, "poses", &poses_dev)) return s;
  if (drr_status s = drr::device_view(loss_out_dev, v->device, true, "loss_out", &loss_out_dev)) return s;
  const int64_t npix = int64_t(dd.H) * dd.W;
  if (chunk == 0) chunk = int32_t(std::max<int64_t>(1, std::min<int64_t>(4096, (int64_t{256} << 20) / (4 * npix))));
  chunk = std::min(chunk, std::min<int32_t>(N, 65535));
  cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
  configure_pool(v->device);
  AsyncBuf<float> E;
  DRR_CUDA(E.alloc(size_t(chunk) * npix, st), "cudaMallocAsync(landscape DRRs)");
  for (int32_t i = 0; i < N; i += chunk) {
    const int32_t c = std::min(chunk, N - i);
    AsyncBuf<drr::PoseGeom> pg;
    if (drr_status s = setup_geometry(v, dd, poses_dev + 6 * size_t(i), c, st, pg)) return s;
    {
      LaunchScope ls(kSiddonFwd, st);
      DRR_CUDA(drr::launch_render(v->vd, dd, pg.p, c, E.p, nullptr, st), "landscape render launch");
    }
    LaunchScope ls(kZncc, st);
    DRR_CUDA(drr::launch_zncc(E.p, fixed_dev, 0, c, int(npix), eps, loss_out_dev + i, nullptr, st),
             "landscape zncc launch");
  }
  return DRR_OK;
}

drr_status drr_stream_check(void* cuda_stream) {
  cudaError_t e = cudaStreamSynchronize(static_cast<cudaStream_t>(cuda_stream));
  if (e != cudaSuccess) return drr::cuda_error(e, "stream");
  e = cudaGetLastError();
  if (e != cudaSuccess) return drr::cuda_error(e, "pending error");
  unsigned int bits = 0u;
  e = drr::read_and_clear_fault(&bits);
  if (e != cudaSuccess) return drr::cuda_error(e, "fault word");
  if (bits)
    return drr::set_error(DRR_ERR_DEVICE, "a bounds check failed in a kernel (fault bits 0x%x: 1 gather, 2 back-projection)",
                          bits);
  return DRR_OK;
}

int32_t drr_bounds_checked(void) { return drr::bounds_checked() ? 1 : 0; }

}  // extern "C"
