/*
 * drr.h -- C ABI of libdrr, a GB300 (sm_103a) library for differentiable
 * digitally reconstructed radiographs by Siddon ray tracing
 * (Gopalakrishnan & Golland, arXiv 2208.12737).
 *
 * Conventions shared by every call
 * --------------------------------
 *  - Geometry (Sec. 2.2, 2.4 and Eq. 1-3 of the paper, with these readings):
 *      volume box [b, b + n*delta] with b = -(n*delta)/2 (centred at the origin),
 *      voxel (i,j,k) is the half-open box [b + (i,j,k)*delta, b + (i+1,j+1,k+1)*delta);
 *      pose eta = (rz, ry, rx, tx, ty, tz) in radians / mm,
 *      R = Rz(rz) Ry(ry) Rx(rx), source s = R (rho, 0, 0) + t with rho = sdr/2,
 *      pixel (h, w) centre p = R (-rho, (w - (W-1)/2) dw, (h - (H-1)/2) dh) + t.
 *    The output E(h,w) is the radiologic path length of Eq. (2):
 *      E = |p - s| * sum_m (alpha_{m+1} - alpha_m) V[voxel at the segment midpoint],
 *    with alpha clipped to the volume (Sec. 2.3) and clamped to [0, 1].
 *  - Volumes are passed x fastest: a C array of shape (nz, ny, nx).
 *  - Pointers named *_dev are caller-owned buffers the kernels access: device
 *    memory of the current device, or mapped page-locked host memory (see
 *    "Buffers" below; each is checked before any launch).  The library never
 *    frees them.  Other host pointers are only read during the call.
 *  - Calls taking a `cuda_stream` (a cudaStream_t, NULL = legacy default
 *    stream) enqueue their work on it and return without synchronising.
 *    Argument errors are reported synchronously; errors raised by device work
 *    surface as DRR_ERR_CUDA from a later call or from drr_stream_check().
 *  - Every call returns a drr_status; on failure drr_last_error() gives a
 *    message (thread-local, valid until the next failing call on that thread).
 *  - Empty work (B == 0, H*W == 0) and non-positive sizes or spacings are
 *    DRR_ERR_INVALID.  Non-finite poses give NaN outputs, not an error.
 *  - Limits, checked on the host before any device work (DRR_ERR_INVALID):
 *    B <= 65535 poses per call; H*W <= 2^30 pixels; B * ceil(W/8) * ceil(H/4)
 *    and B * ceil(W/4) * ceil(H/8) < 2^31 (warp tiles of the walks and of the
 *    back-projection); (nx+2)(ny+2)(nz+2) < 2^31 voxels; longest ray |p - s| divided by
 *    the smallest voxel spacing < 2^20 (the walk's FP32 positions need the
 *    plane spacing well above their resolution).
 */
#ifndef DRR_H_
#define DRR_H_

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct drr_volume_s* drr_volume;
typedef struct drr_server_s* drr_server;

typedef enum {
  DRR_OK = 0,
  DRR_ERR_INVALID = 1,   /* bad argument */
  DRR_ERR_OOM = 2,       /* device allocation failed, or a server budget is exhausted */
  DRR_ERR_CUDA = 3,      /* a CUDA runtime call failed */
  DRR_ERR_TIMEOUT = 4,   /* a bounded wait ran out */
  DRR_ERR_BUSY = 5,      /* the object is still referenced (e.g. a volume held by a server) */
  DRR_ERR_NOT_FOUND = 6, /* unknown ticket */
  DRR_ERR_DEVICE = 7,    /* a kernel reported an error through its status word */
  DRR_ERR_CANCELLED = 8  /* the request was cancelled */
} drr_status;

typedef enum {
  DRR_F32 = 0,   /* float32 */
  DRR_BF16 = 1,  /* bfloat16 (storage only) */
  DRR_F16 = 2,   /* IEEE half (storage only; values are stored times a power-of-two scale) */
  DRR_I16_HU = 3 /* int16 Hounsfield units (input only) */
} drr_dtype;

/* Detector of Sec. 2.4: source-to-detector distance sdr (= 2 rho), height x
 * width pixels of spacing delta_h x delta_w (mm). */
typedef struct {
  float sdr_mm;
  int32_t height;
  int32_t width;
  float delta_h_mm;
  float delta_w_mm;
} drr_detector;

/* Storage layouts of a device-resident volume.  Every layout is padded
 * linear storage (one zero voxel of padding on each face, so every gather of
 * the walk is in bounds): a voxel step along any axis moves the walk's offset
 * by one fixed signed stride.  They differ in which axis is fastest, i.e. in
 * which neighbouring voxels share a cache line.  A ray reuses a line for as
 * long as it moves along the fastest axis, so the best choice is the axis the
 * rays mostly run along: x for poses near the canonical one (source on +x).
 * On the 16-pose CT batch (rays within 45 degrees of x) the fwd+Jacobian walk
 * takes 0.567 / 0.583 / 0.643 ms with x / y / z fastest (same bits). */
typedef enum {
  DRR_LAYOUT_DEFAULT = 0,  /* = DRR_LAYOUT_LINEAR_X */
  DRR_LAYOUT_LINEAR_X = 1, /* x fastest, then y, then z */
  DRR_LAYOUT_LINEAR_Y = 2, /* y fastest, then x, then z */
  DRR_LAYOUT_LINEAR_Z = 3  /* z fastest, then x, then y */
} drr_layout;

/* Options for drr_volume_create.  Zero-initialised fields take defaults. */
typedef struct {
  drr_dtype storage;  /* DRR_F32 (default), DRR_BF16 or DRR_F16 */
  float hu_mu_water;  /* attenuation of water in /mm for DRR_I16_HU input:
                         mu = max(0, mu_water (1 + HU/1000)); 0 -> 0.02 */
  int32_t layout;     /* a drr_layout; other values are DRR_ERR_INVALID.  (A
                         bricked layout, 8 x 4 x 1 voxels per 128-byte line, was
                         measured slower than DRR_LAYOUT_LINEAR_X: 0.471 against
                         0.370 ms for the 16-pose CT forward batch; it is not
                         offered.) */
} drr_volume_options;

/* ---- volumes (Sec. 2.2: the CT volume V and its spacing) ---------------- */

/* Upload and convert a volume into device-resident storage.
 *  data           : nz*ny*nx values of src_dtype, x fastest; host memory if
 *                   data_on_device == 0, device memory otherwise.  Only read.
 *  src_dtype      : DRR_F32 (attenuation, /mm) or DRR_I16_HU (mapped to /mm).
 *  nx, ny, nz     : voxel counts (>= 1); dx, dy, dz: spacing in mm (> 0).
 *  opt            : NULL for defaults.
 *  cuda_stream    : stream for the upload/conversion; the call synchronises
 *                   it before returning (the volume is ready on return).
 *  out            : receives the handle; destroy with drr_volume_destroy.
 * FP16 storage multiplies values by scale = 2^(14 - e) where max(V) = m 2^e,
 * m in [0.5, 1) (scale 1 when max(V) == 0); outputs are divided by it again.
 * Errors: DRR_ERR_INVALID, DRR_ERR_OOM, DRR_ERR_CUDA. */
drr_status drr_volume_create(const void* data, int32_t data_on_device, drr_dtype src_dtype, int32_t nx,
                             int32_t ny, int32_t nz, float dx_mm, float dy_mm, float dz_mm,
                             const drr_volume_options* opt, void* cuda_stream, drr_volume* out);

/* Release a volume.  DRR_ERR_BUSY while a server still references it.
 * The caller must ensure no enqueued render still uses it. */
drr_status drr_volume_destroy(drr_volume v);

/* Query a volume: dims (nx, ny, nz), spacing (mm), storage dtype, the storage
 * scale (1 except FP16) and the device bytes it holds.  Any out pointer may be NULL. */
drr_status drr_volume_info(drr_volume v, int32_t dims[3], float spacing[3], drr_dtype* storage,
                           float* storage_scale, size_t* device_bytes);

/* ---- rendering (Eq. 2 for every detector pixel, Sec. 2.3) ---------------- */

/* Buffers.  Every call that takes buffers for the kernels ("_dev"
 * arguments, and volume data with data_on_device != 0) checks each one before
 * any launch: it must be device memory of the current device (the volume's,
 * for calls on a volume) or page-locked host memory mapped for that device
 * (cudaHostAlloc / cudaHostRegister, or a pinned torch tensor).  The kernels
 * read and write host buffers in place across the host link, so a caller whose
 * poses live on the host and who wants E on the host needs no staging copies.
 * Two buffers must be device memory: drr_render_backward's grad_volume_dev
 * (accumulated with atomic adds) and the L2 probe's buffer.  Anything else
 * (pageable host memory, another device's memory) is DRR_ERR_INVALID, before
 * a kernel could fault on it.  The caller keeps ownership; host buffers must
 * stay valid until the stream work is done. */

/* Forward DRR for B poses.
 *  poses_dev   : [B][6] float32 (rz, ry, rx radians; tx, ty, tz mm).
 *  drr_out_dev : [B][H][W] float32, overwritten with E.
 *  jac_out_dev : NULL, or [B][6][H][W] float32 (planar) overwritten with
 *                dE/d eta_k per pixel (Sec. 2.4 gradient, voxel lookup held
 *                fixed), for a later drr_render_backward.
 * With a Jacobian, a launch too small to fill the GPU (up to a few hundred
 * 8x4-pixel tiles, e.g. one 128x128 pose) walks each ray on 4 or 8 warps, each
 * taking a run of the ray's chunks; the results are the same bits as the
 * one-lane walk's.
 * Errors: DRR_ERR_INVALID, DRR_ERR_OOM, DRR_ERR_CUDA. */
drr_status drr_render(drr_volume v, const drr_detector* det, const float* poses_dev, int32_t B,
                      float* drr_out_dev, float* jac_out_dev, void* cuda_stream);

/* Reverse pass (Sec. 2.4: gradient of a loss through the DRR).
 *  grad_drr_dev    : [B][H][W] float32 upstream gradient dL/dE.
 *  jac_dev         : [B][6][H][W] from drr_render, or NULL to re-trace the
 *                    rays and form the Jacobian on the fly.
 *  grad_pose_dev   : NULL, or [B][6] float32, overwritten with
 *                    sum_{h,w} dL/dE(h,w) dE(h,w)/d eta (deterministic:
 *                    fixed-order reduction, FP64 across threads and blocks).
 *  grad_volume_dev : NULL, or [nz][ny][nx] float32 dL/dV (attenuation units),
 *                    ACCUMULATED into (back-projection with atomic adds; the
 *                    summation order, hence the last bits, is not deterministic).
 * At least one of grad_pose_dev / grad_volume_dev must be non-NULL.
 * Errors: DRR_ERR_INVALID, DRR_ERR_OOM, DRR_ERR_CUDA. */
drr_status drr_render_backward(drr_volume v, const drr_detector* det, const float* poses_dev, int32_t B,
                               const float* grad_drr_dev, const float* jac_dev, float* grad_pose_dev,
                               float* grad_volume_dev, void* cuda_stream);

/* Pose gradient from a stored Jacobian without allocating any device memory.
 * The paper has no counterpart: this exists for callers that may not call
 * cudaMalloc or cudaMallocAsync at all -- an application that fixes its whole
 * device-memory footprint up front and forbids later allocations, or a plugin
 * whose host framework owns every device allocation.
 *  det, B, grad_drr_dev, jac_dev, grad_pose_dev: as for drr_render_backward with
 *  a stored Jacobian and grad_volume_dev == NULL; the result is bitwise the same
 *  (the same single launch: one thread-block cluster per pose keeps every
 *  partial sum on chip, so no scratch memory is involved and calls on any
 *  streams may overlap).  Errors: DRR_ERR_INVALID (sizes, NULL pointers),
 *  DRR_ERR_CUDA (launch). */
drr_status drr_pose_grad_noalloc(const drr_detector* det, int32_t B, const float* grad_drr_dev,
                                 const float* jac_dev, float* grad_pose_dev, void* cuda_stream);

/* Ray setup alone (Sec. 2.4): for every pose and pixel write the source s
 * and pixel centre p in world coordinates, rays_out_dev = [B][H][W][6] float32
 * (sx, sy, sz, px, py, pz).  Used to test the geometry kernel. */
drr_status drr_ray_setup(const drr_detector* det, const float* poses_dev, int32_t B, float* rays_out_dev,
                         void* cuda_stream);

/* Number of Siddon segments (Eq. 2 terms) of every ray: segments_out_dev =
 * [B][H][W] int32, 0 for rays that miss.  A segment is the part of a ray
 * inside one voxel between consecutive plane crossings (Eq. 4), counting the
 * zero-length ones produced when two crossings coincide. */
drr_status drr_count_segments(drr_volume v, const drr_detector* det, const float* poses_dev, int32_t B,
                              int32_t* segments_out_dev, void* cuda_stream);

/* ---- registration (Sec. 3.2: gradient descent on negative ZNCC) ---------- */

/* Negative zero-normalised cross-correlation of B image pairs and its gradient
 * with respect to the moving image (population statistics):
 *   c = I - mean(I), s = sqrt(mean(c^2)), I^ = c / (s + eps), F^ likewise,
 *   loss[b] = -mean(I^ F^)        (-1 for a perfect match, eps e.g. 1e-8).
 *  moving_dev, fixed_dev : [B][npix] float32.
 *  loss_dev              : NULL or [B] float32.
 *  grad_dev              : NULL or [B][npix] float32, overwritten with d loss / d moving.
 * Statistics are accumulated in FP64.  Errors: DRR_ERR_INVALID, DRR_ERR_CUDA. */
drr_status drr_zncc(const float* moving_dev, const float* fixed_dev, int32_t B, int32_t npix, float eps,
                    float* loss_dev, float* grad_dev, void* cuda_stream);

/* One Adam step on B six-parameter poses, in place (the paper uses momentum
 * gradient descent with separate rates for rotations and translations; Adam
 * with the same split is used here):
 *  params_dev, grads_dev, m_dev, v_dev : [B][6] float32 (m, v start at zero);
 *  step : 1-based step count (bias correction); lr_rot for the three angles,
 *  lr_trans for the three translations. */
drr_status drr_adam_step(float* params_dev, const float* grads_dev, float* m_dev, float* v_dev, int32_t B,
                         int32_t step, float lr_rot, float lr_trans, float beta1, float beta2, float eps,
                         void* cuda_stream);

/* Gradient with respect to the detector parameters (Sec. 3.2 notes that the
 * generator also differentiates with respect to the source-to-detector
 * distance 2 rho and the pixel spacing; Sec. 2.4 gives s = R (rho,0,0) + t and
 * p = R (-rho, (w-(W-1)/2) dw, (h-(H-1)/2) dh) + t with rho = sdr/2):
 *  grad_drr_dev      : [B][H][W] float32, device, dL/dE;
 *  grad_geometry_dev : [B][3] float32, device, overwritten with
 *                      sum over pixels of dL/dE * dE/d(sdr_mm, delta_h_mm, delta_w_mm)
 *                      for each pose (sum over B for a detector shared by all poses).
 * A re-walk with the fused per-ray Jacobian (same arithmetic as drr_render with
 * a Jacobian), reduced per 8x4-pixel tile and then in FP64 in a fixed order.
 * Asynchronous on cuda_stream.  Errors: DRR_ERR_INVALID, DRR_ERR_CUDA. */
drr_status drr_geometry_grad(drr_volume v, const drr_detector* det, const float* poses_dev, int32_t B,
                             const float* grad_drr_dev, float* grad_geometry_dev, void* cuda_stream);

/* Loss landscape (Sec. 3.2, the study of the negative-ZNCC landscape around the
 * true pose): loss_out[i] = -ZNCC(E(pose_i), fixed) for N poses and one fixed
 * image, with the statistics of drr_zncc (population, FP64, eps).
 *  fixed_dev    : [H][W] float32, device;
 *  poses_dev    : [N][6] float32, device (e.g. a grid of displacements around a pose);
 *  loss_out_dev : [N] float32, device, overwritten;
 *  chunk        : poses rendered per pass (0: as many as fit in 256 MB of DRRs,
 *                 at most 4096); the DRR scratch is allocated from the device's
 *                 stream-ordered pool and released on the stream.
 * Asynchronous on cuda_stream.  Errors: DRR_ERR_INVALID (bad sizes, NULL
 * pointers, eps < 0), DRR_ERR_CUDA. */
drr_status drr_loss_landscape(drr_volume v, const drr_detector* det, const float* fixed_dev, const float* poses_dev,
                              int32_t N, float eps, float* loss_out_dev, int32_t chunk, void* cuda_stream);

/* Comparison baseline, not the product path: the plain FP32 forward walk (the
 * textbook incremental Siddon-Jacobs traversal of Sec. 2.2 with every quantity
 * in FP32: FP32 clip, next crossings advanced by repeated FP32 addition, one
 * thread per ray, linear volume layout, no fusion).  Same arguments and output
 * layout as drr_render without a Jacobian.  Its error against the FP64
 * definition is not bounded by this library's tolerances; it exists so that the
 * product path's speed can be reported against it on the same GPU.
 * Errors: DRR_ERR_INVALID, DRR_ERR_CUDA. */
drr_status drr_render_plain_fp32(drr_volume v, const drr_detector* det, const float* poses_dev, int32_t B,
                                 float* drr_out_dev, void* cuda_stream);

/* Read-bandwidth probe (no counterpart in the paper; it measures the ceiling
 * of the walk's voxel gathers, which are served from L2): streams `bytes` of
 * buf_dev (16-byte aligned, caller-owned device memory; use a buffer smaller
 * than L2) `reps` times with 16-byte loads cached in L2 only, on cuda_stream.
 * Time it with events: achieved L2 read bandwidth = reps * bytes / time.
 * sink_dev: one float the kernel may write.  Errors: DRR_ERR_INVALID, DRR_ERR_CUDA. */
drr_status drr_probe_l2_read(const void* buf_dev, size_t bytes, int32_t reps, float* sink_dev, void* cuda_stream);

/* ---- serving: continuous batching of renders, gradients, registration steps ---- */
/* No counterpart in the paper (whose method is a library call); this is the
 * request loop of the serving workload.  A host thread forms "ticks": it admits
 * queued requests while slots and the explicit memory budgets allow, stages
 * their poses (and upstream gradients) in the server's pinned host memory, which
 * the kernels read in place, and runs one pose-setup, one persistent
 * ray-walk and one gradient-finalise launch that cover the rays of every
 * admitted request, mixed volumes, dtypes and detectors included (optionally
 * replayed from a captured CUDA graph).  Several ticks can be in flight
 * (tick_depth): requests arriving while one tick runs are admitted into the next.  Results of a request
 * are identical whether it ran alone or in a mix (the per-ray arithmetic and the
 * gradient reduction order do not depend on the other requests). */

typedef struct {
  size_t device_budget_bytes; /* device memory reserved for request buffers; 0 -> 512 MiB */
  size_t host_budget_bytes;   /* pinned host memory (mapped for the device) holding each request's
                                 poses, upstream gradient and results; 0 -> the device budget */
  int32_t max_inflight;       /* requests admitted at once (slots); 0 -> 64 (see tick_depth) */
  int32_t max_tick_poses;     /* poses packed into one tick; 0 -> 4096 (also the largest B accepted) */
  int32_t use_cuda_graph;     /* nonzero: replay the tick's three launches from a captured graph */
  int32_t device;             /* CUDA device ordinal; -1 -> the current device */
  int64_t max_tick_work;      /* estimated work admitted into one tick, in ray-planes: a request
                                 counts B*H*W*(nx+ny+nz), times 3/2 with a gradient.  Bounds a
                                 tick's duration, hence the wait of the requests queued behind it
                                 (a request larger than the cap goes alone).  0 -> no cap */
  int32_t plain_fp32_baseline; /* nonzero: the comparison server, not the product: one request per
                                 tick, rendered by the plain FP32 forward walk
                                 (drr_render_plain_fp32), a gradient request by central differences
                                 on it (13 renders per pose, h = 1e-3 rad / 1e-2 mm) */
  int32_t tick_depth;         /* ticks in flight at once, 2 .. 4; 0 -> 3.  One tick takes at most
                                 1/tick_depth of the slots and of each budget, so that the next
                                 ticks can be formed and queued while it runs */
  int32_t spin_poll_us;       /* 0 .. 10^6; 0: the request loop sleeps until a tick's completion
                                 wakes it.  > 0: while a single tick is in flight the loop polls
                                 its completion for up to this many microseconds instead (one
                                 busy host core), which returns a lone request's results
                                 sooner (a 128^2 render served in 0.12 instead of 0.16 ms);
                                 with two or more ticks in flight it sleeps, so that arrivals
                                 gather into the next tick */
} drr_server_config;

/* A request is one of three kinds:
 *  - a render: E for each pose;
 *  - a render with a pose gradient, the upstream gradient dL/dE given
 *    (grad_drr): E and sum_{h,w} dL/dE dE/d eta per pose, from the tick's one
 *    packed walk (each tile's g . J summed in the walk);
 *  - a registration step (Sec. 3.2), fixed images given (fixed): E, the loss
 *    -ZNCC(E, fixed) per pose (population statistics, as drr_zncc) and its pose
 *    gradient.  dL/dE exists only once the whole DRR does, so such a request is
 *    not packed into the tick's walk: the tick runs for it, after the walk, the
 *    direct calls' launches (the fused forward + Jacobian render, drr_zncc, the
 *    stored-Jacobian reduction), and its results are the same bits as
 *    drr_render + drr_zncc + drr_render_backward on the same inputs.
 * The comparison server (plain_fp32_baseline) takes the first two kinds. */
typedef struct {
  drr_volume volume;        /* must stay alive until the request completes (destroy returns BUSY) */
  drr_detector detector;
  int32_t B;                /* poses, 1 .. max_tick_poses */
  const float* poses;       /* host [B][6] */
  const float* grad_drr;    /* host [B][H][W] dL/dE for a render+gradient request, or NULL */
  float* drr_out;           /* host [B][H][W], written before drr_server_wait returns DRR_OK */
  float* grad_pose_out;     /* host [B][6], required iff grad_drr or fixed is given */
  const float* fixed;       /* host [B][H][W] fixed images of a registration step, or NULL
                               (grad_drr must then be NULL) */
  float* loss_out;          /* host [B] -ZNCC per pose, required iff fixed != NULL */
  float zncc_eps;           /* the ZNCC's eps (>= 0); 0 -> 1e-8 */
} drr_request;
/* All host buffers of a request are caller-owned and must stay valid until
 * drr_server_wait has returned for its ticket. */

typedef struct {
  int32_t status;    /* drr_status of the request */
  double queue_ms;   /* submit -> admitted into a tick */
  double latency_ms; /* submit -> results written to the caller's buffers */
  int64_t tick;      /* tick that ran it (-1 if it never ran) */
} drr_result;

typedef struct {
  int64_t submitted, completed, failed, cancelled, ticks;
  int32_t pending, inflight;
  size_t device_in_use, device_budget;
  double p50_ms, p99_ms, mean_ms, max_ms; /* latency of completed requests (p50/p99 over
                                          * the last 2^20 of them, mean and max over all) */
  double gpu_busy_ms;                     /* summed device time of the ticks */
} drr_server_stats;

/* Start a server (allocates both budgets up front; DRR_ERR_OOM if it cannot). */
drr_status drr_server_create(const drr_server_config* cfg, drr_server* out);
/* Queue a request; returns a ticket.  Validation errors are DRR_ERR_INVALID; a
 * request that can never fit the budgets is DRR_ERR_OOM. */
drr_status drr_server_submit(drr_server s, const drr_request* req, uint64_t* ticket);
/* Wait up to timeout_ms (< 0: forever) for a ticket.  Returns the request's
 * status (DRR_OK, DRR_ERR_CANCELLED, ...) and releases the ticket, or
 * DRR_ERR_TIMEOUT (ticket kept), or DRR_ERR_NOT_FOUND for an unknown ticket.
 * DRR_ERR_DEVICE: a serving kernel found the request's part of the tick table
 * inconsistent (a decoded pose index outside the request) and set the
 * request's device status word instead of touching memory; its outputs were
 * not written.  Several threads may wait at once, also on one ticket: each
 * that is waiting when the request finishes gets its result, and the last of
 * them releases the ticket. */
drr_status drr_server_wait(drr_server s, uint64_t ticket, int32_t timeout_ms, drr_result* res);

/* State of a ticket without waiting (no counterpart in the paper). */
typedef enum {
  DRR_REQ_QUEUED = 0,  /* submitted, not yet admitted into a tick */
  DRR_REQ_RUNNING = 1, /* admitted: its tick is on the GPU or its results are being copied */
  DRR_REQ_DONE = 2     /* finished (any status); drr_server_wait returns at once */
} drr_request_state;
/* Non-blocking: *state receives a drr_request_state.  The ticket is kept
 * (release it with drr_server_wait).  DRR_ERR_NOT_FOUND for an unknown ticket. */
drr_status drr_server_poll(drr_server s, uint64_t ticket, int32_t* state);
/* Cancel a request that has not been admitted yet; DRR_ERR_BUSY once it has. */
drr_status drr_server_cancel(drr_server s, uint64_t ticket);
drr_status drr_server_get_stats(drr_server s, drr_server_stats* out);
/* paused != 0: admit no new requests (queued ones wait; ticks already running
 * finish), e.g. to drain the GPU for maintenance.  paused == 0 resumes. */
drr_status drr_server_pause(drr_server s, int32_t paused);
/* Finish in-flight ticks, cancel queued requests and free everything.
 * Threads blocked in drr_server_wait at the time return first (their requests
 * finish or are cancelled); no other call on s may start once destroy has. */
drr_status drr_server_destroy(drr_server s);

/* Fault injection on the host, for tests of the device-status path (no
 * counterpart in the paper): the queued request's device status word is
 * uploaded with `bits` set instead of zero, so after its tick the server
 * reports DRR_ERR_DEVICE for it exactly as if a kernel had flagged it.  No
 * kernel is given an inconsistent table.  DRR_ERR_BUSY once the request has
 * been admitted, DRR_ERR_NOT_FOUND for an unknown ticket. */
drr_status drr_server_inject_device_status(drr_server s, uint64_t ticket, uint32_t bits);

/* Layout of one serving tick (host only, no CUDA call; no counterpart in the
 * paper): for n admitted requests of B[i] poses on detectors dets[i], in
 * admission order, request i owns the tick's 8x4-pixel warp tiles
 * [tile_start[i], tile_start[i] + B[i] * ceil(W/8) * ceil(H/4)) and poses
 * [pose_start[i], pose_start[i] + B[i]); totals[0] = all tiles, totals[1] =
 * all poses.  The serving kernels decode tile and pose indices against these
 * starts.  Exposed so the layout's invariants can be tested on their own. */
drr_status drr_serve_tick_layout(int32_t n, const int32_t* B, const drr_detector* dets, int32_t* tile_start,
                                 int32_t* pose_start, int32_t* totals);

/* ---- host-side offset arena (the servers' admission allocator) ----------- */
/* A first-fit allocator over [0, capacity) with alignment and coalescing; it
 * makes no CUDA calls.  Exposed so its policy can be tested on its own. */
typedef struct drr_arena_s* drr_arena;
drr_status drr_arena_create(size_t capacity, size_t align, drr_arena* out);
drr_status drr_arena_alloc(drr_arena a, size_t bytes, size_t* offset); /* DRR_ERR_OOM if no run fits */
drr_status drr_arena_free(drr_arena a, size_t offset);                 /* DRR_ERR_NOT_FOUND if unknown */
size_t drr_arena_in_use(drr_arena a);
size_t drr_arena_largest_free(drr_arena a);
drr_status drr_arena_destroy(drr_arena a);

/* ---- profiling (no counterpart in the paper) ------------------------------ */

/* While enabled, every kernel launch is bracketed by CUDA events recorded on
 * its stream.  Kernel names: "pose_setup", "siddon_fwd", "siddon_fwd_jac",
 * "siddon_pose_grad", "jac_reduce", "pose_grad_finalize", "siddon_backproject",
 * "count_segments", "zncc", "siddon_geometry_grad", "plain_fp32_fwd",
 * "siddon_fwd_jac_split" (a fused forward + Jacobian launch small enough to
 * walk each ray on 4 or 8 lanes; same results as "siddon_fwd_jac"). */
drr_status drr_profile_enable(int32_t on);
/* Synchronise the recorded events and return the summed device time (ms) and
 * the number of launches of one kernel since the last reset. */
drr_status drr_profile_read(const char* kernel, double* total_ms, int64_t* launches);
/* Drop all recorded events. */
drr_status drr_profile_reset(void);
/* Total kernel launches issued by the library since it was loaded. */
int64_t drr_launch_count(void);

/* Synchronise a stream and report any pending device error as DRR_ERR_CUDA.
 * In a bounds-checked build, also DRR_ERR_DEVICE when a kernel's bounds check
 * failed since the last call (the fault word is then cleared). */
drr_status drr_stream_check(void* cuda_stream);

/* 1 for a bounds-checked build of the library (every voxel gather checked
 * against the padded volume, every back-projection add against the gradient
 * volume; a failed check skips the access and is reported by
 * drr_stream_check), 0 for the product build, which has no checks.  No
 * counterpart in the paper. */
int32_t drr_bounds_checked(void);

/* Thread-local message for the last failing call (never NULL). */
const char* drr_last_error(void);

/* Library version string. */
const char* drr_version(void);

#ifdef __cplusplus
}
#endif

#endif /* DRR_H_ */
