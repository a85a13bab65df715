// Continuous-batching request loop (include/drr.h, "serving").
//
// A host thread forms ticks.  Each tick admits queued requests in FIFO order
// while request slots and the two explicit budgets (device buffers, pinned
// host buffers) allow, stages their inputs in the pinned host arena, and runs
// one pose-setup, one persistent ray-walk and one gradient-finalise launch
// covering all the rays of its renders and gradient requests; the three
// launches can be replayed from a CUDA graph captured at start-up (the kernels
// read the tick's size from a device-resident table).  Its registration-step
// requests (fixed images in, -ZNCC and its pose gradient out) follow with the
// direct calls' launches.  The kernels read the poses and upstream gradients
// from, and write the DRRs, pose gradients and status words to, the mapped
// pinned arena in place, so a tick has no input or result copies besides its
// table.  Up to tick_depth ticks (3 by default) are in flight, so requests that
// arrive while a tick is running are admitted into the next one, and an
// optional cap on the work per tick bounds how long a tick runs.  The loop
// learns that a tick is done from its event (woken by a host function after
// the tick, or polling it when spin_poll_us is set and the tick is alone); it
// then writes each request's results into its caller's buffers (without the
// server lock, so submissions go on), frees its memory and wakes its waiter.
//
// Nothing on the device waits on the host: there are no spin loops in the
// kernels, so a stalled client cannot hang the GPU.
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <mutex>
#include <thread>
#include <unordered_map>
#include <vector>

#include "drr.h"
#include "drr_arena.h"
#include "drr_internal.cuh"

namespace {

using Clock = std::chrono::steady_clock;

constexpr size_t kAlign = 256;

size_t up(size_t b) { return (b + kAlign - 1) / kAlign * kAlign; }

double ms_between(Clock::time_point a, Clock::time_point b) {
  return std::chrono::duration<double, std::milli>(b - a).count();
}

enum ReqState { kPending, kAdmitted, kDone };

struct Req {
  uint64_t id = 0;
  drr_request r{};
  drr::DetDev det{};
  bool grad = false;  // a pose gradient is wanted (upstream gradient given, or a registration step)
  bool zncc = false;  // a registration step: fixed images given, the loss -ZNCC and its gradient
  size_t npix = 0;
  int64_t work = 0;  // estimated ray-planes (the tick-work cap's unit)
  int nposes = 0;    // poses rendered: B, or 13 B for a central-difference gradient (comparison server)
  size_t dev_bytes = 0, host_bytes = 0;
  size_t dev_off = 0, host_off = 0;
  bool has_dev = false, has_host = false;
  // device buffers (inside the device arena)
  float *d_poses = nullptr, *d_grad = nullptr, *d_out = nullptr, *d_partials = nullptr, *d_gpose = nullptr;
  float *d_e13 = nullptr, *d_jac = nullptr;  // comparison server: the 13 renders per pose and the FD Jacobian
  // registration step: E and its Jacobian, the fixed images and dL/dE on the device; the loss
  float *d_e = nullptr, *d_fixed = nullptr, *d_loss = nullptr;
  drr::PoseGeom* d_geom = nullptr;
  // pinned staging (inside the host arena)
  float *h_poses = nullptr, *h_grad = nullptr, *h_out = nullptr, *h_gpose = nullptr;
  float *h_fixed = nullptr, *h_loss = nullptr;
  Clock::time_point t_submit, t_admit, t_done;
  int64_t tick = -1;
  ReqState state = kPending;
  drr_status status = DRR_OK;
  unsigned int device_status = 0;  // the tick's status word for this request, after the tick
  unsigned int inject_status = 0;  // host-side fault injection: uploaded as the initial status word
  int waiters = 0;                 // threads inside drr_server_wait on this ticket (the last one frees it)
};

struct Tick {
  int64_t id = 0;
  int set = 0;  // the table set (and its events) the tick uses
  std::vector<Req*> reqs;
  bool timed = false;  // its start / stop events were recorded
  std::atomic<bool> done{false};
  struct drr_server_s* owner = nullptr;
};

// Ticks in flight at once at most (each has its own table set, graph and events).
constexpr int kMaxTickSets = 4;

// Layout of a tick's work: request i owns the tick's warp tiles
// [tile_start[i], tile_start[i] + B_i * pose_tiles(det_i)) and poses
// [pose_start[i], pose_start[i] + B_i), in admission order, back to back.  The
// serving kernels decode a tile or pose index by a binary search over these
// starts, so the ranges must be contiguous, ascending and cover every index
// exactly once (tested on the CPU through drr_serve_tick_layout).
bool layout_tick(int n, const int32_t* B, const drr::DetDev* det, int32_t* tile_start, int32_t* pose_start,
                 int32_t* total_tiles, int32_t* total_poses) {
  int64_t tiles = 0, poses = 0;
  for (int i = 0; i < n; ++i) {
    tile_start[i] = static_cast<int32_t>(tiles);
    pose_start[i] = static_cast<int32_t>(poses);
    tiles += int64_t(B[i]) * drr::pose_tiles(det[i]);  // the walk claims 8x4 warp tiles
    poses += B[i];
    if (tiles >= (int64_t{1} << 31) || poses >= (int64_t{1} << 31)) return false;
  }
  *total_tiles = static_cast<int32_t>(tiles);
  *total_poses = static_cast<int32_t>(poses);
  return true;
}

// Sizes of a request's device and staging buffers (each piece 256-B aligned).
// The comparison server stages 13 poses per pose of a gradient request, keeps
// their renders and the FD Jacobian, and gives pose setup its counter slot.
// Where a request's inputs and results live.  With DRR_SERVE_HOST_IO (the
// default) the kernels read the poses and the upstream gradient from, and write
// E and dL/d eta to, the request's part of the pinned host arena (mapped into
// the device's address space), so a tick needs no input or result copies and
// its requests finish when its kernels do; device memory holds only the pose
// geometry and the gradient partials (and the comparison server's 13 renders
// per pose and their Jacobian).  With DRR_SERVE_HOST_IO=0 those buffers are
// staged in device memory and copied up and down around the kernels.
#ifndef DRR_SERVE_HOST_IO
#define DRR_SERVE_HOST_IO 1
#endif
constexpr bool kHostIo = DRR_SERVE_HOST_IO != 0;
// How the loop learns that a tick is done: the tick's completion event (queried
// by the loop), and a host function enqueued after the tick that wakes the loop.
// With spin_poll_us > 0 in the configuration, while a single tick is in flight
// the loop polls that event instead of sleeping, yielding the core between
// queries, for up to that long (a submission ends the spin early): a lone
// request's results come back without the host function's wake-up latency.
// With two or more ticks in flight it sleeps until woken, so requests that
// arrive meanwhile gather into the next tick.

void size_request(Req& q, bool plain) {
  const size_t B = static_cast<size_t>(q.r.B);
  const size_t nt = static_cast<size_t>(drr::pose_tiles(q.det));  // gradient partials per pose
  const size_t P = static_cast<size_t>(q.nposes);
  if (q.zncc) {  // geometry (+ the tile counters), E, its 6 Jacobian planes, dL/dE, the fixed images
    q.dev_bytes = up((B + 1) * sizeof(drr::PoseGeom)) + up(B * q.npix * 4) + up(6 * B * q.npix * 4) +
                  up(B * q.npix * 4) + up(B * q.npix * 4);
    if (!kHostIo) q.dev_bytes += up(B * 6 * 4) + up(B * 6 * 4) + up(B * 4);
    q.host_bytes = up(B * 6 * 4) + up(B * q.npix * 4) + up(B * q.npix * 4) + up(B * 6 * 4) + up(B * 4);
    return;
  }
  q.dev_bytes = up((P + (plain ? 1 : 0)) * sizeof(drr::PoseGeom));
  if (!kHostIo) q.dev_bytes += up(P * 6 * 4) + up(B * q.npix * 4);
  q.host_bytes = up(P * 6 * 4) + up(B * q.npix * 4);
  if (q.grad) {
    q.dev_bytes += up(B * nt * 6 * 4);
    if (!kHostIo) q.dev_bytes += up(B * q.npix * 4) + up(B * 6 * 4);
    q.host_bytes += up(B * q.npix * 4) + up(B * 6 * 4);
    if (plain) q.dev_bytes += up(P * q.npix * 4) + up(B * 6 * q.npix * 4);
  }
}

// The comparison server's central-difference steps (rad, mm).
constexpr float kFdRot = 1e-3f, kFdTrans = 1e-2f;

}  // namespace

struct drr_server_s {
  drr_server_config cfg{};
  int device = 0;
  cudaStream_t h2d = nullptr;     // input copies (the kernels run on sets[0].ks)
  cudaStream_t d2h = nullptr;     // result copies
  char* dev_base = nullptr;
  char* host_base = nullptr;
  char* host_dev_base = nullptr;  // the host arena's address on the device (mapped pinned memory)
  drr::OffsetArena* dev_arena = nullptr;
  drr::OffsetArena* host_arena = nullptr;
  struct Set {
    char* h_table = nullptr;  // pinned: header + requests + per-request status words
    char* d_table = nullptr;
    int* d_counter = nullptr;
    cudaGraphExec_t graph = nullptr;
    cudaEvent_t start = nullptr, stop = nullptr;  // around the kernels; stop also orders the result copies
    cudaEvent_t in_ready = nullptr;               // the tick's inputs are on the device
    cudaEvent_t done_ev = nullptr;                // after the tick's last kernel and copy
    unsigned int* status_dev = nullptr;           // the status words as the kernels address them
    cudaStream_t ks = nullptr;                    // the kernel stream (shared by all sets)
  } sets[kMaxTickSets];
  int depth = 3;  // ticks in flight at most (table sets in use)
  size_t table_bytes = 0;
  size_t status_off = 0;  // offset of the status words in a table
  int walk_grid = 1;
  int waiters = 0;  // threads inside drr_server_wait (destroy waits for them to leave)
  std::atomic<uint64_t> submit_seq{0};  // bumped by every submission (ends the loop's poll early)

  std::mutex mu;
  std::condition_variable cv_loop, cv_done;
  std::deque<Req*> pending;
  std::unordered_map<uint64_t, Req*> reqs;
  std::deque<Tick*> inflight;
  // latencies of completed requests: the last kLatencyWindow for the
  // percentiles (a server that runs for days keeps a bounded record), and the
  // count, sum and maximum of all of them
  static constexpr size_t kLatencyWindow = size_t(1) << 20;
  std::vector<double> latencies;
  size_t lat_next = 0;
  int64_t lat_count = 0;
  double lat_sum = 0.0, lat_max = 0.0;
  void record_latency(double ms) {
    if (latencies.size() < kLatencyWindow) {
      latencies.push_back(ms);
    } else {
      latencies[lat_next] = ms;
      lat_next = (lat_next + 1) % kLatencyWindow;
    }
    ++lat_count;
    lat_sum += ms;
    lat_max = std::max(lat_max, ms);
  }
  int64_t submitted = 0, completed = 0, failed = 0, cancelled = 0, ticks = 0;
  double gpu_busy_ms = 0.0;
  int admitted = 0;
  uint64_t next_id = 1;
  int64_t next_tick = 0;
  bool stop = false;
  bool paused = false;
  std::thread loop;

  void run();
  bool form_tick(std::unique_lock<std::mutex>& lk);
  void copy_result(Tick* t, size_t i);
  void finish_request(Req* q);
  void sync_streams();
  cudaError_t launch_kernels(int set);
  cudaError_t launch_plain(const Req& q, cudaStream_t ks);
  cudaError_t launch_registration_step(const Req& q, cudaStream_t ks);
  bool tick_ready(Tick* t);
};

namespace {

// Runs on a CUDA runtime thread once a tick's stream work is complete: it wakes
// the loop, which decides completion from the tick's event (the tick itself may
// already be gone).  It takes no lock, so it never stalls the stream behind the
// loop thread; the loop re-checks at least every 200 us anyway.
void CUDART_CB tick_done(void* p) { static_cast<drr_server_s*>(p)->cv_loop.notify_all(); }

}  // namespace

cudaError_t drr_server_s::launch_kernels(int set) {
  Set& st = sets[set];
  if (st.graph) return cudaGraphLaunch(st.graph, st.ks);
  const auto* hdr = reinterpret_cast<const drr::ServeHeader*>(st.d_table);
  const auto* rq = reinterpret_cast<const drr::ServeRequest*>(st.d_table + sizeof(drr::ServeHeader));
  return drr::launch_serve_tick(hdr, rq, st.status_dev, st.d_counter, cfg.max_tick_poses, walk_grid, st.ks);
}

// The comparison server's tick: one request, the plain FP32 forward walk over
// its poses (13 per pose for a gradient request), then for a gradient the
// central differences and their sum against the upstream gradient.
cudaError_t drr_server_s::launch_plain(const Req& q, cudaStream_t ks) {
  const drr::VolumeDev& vd = q.r.volume->vd;
  cudaError_t e = drr::launch_pose_setup(q.d_poses, q.nposes, q.det, &vd, q.d_geom, ks);
  if (e != cudaSuccess) return e;
  if (!q.grad) return drr::launch_render_plain_fp32(vd, q.det, q.d_geom, q.nposes, q.d_out, ks);
  e = drr::launch_render_plain_fp32(vd, q.det, q.d_geom, q.nposes, q.d_e13, ks);
  if (e == cudaSuccess)
    e = drr::launch_plain_fd_finish(q.d_e13, q.r.B, static_cast<int>(q.npix), kFdRot, kFdTrans, q.d_out, q.d_jac, ks);
  if (e == cudaSuccess) e = drr::launch_pose_grad_from_jacobian(q.det, q.r.B, q.d_grad, q.d_jac, q.d_gpose, ks);
  return e;
}

// A registration step (Sec. 3.2): the direct calls' launches in their order --
// pose setup, the fused forward + Jacobian render (the same split-walk choice
// as drr_render), the ZNCC loss and dL/dE, and the stored-Jacobian pose
// gradient -- so its results are the direct path's bits.
cudaError_t drr_server_s::launch_registration_step(const Req& q, cudaStream_t ks) {
  const drr::VolumeDev& vd = q.r.volume->vd;
  const int B = q.r.B;
  cudaError_t e = drr::launch_pose_setup(q.d_poses, B, q.det, &vd, q.d_geom, ks);
  if (e == cudaSuccess)
    e = drr::launch_render(vd, q.det, q.d_geom, B, q.d_e, q.d_jac, ks, drr::render_split_lanes(vd, q.det, B));
  if (e == cudaSuccess)
    e = drr::launch_zncc(q.d_e, q.d_fixed, q.npix, B, static_cast<int>(q.npix), q.r.zncc_eps, q.d_loss, q.d_grad, ks);
  if (e == cudaSuccess) e = drr::launch_pose_grad_from_jacobian(q.det, B, q.d_grad, q.d_jac, q.d_gpose, ks);
  return e;
}

// Admit requests (FIFO) into a new tick and enqueue it.  Called with lk held;
// drops it while staging inputs and issuing CUDA calls.
bool drr_server_s::form_tick(std::unique_lock<std::mutex>& lk) {
  // One tick takes at most 1/depth of the request slots and of each memory
  // budget (a request that needs more goes alone), so that the next ticks can
  // be formed and queued while this one runs.  Without the cap a backlog puts
  // every slot into one tick, the next tick finds none free until it ends, and
  // the GPU idles between ticks.
  // The tick-work cap bounds a tick's duration, and with it the wait of the
  // requests queued behind it; the comparison server takes one request per tick.
  const int slot_cap = cfg.plain_fp32_baseline ? 1 : std::max(1, cfg.max_inflight / depth);
  std::vector<Req*> batch;
  int poses = 0;
  int64_t tick_work = 0;
  size_t tick_dev = 0, tick_host = 0;
  while (!pending.empty() && admitted + static_cast<int>(batch.size()) < cfg.max_inflight &&
         static_cast<int>(batch.size()) < slot_cap) {
    Req* q = pending.front();
    if (poses + q->r.B > cfg.max_tick_poses) break;
    if (!batch.empty() && cfg.max_tick_work > 0 && tick_work + q->work > cfg.max_tick_work) break;
    if (!batch.empty() && (tick_dev + q->dev_bytes > cfg.device_budget_bytes / depth ||
                           tick_host + q->host_bytes > cfg.host_budget_bytes / depth))
      break;
    size_t doff = 0, hoff = 0;
    if (!dev_arena->alloc(q->dev_bytes, &doff)) break;
    if (!host_arena->alloc(q->host_bytes, &hoff)) {
      dev_arena->release(doff);
      break;
    }
    pending.pop_front();
    q->dev_off = doff;
    q->host_off = hoff;
    q->has_dev = q->has_host = true;
    q->state = kAdmitted;
    q->t_admit = Clock::now();
    poses += q->r.B;
    tick_work += q->work;
    tick_dev += q->dev_bytes;
    tick_host += q->host_bytes;
    batch.push_back(q);
  }
  if (batch.empty()) return false;
  admitted += static_cast<int>(batch.size());
  // the packed walk's requests first (table entries 0 .. nw - 1), then the
  // registration steps, which run their own launches after the walk
  std::stable_partition(batch.begin(), batch.end(), [](const Req* q) { return !q->zncc; });
  const int nw = static_cast<int>(std::count_if(batch.begin(), batch.end(), [](const Req* q) { return !q->zncc; }));
  Tick* t = new Tick();
  t->id = next_tick++;
  t->set = static_cast<int>(t->id % depth);
  t->owner = this;
  t->reqs = batch;
  lk.unlock();
  cudaError_t e = cudaSuccess;

  // carve the buffers and stage the inputs
  Set& st = sets[t->set];
  auto* hdr = reinterpret_cast<drr::ServeHeader*>(st.h_table);
  auto* rq = reinterpret_cast<drr::ServeRequest*>(st.h_table + sizeof(drr::ServeHeader));
  const int n = static_cast<int>(batch.size());
  std::vector<int32_t> Bs(n), tstart(n), pstart(n);
  std::vector<drr::DetDev> dets(n);
  for (int i = 0; i < n; ++i) {
    Bs[i] = batch[i]->r.B;
    dets[i] = batch[i]->det;
  }
  int32_t total_tiles = 0, total_poses = 0;
  // admission caps the tick at max_tick_poses <= 2^20 poses of < 2^30 tiles each
  // request, so the layout always fits; a failure leaves the tick empty
  if (nw > 0 && !layout_tick(nw, Bs.data(), dets.data(), tstart.data(), pstart.data(), &total_tiles, &total_poses)) {
    total_tiles = total_poses = 0;
    if (e == cudaSuccess) e = cudaErrorInvalidValue;
  }
  for (size_t i = 0; i < batch.size(); ++i) {
    Req* q = batch[i];
    q->tick = t->id;
    const size_t B = static_cast<size_t>(q->r.B);
    const size_t nt = static_cast<size_t>(drr::pose_tiles(q->det));  // walk tiles and gradient partials per pose
    char* d = dev_base + q->dev_off;
    char* h = host_base + q->host_off;
    const bool plain = cfg.plain_fp32_baseline != 0;
    const size_t P = static_cast<size_t>(q->nposes);
    // a host-arena buffer under its device address (host I/O), or a device buffer carved from d
    auto io = [&](char* hp, size_t bytes) {
      if (kHostIo) return reinterpret_cast<float*>(host_dev_base + (hp - host_base));
      float* dp = reinterpret_cast<float*>(d);
      d += up(bytes);
      return dp;
    };
    if (q->zncc) {
      auto dev = [&](size_t bytes) {
        float* dp = reinterpret_cast<float*>(d);
        d += up(bytes);
        return dp;
      };
      q->d_geom = reinterpret_cast<drr::PoseGeom*>(dev((B + 1) * sizeof(drr::PoseGeom)));
      q->d_e = dev(B * q->npix * 4);
      q->d_jac = dev(6 * B * q->npix * 4);
      q->d_grad = dev(B * q->npix * 4);
      q->d_fixed = dev(B * q->npix * 4);
      q->h_poses = reinterpret_cast<float*>(h);
      q->d_poses = io(h, B * 6 * 4);
      h += up(B * 6 * 4);
      q->h_out = reinterpret_cast<float*>(h);
      h += up(B * q->npix * 4);
      q->h_fixed = reinterpret_cast<float*>(h);
      h += up(B * q->npix * 4);
      q->h_gpose = reinterpret_cast<float*>(h);
      q->d_gpose = io(h, B * 6 * 4);
      h += up(B * 6 * 4);
      q->h_loss = reinterpret_cast<float*>(h);
      q->d_loss = io(h, B * 4);
      std::memcpy(q->h_poses, q->r.poses, B * 6 * 4);
      std::memcpy(q->h_fixed, q->r.fixed, B * q->npix * 4);
      rq[i] = drr::ServeRequest{};  // no table entry of the walk (its status word stays as uploaded)
      continue;
    }
    q->h_poses = reinterpret_cast<float*>(h);
    q->d_poses = io(h, P * 6 * 4);
    h += up(P * 6 * 4);
    q->h_out = reinterpret_cast<float*>(h);
    q->d_out = io(h, B * q->npix * 4);
    h += up(B * q->npix * 4);
    q->d_geom = reinterpret_cast<drr::PoseGeom*>(d); d += up((P + (plain ? 1 : 0)) * sizeof(drr::PoseGeom));
    if (q->grad) {
      q->h_grad = reinterpret_cast<float*>(h);
      q->d_grad = io(h, B * q->npix * 4);
      h += up(B * q->npix * 4);
      q->h_gpose = reinterpret_cast<float*>(h);
      q->d_gpose = io(h, B * 6 * 4);
      q->d_partials = reinterpret_cast<float*>(d); d += up(B * nt * 6 * 4);
      if (plain) {
        q->d_e13 = reinterpret_cast<float*>(d); d += up(P * q->npix * 4);
        q->d_jac = reinterpret_cast<float*>(d);
      }
    }
    if (P == B) {
      std::memcpy(q->h_poses, q->r.poses, B * 6 * 4);
    } else {  // 13 poses per pose: the pose, then +h and -h of each parameter
      for (size_t b = 0; b < B; ++b) {
        for (int c = 0; c < 13; ++c) {
          float* dst = q->h_poses + (b * 13 + c) * 6;
          std::memcpy(dst, q->r.poses + b * 6, 6 * 4);
          if (c > 0) {
            const int k = (c - 1) / 2;
            dst[k] += ((c - 1) % 2 == 0 ? 1.f : -1.f) * (k < 3 ? kFdRot : kFdTrans);
          }
        }
      }
    }
    if (q->grad) std::memcpy(q->h_grad, q->r.grad_drr, B * q->npix * 4);
    drr::ServeRequest& sr = rq[i];
    std::memset(&sr, 0, sizeof(sr));
    sr.vd = q->r.volume->vd;
    sr.det = q->det;
    sr.poses = q->d_poses;
    sr.grad = q->d_grad;
    sr.out = q->d_out;
    sr.partials = q->d_partials;
    sr.grad_pose = q->d_gpose;
    sr.geom = q->d_geom;
    sr.B = q->r.B;
    sr.tile_start = tstart[i];
    sr.pose_start = pstart[i];
  }
  hdr->nreq = nw;
  hdr->total_tiles = total_tiles;
  hdr->total_poses = total_poses;
  hdr->pad_ = 0;
  auto* h_status = reinterpret_cast<unsigned int*>(st.h_table + status_off);
  for (size_t i = 0; i < batch.size(); ++i) h_status[i] = batch[i]->inject_status;  // normally 0
  const size_t tbytes = sizeof(drr::ServeHeader) + size_t(nw) * sizeof(drr::ServeRequest);
  const size_t sbytes = batch.size() * sizeof(unsigned int);
  // The table set and the request buffers written here belong to no tick still
  // in flight: this tick's set was last used `depth` ticks ago, which has finished
  // (its result copies, after its kernels, are done), and the arenas hand out
  // only memory of finished ticks.
  if (e == cudaSuccess) e = cudaMemcpyAsync(st.d_table, st.h_table, tbytes, cudaMemcpyHostToDevice, h2d);
  if (e == cudaSuccess && !kHostIo)  // with host I/O the kernels use the words in place
    e = cudaMemcpyAsync(st.d_table + status_off, h_status, sbytes, cudaMemcpyHostToDevice, h2d);
  for (Req* q : batch) {
    if (e != cudaSuccess) break;
    if (q->zncc)  // the ZNCC kernel reads each fixed image whole: from device memory
      e = cudaMemcpyAsync(q->d_fixed, q->h_fixed, size_t(q->r.B) * q->npix * 4, cudaMemcpyHostToDevice, h2d);
    if (kHostIo) continue;
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(q->d_poses, q->h_poses, size_t(q->nposes) * 6 * 4, cudaMemcpyHostToDevice, h2d);
    if (e == cudaSuccess && q->grad && !q->zncc)
      e = cudaMemcpyAsync(q->d_grad, q->h_grad, size_t(q->r.B) * q->npix * 4, cudaMemcpyHostToDevice, h2d);
  }
  if (e == cudaSuccess) e = cudaEventRecord(st.in_ready, h2d);
  if (e == cudaSuccess) e = cudaStreamWaitEvent(st.ks, st.in_ready, 0);
  if (e == cudaSuccess) e = cudaEventRecord(st.start, st.ks);
  if (cfg.plain_fp32_baseline) {
    if (e == cudaSuccess) e = launch_plain(*batch[0], st.ks);
    if (e == cudaSuccess) drr::count_launches(batch[0]->grad ? 4 : 2);
  } else {
    if (nw > 0) {
      if (e == cudaSuccess) e = launch_kernels(t->set);
      if (e == cudaSuccess) drr::count_launches(3);
    }
    for (int i = nw; i < n && e == cudaSuccess; ++i) {
      e = launch_registration_step(*batch[i], st.ks);
      if (e == cudaSuccess) drr::count_launches(4);
    }
  }
  if (e == cudaSuccess) e = cudaEventRecord(st.stop, st.ks);
  if (e == cudaSuccess) t->timed = true;
  if (e == cudaSuccess) e = cudaStreamWaitEvent(d2h, st.stop, 0);
  if (e == cudaSuccess && !kHostIo)
    e = cudaMemcpyAsync(h_status, st.d_table + status_off, sbytes, cudaMemcpyDeviceToHost, d2h);
  for (Req* q : batch) {
    if (e != cudaSuccess) break;
    if (q->zncc)  // E stays on the device for the ZNCC kernel; it comes down here
      e = cudaMemcpyAsync(q->h_out, q->d_e, size_t(q->r.B) * q->npix * 4, cudaMemcpyDeviceToHost, d2h);
    if (kHostIo) continue;
    if (e == cudaSuccess && !q->zncc)
      e = cudaMemcpyAsync(q->h_out, q->d_out, size_t(q->r.B) * q->npix * 4, cudaMemcpyDeviceToHost, d2h);
    if (e == cudaSuccess && q->grad)
      e = cudaMemcpyAsync(q->h_gpose, q->d_gpose, size_t(q->r.B) * 6 * 4, cudaMemcpyDeviceToHost, d2h);
    if (e == cudaSuccess && q->zncc)
      e = cudaMemcpyAsync(q->h_loss, q->d_loss, size_t(q->r.B) * 4, cudaMemcpyDeviceToHost, d2h);
  }
  if (e == cudaSuccess) e = cudaEventRecord(st.done_ev, d2h);
  if (e == cudaSuccess) e = cudaLaunchHostFunc(d2h, tick_done, this);
  if (e != cudaSuccess) {
    // the tick could not be enqueued completely: let what was queued drain, then fail its requests
    sync_streams();
    for (Req* q : batch) q->status = drr::cuda_error(e, "serving tick");
    t->timed = false;
    t->done.store(true);
  }
  lk.lock();
  inflight.push_back(t);
  ++ticks;
  return true;
}

void drr_server_s::sync_streams() {
  cudaStreamSynchronize(h2d);
  if (sets[0].ks) cudaStreamSynchronize(sets[0].ks);
  cudaStreamSynchronize(d2h);
}

// Called WITHOUT the lock once the tick's device work is done: the tick is off
// the in-flight list and its requests are admitted (not done), so no other
// thread touches them or their callers' buffers meanwhile.
void drr_server_s::copy_result(Tick* t, size_t i) {
  const auto* h_status = reinterpret_cast<const unsigned int*>(sets[t->set].h_table + status_off);
  Req* q = t->reqs[i];
  if (q->status != DRR_OK) return;
  q->device_status = h_status[i];
  if (q->device_status != 0) {  // a kernel flagged this request: its outputs are not trusted
    q->status = DRR_ERR_DEVICE;
    return;
  }
  std::memcpy(q->r.drr_out, q->h_out, size_t(q->r.B) * q->npix * 4);
  if (q->grad) std::memcpy(q->r.grad_pose_out, q->h_gpose, size_t(q->r.B) * 6 * 4);
  if (q->zncc) std::memcpy(q->r.loss_out, q->h_loss, size_t(q->r.B) * 4);
}

// Called with the lock held after copy_result: the request is done (its
// waiter wakes) and its memory goes back to the arenas.
void drr_server_s::finish_request(Req* q) {
  if (q->status == DRR_OK) {
    ++completed;
  } else {
    ++failed;
  }
  if (q->has_dev) dev_arena->release(q->dev_off);
  if (q->has_host) host_arena->release(q->host_off);
  q->has_dev = q->has_host = false;
  q->t_done = Clock::now();
  if (q->status == DRR_OK) record_latency(ms_between(q->t_submit, q->t_done));
  q->state = kDone;
  q->r.volume->refs.fetch_sub(1);
  --admitted;
  cv_done.notify_all();
}

// Whether a tick's work is complete (or failed: its requests then fail when
// their results are read).  Called by the loop thread only.
bool drr_server_s::tick_ready(Tick* t) {
  if (!t->done.load()) {
    const cudaError_t q = cudaEventQuery(sets[t->set].done_ev);
    if (q != cudaErrorNotReady) t->done.store(true);
  }
  return t->done.load();
}

void drr_server_s::run() {
  cudaSetDevice(device);
  std::unique_lock<std::mutex> lk(mu);
  for (;;) {
    while (!inflight.empty() && tick_ready(inflight.front())) {
      Tick* t = inflight.front();
      inflight.pop_front();
      if (t->timed) {
        float ms = 0.f;
        if (cudaEventElapsedTime(&ms, sets[t->set].start, sets[t->set].stop) == cudaSuccess) gpu_busy_ms += ms;
      }
      // each request is done as soon as its own results are in the caller's
      // buffers, not once the whole tick's are (a tick's copies take ~20 us per MB)
      for (size_t i = 0; i < t->reqs.size(); ++i) {
        lk.unlock();
        copy_result(t, i);
        lk.lock();
        finish_request(t->reqs[i]);
      }
      delete t;
    }
    if (stop && inflight.empty()) break;
    bool launched = false;
    if (!stop && !paused && static_cast<int>(inflight.size()) < depth && !pending.empty()) launched = form_tick(lk);
    if (!launched && cfg.spin_poll_us > 0 && inflight.size() == 1) {
      // one tick in flight: poll its completion event without the lock
      Tick* f = inflight.front();
      const cudaEvent_t ev = sets[f->set].done_ev;
      const uint64_t seq = submit_seq.load();
      lk.unlock();
      const auto t0 = Clock::now();
      bool ready = false;
      for (;;) {
        if (cudaEventQuery(ev) != cudaErrorNotReady) {
          ready = true;
          break;
        }
        if (submit_seq.load() != seq) break;
        if (Clock::now() - t0 > std::chrono::microseconds(cfg.spin_poll_us)) break;
        std::this_thread::yield();
      }
      lk.lock();
      if (ready || submit_seq.load() != seq) continue;
    }
    if (!launched) {
      cv_loop.wait_for(lk, std::chrono::microseconds(200), [this] {
        return stop || (!inflight.empty() && tick_ready(inflight.front())) ||
               (!paused && static_cast<int>(inflight.size()) < depth && !pending.empty());
      });
    }
  }
}

extern "C" {

drr_status drr_server_create(const drr_server_config* cfg_in, drr_server* out) {
  if (!out) return drr::set_error(DRR_ERR_INVALID, "out is NULL");
  *out = nullptr;
  drr_server_config cfg{};
  if (cfg_in) cfg = *cfg_in;
  if (cfg.device_budget_bytes == 0) cfg.device_budget_bytes = size_t(512) << 20;
  if (cfg.host_budget_bytes == 0) cfg.host_budget_bytes = cfg.device_budget_bytes;
  if (cfg.max_inflight <= 0) cfg.max_inflight = 64;
  if (cfg.max_tick_poses <= 0) cfg.max_tick_poses = 4096;
  if (cfg.max_inflight > 4096 || cfg.max_tick_poses > (1 << 20))
    return drr::set_error(DRR_ERR_INVALID, "max_inflight <= 4096 and max_tick_poses <= 2^20 required");
  if (cfg.max_tick_work < 0) return drr::set_error(DRR_ERR_INVALID, "max_tick_work must be >= 0");
  if (cfg.tick_depth == 0) cfg.tick_depth = 3;
  if (cfg.tick_depth < 2 || cfg.tick_depth > kMaxTickSets)
    return drr::set_error(DRR_ERR_INVALID, "tick_depth must be in [2, %d]", kMaxTickSets);
  if (cfg.spin_poll_us < 0 || cfg.spin_poll_us > 1000000)
    return drr::set_error(DRR_ERR_INVALID, "spin_poll_us must be in [0, 10^6]");
  drr_server_s* s = new drr_server_s();
  s->cfg = cfg;
  cudaError_t e = cudaSuccess;
  if (cfg.device >= 0) e = cudaSetDevice(cfg.device);
  if (e == cudaSuccess) e = cudaGetDevice(&s->device);
  if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&s->h2d, cudaStreamNonBlocking);
  if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&s->d2h, cudaStreamNonBlocking);
  if (e == cudaSuccess) e = cudaMalloc(reinterpret_cast<void**>(&s->dev_base), cfg.device_budget_bytes);
  if (e == cudaSuccess)
    e = cudaHostAlloc(reinterpret_cast<void**>(&s->host_base), cfg.host_budget_bytes, cudaHostAllocMapped);
  if (e == cudaSuccess) e = cudaHostGetDevicePointer(reinterpret_cast<void**>(&s->host_dev_base), s->host_base, 0);
  s->status_off = up(sizeof(drr::ServeHeader) + size_t(cfg.max_inflight) * sizeof(drr::ServeRequest));
  s->table_bytes = s->status_off + size_t(cfg.max_inflight) * sizeof(unsigned int);
  s->depth = cfg.tick_depth;
  for (int i = 0; i < s->depth && e == cudaSuccess; ++i) {
    e = cudaHostAlloc(reinterpret_cast<void**>(&s->sets[i].h_table), s->table_bytes, cudaHostAllocMapped);
    if (e == cudaSuccess) e = cudaMalloc(reinterpret_cast<void**>(&s->sets[i].d_table), s->table_bytes);
    if (e == cudaSuccess) e = cudaMalloc(reinterpret_cast<void**>(&s->sets[i].d_counter), sizeof(int));
    if (e == cudaSuccess) e = cudaMemset(s->sets[i].d_table, 0, s->table_bytes);
    if (e == cudaSuccess) e = cudaEventCreate(&s->sets[i].start);
    if (e == cudaSuccess) e = cudaEventCreate(&s->sets[i].stop);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&s->sets[i].in_ready, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&s->sets[i].done_ev, cudaEventDisableTiming);
    if (e == cudaSuccess) {
      if (kHostIo) {
        char* mapped = nullptr;
        e = cudaHostGetDevicePointer(reinterpret_cast<void**>(&mapped), s->sets[i].h_table, 0);
        if (e == cudaSuccess) s->sets[i].status_dev = reinterpret_cast<unsigned int*>(mapped + s->status_off);
      } else {
        s->sets[i].status_dev = reinterpret_cast<unsigned int*>(s->sets[i].d_table + s->status_off);
      }
    }
    // one kernel stream for every set: ticks run one after another.  (A stream
    // per set, so that consecutive ticks overlap, measured slower: saturation
    // 8.6k-9.2k against 12.1k-13.7k requests/s on the serving mix, the
    // concurrent walks over different volumes competing for L2.)
    if (e == cudaSuccess && i == 0) e = cudaStreamCreateWithFlags(&s->sets[0].ks, cudaStreamNonBlocking);
    s->sets[i].ks = s->sets[0].ks;
  }
  if (e == cudaSuccess) s->walk_grid = drr::serve_walk_grid(s->device);
  if (e == cudaSuccess && cfg.use_cuda_graph && !cfg.plain_fp32_baseline) {
    for (int i = 0; i < s->depth && e == cudaSuccess; ++i) {
      cudaGraph_t g = nullptr;
      e = cudaStreamBeginCapture(s->sets[i].ks, cudaStreamCaptureModeThreadLocal);
      if (e == cudaSuccess) {
        cudaError_t le = s->launch_kernels(i);
        e = cudaStreamEndCapture(s->sets[i].ks, &g);
        if (le != cudaSuccess) e = le;
      }
      if (e == cudaSuccess) e = cudaGraphInstantiate(&s->sets[i].graph, g, 0);
      if (g) cudaGraphDestroy(g);
    }
  }
  if (e != cudaSuccess) {
    drr_status st = drr::cuda_error(e, "drr_server_create");
    for (auto& st2 : s->sets) {
      if (st2.graph) cudaGraphExecDestroy(st2.graph);
      if (st2.h_table) cudaFreeHost(st2.h_table);
      if (st2.d_table) cudaFree(st2.d_table);
      if (st2.d_counter) cudaFree(st2.d_counter);
      if (st2.start) cudaEventDestroy(st2.start);
      if (st2.stop) cudaEventDestroy(st2.stop);
      if (st2.in_ready) cudaEventDestroy(st2.in_ready);
      if (st2.done_ev) cudaEventDestroy(st2.done_ev);
    }
    if (s->sets[0].ks) cudaStreamDestroy(s->sets[0].ks);
    if (s->dev_base) cudaFree(s->dev_base);
    if (s->host_base) cudaFreeHost(s->host_base);
    if (s->h2d) cudaStreamDestroy(s->h2d);
    if (s->d2h) cudaStreamDestroy(s->d2h);
    delete s;
    return st;
  }
  s->dev_arena = new drr::OffsetArena(cfg.device_budget_bytes, kAlign);
  s->host_arena = new drr::OffsetArena(cfg.host_budget_bytes, kAlign);
  s->loop = std::thread([s] { s->run(); });
  *out = s;
  return DRR_OK;
}

drr_status drr_server_submit(drr_server s, const drr_request* req, uint64_t* ticket) {
  if (!s || !req || !ticket) return drr::set_error(DRR_ERR_INVALID, "NULL argument");
  drr_volume v = req->volume;
  if (!v || !v->storage) return drr::set_error(DRR_ERR_INVALID, "request volume is NULL or destroyed");
  if (v->device != s->device) return drr::set_error(DRR_ERR_INVALID, "volume lives on another device");
  drr::DetDev dd;
  if (drr_status st = drr::check_detector(&req->detector, &dd)) return st;
  if (drr_status st = drr::check_geometry(v->vd, dd)) return st;
  if (req->B <= 0 || req->B > s->cfg.max_tick_poses)
    return drr::set_error(DRR_ERR_INVALID, "B must be in [1, %d]", s->cfg.max_tick_poses);
  if (!req->poses || !req->drr_out) return drr::set_error(DRR_ERR_INVALID, "poses and drr_out are required");
  if (req->grad_drr && !req->grad_pose_out)
    return drr::set_error(DRR_ERR_INVALID, "grad_pose_out is required with grad_drr");
  if (req->fixed) {
    if (req->grad_drr) return drr::set_error(DRR_ERR_INVALID, "a request takes grad_drr or fixed, not both");
    if (!req->grad_pose_out || !req->loss_out)
      return drr::set_error(DRR_ERR_INVALID, "grad_pose_out and loss_out are required with fixed");
    if (s->cfg.plain_fp32_baseline)
      return drr::set_error(DRR_ERR_INVALID, "the comparison server takes no registration-step requests");
    if (!(req->zncc_eps >= 0.f) || !std::isfinite(req->zncc_eps))
      return drr::set_error(DRR_ERR_INVALID, "zncc_eps must be finite and >= 0");
  }
  Req* q = new Req();
  q->r = *req;
  if (req->fixed && q->r.zncc_eps == 0.f) q->r.zncc_eps = 1e-8f;
  q->det = dd;
  q->grad = req->grad_drr != nullptr || req->fixed != nullptr;
  q->zncc = req->fixed != nullptr;
  q->npix = size_t(dd.H) * dd.W;
  if (size_t(req->B) * size_t(drr::pose_tiles(dd)) >= (size_t(1) << 30)) {
    delete q;
    return drr::set_error(DRR_ERR_INVALID, "request has too many tiles");
  }
  q->nposes = (s->cfg.plain_fp32_baseline && q->grad) ? 13 * req->B : req->B;
  if (q->nposes > 65535) {
    delete q;
    return drr::set_error(DRR_ERR_INVALID, "the comparison server renders at most 65535 poses per request");
  }
  {
    // B * H * W * (nx + ny + nz), x 3/2 with a gradient, saturated at 2^62 (the factors
    // are each below 2^32, so their product can exceed int64)
    const double w = double(req->B) * double(q->npix) * (double(v->vd.n[0]) + v->vd.n[1] + v->vd.n[2]) *
                     (q->grad ? 1.5 : 1.0);
    q->work = w < 4.6e18 ? static_cast<int64_t>(w) : (int64_t{1} << 62);
  }
  size_request(*q, s->cfg.plain_fp32_baseline != 0);
  if (q->dev_bytes > s->cfg.device_budget_bytes || q->host_bytes > s->cfg.host_budget_bytes) {
    size_t need = q->dev_bytes;
    delete q;
    return drr::set_error(DRR_ERR_OOM, "request needs %zu device bytes, more than the server budget", need);
  }
  q->t_submit = Clock::now();
  v->refs.fetch_add(1);
  {
    std::lock_guard<std::mutex> lk(s->mu);
    if (s->stop) {
      v->refs.fetch_sub(1);
      delete q;
      return drr::set_error(DRR_ERR_INVALID, "server is shutting down");
    }
    q->id = s->next_id++;
    s->reqs[q->id] = q;
    s->pending.push_back(q);
    ++s->submitted;
    s->submit_seq.fetch_add(1);
    *ticket = q->id;
  }
  s->cv_loop.notify_all();
  return DRR_OK;
}

drr_status drr_server_wait(drr_server s, uint64_t ticket, int32_t timeout_ms, drr_result* res) {
  if (!s) return drr::set_error(DRR_ERR_INVALID, "server is NULL");
  std::unique_lock<std::mutex> lk(s->mu);
  auto it = s->reqs.find(ticket);
  if (it == s->reqs.end()) return drr::set_error(DRR_ERR_NOT_FOUND, "unknown ticket %llu", (unsigned long long)ticket);
  Req* q = it->second;
  auto ready = [q] { return q->state == kDone; };
  ++s->waiters;  // drr_server_destroy frees nothing while a waiter is inside
  ++q->waiters;  // nor does another waiter on the same ticket
  bool finished = true;
  if (timeout_ms < 0) {
    s->cv_done.wait(lk, ready);
  } else {
    finished = s->cv_done.wait_for(lk, std::chrono::milliseconds(timeout_ms), ready);
  }
  --q->waiters;
  if (--s->waiters == 0) s->cv_done.notify_all();
  if (!finished)
    return drr::set_error(DRR_ERR_TIMEOUT, "ticket %llu not finished after %d ms", (unsigned long long)ticket,
                          timeout_ms);
  if (res) {
    res->status = q->status;
    res->queue_ms = q->tick >= 0 ? ms_between(q->t_submit, q->t_admit) : 0.0;
    res->latency_ms = ms_between(q->t_submit, q->t_done);
    res->tick = q->tick;
  }
  drr_status st = q->status;
  const unsigned int dev_bits = q->device_status;
  // the ticket is released by the last thread that waited on it (every waiter
  // that was inside when the request finished gets its result)
  if (q->waiters == 0) {
    s->reqs.erase(ticket);
    delete q;
  }
  if (st == DRR_ERR_DEVICE)
    return drr::set_error(st, "request %llu: a serving kernel set its status word (bits 0x%x); outputs not written",
                          (unsigned long long)ticket, dev_bits);
  if (st != DRR_OK) return drr::set_error(st, "request %llu did not complete", (unsigned long long)ticket);
  return DRR_OK;
}

drr_status drr_server_poll(drr_server s, uint64_t ticket, int32_t* state) {
  if (!s || !state) return drr::set_error(DRR_ERR_INVALID, "NULL argument");
  std::lock_guard<std::mutex> lk(s->mu);
  auto it = s->reqs.find(ticket);
  if (it == s->reqs.end()) return drr::set_error(DRR_ERR_NOT_FOUND, "unknown ticket %llu", (unsigned long long)ticket);
  const Req* q = it->second;
  *state = q->state == kPending ? DRR_REQ_QUEUED : (q->state == kAdmitted ? DRR_REQ_RUNNING : DRR_REQ_DONE);
  return DRR_OK;
}

drr_status drr_server_inject_device_status(drr_server s, uint64_t ticket, uint32_t bits) {
  if (!s) return drr::set_error(DRR_ERR_INVALID, "server is NULL");
  std::lock_guard<std::mutex> lk(s->mu);
  auto it = s->reqs.find(ticket);
  if (it == s->reqs.end()) return drr::set_error(DRR_ERR_NOT_FOUND, "unknown ticket %llu", (unsigned long long)ticket);
  if (it->second->state != kPending) return drr::set_error(DRR_ERR_BUSY, "request already admitted");
  it->second->inject_status = bits;
  return DRR_OK;
}

drr_status drr_server_cancel(drr_server s, uint64_t ticket) {
  if (!s) return drr::set_error(DRR_ERR_INVALID, "server is NULL");
  std::lock_guard<std::mutex> lk(s->mu);
  auto it = s->reqs.find(ticket);
  if (it == s->reqs.end()) return drr::set_error(DRR_ERR_NOT_FOUND, "unknown ticket %llu", (unsigned long long)ticket);
  Req* q = it->second;
  if (q->state != kPending) return drr::set_error(DRR_ERR_BUSY, "request already admitted");
  s->pending.erase(std::find(s->pending.begin(), s->pending.end(), q));
  q->state = kDone;
  q->status = DRR_ERR_CANCELLED;
  q->t_done = Clock::now();
  q->r.volume->refs.fetch_sub(1);
  ++s->cancelled;
  s->cv_done.notify_all();
  return DRR_OK;
}

drr_status drr_server_get_stats(drr_server s, drr_server_stats* out) {
  if (!s || !out) return drr::set_error(DRR_ERR_INVALID, "NULL argument");
  std::lock_guard<std::mutex> lk(s->mu);
  std::memset(out, 0, sizeof(*out));
  out->submitted = s->submitted;
  out->completed = s->completed;
  out->failed = s->failed;
  out->cancelled = s->cancelled;
  out->ticks = s->ticks;
  out->pending = static_cast<int32_t>(s->pending.size());
  out->inflight = s->admitted;
  out->device_in_use = s->dev_arena->in_use();
  out->device_budget = s->cfg.device_budget_bytes;
  out->gpu_busy_ms = s->gpu_busy_ms;
  if (!s->latencies.empty()) {
    std::vector<double> v = s->latencies;
    std::sort(v.begin(), v.end());
    auto pct = [&v](double p) {
      size_t i = static_cast<size_t>(p * (v.size() - 1) + 0.5);
      return v[std::min(i, v.size() - 1)];
    };
    out->p50_ms = pct(0.50);
    out->p99_ms = pct(0.99);
    out->max_ms = s->lat_max;
    out->mean_ms = s->lat_sum / static_cast<double>(s->lat_count);
  }
  return DRR_OK;
}

drr_status drr_server_pause(drr_server s, int32_t paused) {
  if (!s) return drr::set_error(DRR_ERR_INVALID, "server is NULL");
  {
    std::lock_guard<std::mutex> lk(s->mu);
    s->paused = paused != 0;
  }
  s->cv_loop.notify_all();
  return DRR_OK;
}

drr_status drr_server_destroy(drr_server s) {
  if (!s) return DRR_OK;
  {
    std::lock_guard<std::mutex> lk(s->mu);
    s->stop = true;
    for (Req* q : s->pending) {
      q->state = kDone;
      q->status = DRR_ERR_CANCELLED;
      q->t_done = Clock::now();
      q->r.volume->refs.fetch_sub(1);
      ++s->cancelled;
    }
    s->pending.clear();
  }
  s->cv_loop.notify_all();
  s->cv_done.notify_all();
  if (s->loop.joinable()) s->loop.join();
  s->sync_streams();
  {
    // every request is done now; threads still inside drr_server_wait return
    // once they reacquire the lock, and nothing is freed before they have left
    std::unique_lock<std::mutex> lk(s->mu);
    s->cv_done.notify_all();
    s->cv_done.wait(lk, [s] { return s->waiters == 0; });
  }
  for (auto& kv : s->reqs) delete kv.second;
  s->reqs.clear();
  for (auto& st : s->sets) {
    if (st.graph) cudaGraphExecDestroy(st.graph);
    if (st.h_table) cudaFreeHost(st.h_table);
    if (st.d_table) cudaFree(st.d_table);
    if (st.d_counter) cudaFree(st.d_counter);
    if (st.start) cudaEventDestroy(st.start);
    if (st.stop) cudaEventDestroy(st.stop);
    if (st.in_ready) cudaEventDestroy(st.in_ready);
    if (st.done_ev) cudaEventDestroy(st.done_ev);
  }
  if (s->sets[0].ks) cudaStreamDestroy(s->sets[0].ks);
  cudaFree(s->dev_base);
  cudaFreeHost(s->host_base);
  cudaStreamDestroy(s->h2d);
  cudaStreamDestroy(s->d2h);
  delete s->dev_arena;
  delete s->host_arena;
  delete s;
  return DRR_OK;
}

drr_status drr_serve_tick_layout(int32_t n, const int32_t* B, const drr_detector* dets, int32_t* tile_start,
                                 int32_t* pose_start, int32_t* totals) {
  if (n <= 0 || !B || !dets || !tile_start || !pose_start || !totals)
    return drr::set_error(DRR_ERR_INVALID, "bad arguments");
  std::vector<drr::DetDev> dd(n);
  for (int i = 0; i < n; ++i) {
    if (drr_status s = drr::check_detector(&dets[i], &dd[i])) return s;
    if (B[i] <= 0) return drr::set_error(DRR_ERR_INVALID, "B must be positive");
  }
  if (!layout_tick(n, B, dd.data(), tile_start, pose_start, &totals[0], &totals[1]))
    return drr::set_error(DRR_ERR_INVALID, "tick too large");
  return DRR_OK;
}

// ---- the arena on its own ----------------------------------------------------

struct drr_arena_s {
  drr::OffsetArena a;
  drr_arena_s(size_t c, size_t al) : a(c, al) {}
};

drr_status drr_arena_create(size_t capacity, size_t align, drr_arena* out) {
  if (!out) return drr::set_error(DRR_ERR_INVALID, "out is NULL");
  if (align & (align - 1)) return drr::set_error(DRR_ERR_INVALID, "align must be a power of two");
  *out = new drr_arena_s(capacity, align);
  return DRR_OK;
}

drr_status drr_arena_alloc(drr_arena a, size_t bytes, size_t* offset) {
  if (!a || !offset) return drr::set_error(DRR_ERR_INVALID, "NULL argument");
  if (!a->a.alloc(bytes, offset)) return drr::set_error(DRR_ERR_OOM, "no free run of %zu bytes", bytes);
  return DRR_OK;
}

drr_status drr_arena_free(drr_arena a, size_t offset) {
  if (!a) return drr::set_error(DRR_ERR_INVALID, "NULL argument");
  if (!a->a.release(offset)) return drr::set_error(DRR_ERR_NOT_FOUND, "offset %zu is not allocated", offset);
  return DRR_OK;
}

size_t drr_arena_in_use(drr_arena a) { return a ? a->a.in_use() : 0; }
size_t drr_arena_largest_free(drr_arena a) { return a ? a->a.largest_free() : 0; }

drr_status drr_arena_destroy(drr_arena a) {
  delete a;
  return DRR_OK;
}

}  // extern "C"
