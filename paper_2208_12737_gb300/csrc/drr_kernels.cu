// libdrr kernels: pose/ray setup, incremental Siddon traversal (forward,
// fused pose Jacobian, pose-gradient re-trace, back-projection), the
// deterministic pose-gradient reduction and volume ingest.
//
// Paper: Gopalakrishnan & Golland, arXiv 2208.12737.
//   Eq. (2)  radiologic path length E = |p-s| sum (a_{m+1}-a_m) V[midpoint voxel]
//   Eq. (3)  plane crossings a_x(i) = (b_x + i dX - s_x) / (p_x - s_x)
//   Sec. 2.2 Siddon-Jacobs: the next crossing is the minimum over the axes of
//            each axis' next plane, iterated until the ray leaves the volume
//   Sec. 2.3 entry/exit clip a_min / a_max
//   Sec. 2.4 pose parameterisation and differentiation w.r.t. the pose
#include <algorithm>
#include <cstdint>

#include <cooperative_groups.h>
#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include "drr_internal.cuh"

namespace drr {
namespace {

enum Mode : int { kFwd = 0, kFwdJac = 1, kPoseGrad = 2, kBackproject = 3, kCount = 4, kGeoGrad = 5 };

template <int DT>
struct Voxel;
template <>
struct Voxel<kF32> {
  static __device__ __forceinline__ float load(const void* base, int off) {
    return __ldg(static_cast<const float*>(base) + off);
  }
};
template <>
struct Voxel<kBF16> {
  static __device__ __forceinline__ float load(const void* base, int off) {
    const unsigned short u = __ldg(static_cast<const unsigned short*>(base) + off);
    return __uint_as_float(static_cast<unsigned int>(u) << 16);
  }
};
template <>
struct Voxel<kF16> {
  static __device__ __forceinline__ float load(const void* base, int off) {
    return __half2float(__ldg(static_cast<const __half*>(base) + off));
  }
};

// Bounds-checked build (-DDRR_CHECK_BOUNDS=1, a separate library built for
// tests): every voxel gather is checked against the padded volume and every
// back-projection add of a live segment against the gradient volume; a check
// that fails sets a bit of a device-wide fault word (read and cleared by
// drr_stream_check, which then returns DRR_ERR_DEVICE) and skips the access.
// The product build has no checks: the zero padding keeps every gather of the
// walk in bounds, which the checked build verifies on the parity workloads.
#ifndef DRR_CHECK_BOUNDS
#define DRR_CHECK_BOUNDS 0
#endif
enum FaultBits : unsigned int { kFaultGather = 1u, kFaultBackproject = 2u };
#if DRR_CHECK_BOUNDS
__device__ unsigned int g_fault_word = 0u;
#endif
template <int DT>
__device__ __forceinline__ float gather(const VolumeDev& vd, int off) {
#if DRR_CHECK_BOUNDS
  if (static_cast<unsigned long long>(static_cast<long long>(off)) >= static_cast<unsigned long long>(vd.elems)) {
    atomicOr(&g_fault_word, kFaultGather);
    return 0.f;
  }
#endif
  return Voxel<DT>::load(vd.data, off);
}

// x_a for a runtime axis index without indexing a register array (which
// would move the array to local memory).
template <class T>
__device__ __forceinline__ T pick3(int a, T x0, T x1, T x2) {
  return a == 0 ? x0 : (a == 1 ? x1 : x2);
}

// Programmatic dependent launch (sm_90 and later).  The pose-setup, walk and
// gradient-reduction kernels are launched with programmatic stream
// serialization, so each can be scheduled while the kernel before it in the
// stream is still finishing.  grid_dep_wait() blocks until that kernel has
// completed and its writes are visible; each of these kernels calls it before
// its first global-memory access (read or write).  grid_dep_release() lets the
// next kernel in the stream be scheduled early; its blocks then wait in their
// own grid_dep_wait().  Both are no-ops for a kernel launched without the
// attribute.
__device__ __forceinline__ void grid_dep_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void grid_dep_release() { asm volatile("griddepcontrol.launch_dependents;" :::); }

// ---------------------------------------------------------------------------
// Pose -> frame (Sec. 2.4).  R = Rz(eta0) Ry(eta1) Rx(eta2).
// ---------------------------------------------------------------------------
// World-space frame of one pose: source s, pixel (0,0) centre p00, the
// per-column and per-row pixel steps ew, eh (all FP64), and optionally R and
// the sines / cosines of the three angles.  R = Rz Ry Rx written out.
__device__ void pose_frame(const float* pose, const DetDev& det, double s[3], double p00[3], double ew[3],
                           double eh[3], double sc_out[3], double pc00_out[3], double* R_out /*9 or null*/,
                           float* sincos_out /*6 or null: sz, cz, sy, cy, sx, cx*/) {
  double sz, cz, sy, cy, sx, cx;
  sincos(static_cast<double>(pose[0]), &sz, &cz);
  sincos(static_cast<double>(pose[1]), &sy, &cy);
  sincos(static_cast<double>(pose[2]), &sx, &cx);
  const double szsy = sz * sy, czsy = cz * sy;
  const double R[9] = {cz * cy, fma(czsy, sx, -sz * cx), fma(czsy, cx, sz * sx),
                       sz * cy, fma(szsy, sx, cz * cx),  fma(szsy, cx, -cz * sx),
                       -sy,     cy * sx,                 cy * cx};
  const double rho = 0.5 * static_cast<double>(det.sdr);
  const double pw = -0.5 * static_cast<double>(det.W - 1) * static_cast<double>(det.dw);
  const double ph = -0.5 * static_cast<double>(det.H - 1) * static_cast<double>(det.dh);
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    const double t = static_cast<double>(pose[3 + a]);
    s[a] = fma(rho, R[3 * a], t);                                              // R (rho, 0, 0) + t
    p00[a] = fma(ph, R[3 * a + 2], fma(pw, R[3 * a + 1], fma(-rho, R[3 * a], t)));  // R pc00 + t
    ew[a] = static_cast<double>(det.dw) * R[3 * a + 1];                         // R (0, dw, 0)
    eh[a] = static_cast<double>(det.dh) * R[3 * a + 2];                         // R (0, 0, dh)
  }
  sc_out[0] = rho;
  sc_out[1] = sc_out[2] = 0.0;
  pc00_out[0] = -rho;
  pc00_out[1] = pw;
  pc00_out[2] = ph;
  if (R_out) {
#pragma unroll
    for (int i = 0; i < 9; ++i) R_out[i] = R[i];
  }
  if (sincos_out) {
    sincos_out[0] = static_cast<float>(sz);
    sincos_out[1] = static_cast<float>(cz);
    sincos_out[2] = static_cast<float>(sy);
    sincos_out[3] = static_cast<float>(cy);
    sincos_out[4] = static_cast<float>(sx);
    sincos_out[5] = static_cast<float>(cx);
  }
}

__device__ void mul3f(const float* A, const float* B, float* C) {
#pragma unroll
  for (int r = 0; r < 3; ++r)
#pragma unroll
    for (int c = 0; c < 3; ++c) C[3 * r + c] = fmaf(A[3 * r], B[c], fmaf(A[3 * r + 1], B[3 + c], A[3 * r + 2] * B[6 + c]));
}

__device__ void apply3f(const float* A, const float* x, float* y) {
#pragma unroll
  for (int r = 0; r < 3; ++r) y[r] = fmaf(A[3 * r], x[0], fmaf(A[3 * r + 1], x[1], A[3 * r + 2] * x[2]));
}

// FP32 chain-rule terms of one pose (dR/d eta_j applied to s_c, p_c - s_c and the
// pixel steps), from the FP32-rounded sines and cosines: they are stored as FP32.
__device__ void chain_terms(const float cs[6], const float t[3], double rho, double pw, double ph, const DetDev& det,
                            PoseGeom* g) {
  const float sz = cs[0], cz = cs[1], sy = cs[2], cy = cs[3], sx = cs[4], cx = cs[5];
  const float Rz[9] = {cz, -sz, 0.f, sz, cz, 0.f, 0.f, 0.f, 1.f};
  const float Ry[9] = {cy, 0.f, sy, 0.f, 1.f, 0.f, -sy, 0.f, cy};
  const float Rx[9] = {1.f, 0.f, 0.f, 0.f, cx, -sx, 0.f, sx, cx};
  const float dRz[9] = {-sz, -cz, 0.f, cz, -sz, 0.f, 0.f, 0.f, 0.f};
  const float dRy[9] = {-sy, 0.f, cy, 0.f, 0.f, 0.f, -cy, 0.f, -sy};
  const float dRx[9] = {0.f, 0.f, 0.f, 0.f, -sx, -cx, 0.f, cx, -sx};
  float T[9], U[9], dR[27];
  mul3f(Rz, Ry, T);
  mul3f(dRz, Ry, U);
  mul3f(U, Rx, dR);
  mul3f(Rz, dRy, U);
  mul3f(U, Rx, dR + 9);
  mul3f(T, dRx, dR + 18);
  // angular velocities of the three angles in the world frame, dR_j R^T x =
  // omega_j x x: rz turns about e_z, ry about Rz e_y, rx about Rz Ry e_x
  const float om[9] = {0.f, 0.f, 1.f, -sz, cz, 0.f, cz * cy, sz * cy, -sy};
  const float q[3] = {static_cast<float>(-2.0 * rho), static_cast<float>(pw), static_cast<float>(ph)};
  const float vw[3] = {0.f, det.dw, 0.f};
  const float vh[3] = {0.f, 0.f, det.dh};
#pragma unroll
  for (int j = 0; j < 3; ++j) {
#pragma unroll
    for (int a = 0; a < 3; ++a) g->Om[j][a] = om[3 * j + a];
    apply3f(dR + 9 * j, q, g->Q[j]);
    apply3f(dR + 9 * j, vw, g->Wv[j]);
    apply3f(dR + 9 * j, vh, g->Hv[j]);
  }
#pragma unroll
  for (int a = 0; a < 3; ++a) g->t[a] = t[a];
  g->hc = 0.5f * static_cast<float>(det.H - 1);
  g->wc = 0.5f * static_cast<float>(det.W - 1);
}

// Per-pose geometry in the volume's voxel units plus the chain-rule terms,
// computed by a whole warp and written to *g.  The three FP64 sine/cosine pairs
// run in lanes 0-2 and the per-axis terms in lanes 0-2: FP64 issue is narrow on
// this GPU, and spreading the serial FP64 work over lanes shortens the kernel.
// The arithmetic per value is that of pose_frame.
__device__ void warp_pose_geom(const float* pose, const DetDev& det, const VolumeDev& vd, PoseGeom* g) {
  constexpr unsigned int kFull = 0xffffffffu;
  const int lane = threadIdx.x & 31;
  double sv = 0.0, cv = 1.0;
  if (lane < 3) sincos(static_cast<double>(pose[lane]), &sv, &cv);
  const double sz = __shfl_sync(kFull, sv, 0), cz = __shfl_sync(kFull, cv, 0);
  const double sy = __shfl_sync(kFull, sv, 1), cy = __shfl_sync(kFull, cv, 1);
  const double sx = __shfl_sync(kFull, sv, 2), cx = __shfl_sync(kFull, cv, 2);
  const double szsy = sz * sy, czsy = cz * sy;
  const double R[9] = {cz * cy, fma(czsy, sx, -sz * cx), fma(czsy, cx, sz * sx),
                       sz * cy, fma(szsy, sx, cz * cx),  fma(szsy, cx, -cz * sx),
                       -sy,     cy * sx,                 cy * cx};
  const double rho = 0.5 * static_cast<double>(det.sdr);
  const double pw = -0.5 * static_cast<double>(det.W - 1) * static_cast<double>(det.dw);
  const double ph = -0.5 * static_cast<double>(det.H - 1) * static_cast<double>(det.dh);
  if (lane < 3) {
    const int a = lane;
    const double r0 = pick3(a, R[0], R[3], R[6]), r1 = pick3(a, R[1], R[4], R[7]), r2 = pick3(a, R[2], R[5], R[8]);
    const double t = static_cast<double>(pose[3 + a]);
    const double s = fma(rho, r0, t);                                  // R (rho, 0, 0) + t
    const double p00 = fma(ph, r2, fma(pw, r1, fma(-rho, r0, t)));     // R pc00 + t
    const double ew = static_cast<double>(det.dw) * r1;                 // R (0, dw, 0)
    const double eh = static_cast<double>(det.dh) * r2;                 // R (0, 0, dh)
    const double dl = static_cast<double>(pick3(a, vd.delta[0], vd.delta[1], vd.delta[2]));
    const int na = pick3(a, vd.n[0], vd.n[1], vd.n[2]);
    const double lo = -0.5 * static_cast<double>(na) * dl;  // b_a: volume centred at the origin
    const double u0 = (s - lo) / dl;
    const double un = static_cast<double>(na) - u0;
    g->u0[a] = u0;
    g->un[a] = un;
    g->u0f[a] = static_cast<float>(u0);
    g->unf[a] = static_cast<float>(un);
    g->g00[a] = (p00 - s) / dl;
    g->gw[a] = ew / dl;
    g->gh[a] = eh / dl;
  }
  // columns of R (R e_x, R e_y, R e_z) for the detector-parameter chain
#pragma unroll
  for (int i = 0; i < 9; ++i)
    if (lane == i) g->Rc[i % 3][i / 3] = static_cast<float>(R[i]);
  if (lane == 0) {
    const float cs[6] = {static_cast<float>(sz), static_cast<float>(cz), static_cast<float>(sy),
                         static_cast<float>(cy), static_cast<float>(sx), static_cast<float>(cx)};
    const float tr[3] = {pose[3], pose[4], pose[5]};
    chain_terms(cs, tr, rho, pw, ph, det, g);
  }
}

// One warp (block) per pose.
__global__ void __launch_bounds__(32) pose_setup_kernel(const float* __restrict__ poses, int B, DetDev det,
                                                        VolumeDev vd, PoseGeom* __restrict__ out) {
  grid_dep_wait();
  grid_dep_release();
  const int b = blockIdx.x;
  // the walk kernels' tile counters live in the slot after the last pose
  if (b == 0 && threadIdx.x < kLaunchCounters) reinterpret_cast<unsigned int*>(out + B)[threadIdx.x] = 0u;
  if (b >= B) return;
  warp_pose_geom(poses + 6 * b, det, vd, out + b);
}

__global__ void ray_setup_kernel(const float* __restrict__ poses, int B, DetDev det, float* __restrict__ rays) {
  const int64_t i = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
  const int64_t npix = static_cast<int64_t>(det.H) * det.W;
  if (i >= npix * B) return;
  const int b = static_cast<int>(i / npix);
  const int q = static_cast<int>(i % npix);
  const int h = q / det.W, w = q % det.W;
  double s[3], p00[3], ew[3], eh[3], sc[3], pc00[3];
  pose_frame(poses + 6 * b, det, s, p00, ew, eh, sc, pc00, nullptr, nullptr);
  float* r = rays + 6 * i;
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    r[a] = static_cast<float>(s[a]);
    r[3 + a] = static_cast<float>(fma(static_cast<double>(h), eh[a], fma(static_cast<double>(w), ew[a], p00[a])));
  }
}

// ---------------------------------------------------------------------------
// One ray: FP64 clip and entry (Sec. 2.3), then the FP32 incremental walk.
// ---------------------------------------------------------------------------
struct RayResult {
  float F;     // E (or the raw sum in alpha units before the final scaling)
  float J[6];  // dE/d eta (only for the Jacobian modes)
  int nseg;    // number of segments (0 for a miss)
};

// Per-ray state after the FP64 setup: everything the walk needs.
//
// Crossing parameters are fixed point: alpha measured from the entry is held
// as a 32.32 number in units of span / 2^24 (span = alpha_max - alpha_min), so
// the high word of every crossing inside the ray lies in [0, 2^24] and the
// exit is exactly 2^24; every value the walk forms stays below 2^58.  Each
// axis' crossings form the arithmetic sequence first + k * delta (Eq. 3),
// advanced by exact 64-bit additions: ordering is exact to 2^-56 of the span
// and segment lengths are exact integers, so the FP32 arithmetic is confined
// to the accumulation of length x density.  (A high word below 2^24 converts
// to FP32 exactly; see fix_to_float.)
struct RaySetup {
  int nseg;                  // segments = plane crossings + 1 (0: the ray misses)
  int off;                   // element offset of the entry voxel (padded layout)
  int ient[3];               // entry voxel index per axis
  int cnt[3];                // plane crossings per axis between the entry and exit voxels
  int step[3];               // signed element stride per axis
  int ea, xa;                // axis of the entry / exit plane, -1 when clamped to alpha = 0 / 1
  unsigned long long A0[3];  // first crossing per axis (32.32 fixed point)
  unsigned long long D[3];   // fixed-point distance between consecutive planes
  float unit;                // alpha per high-word unit: span / 2^24
  double amin;               // absolute alpha of the entry
  float d[3];                // p - s in mm
};

constexpr unsigned int kExitUnits = 1u << 24;              // the exit, in high-word units
constexpr unsigned long long kFixMax = 1ull << 56;         // fixed-point value of the exit
constexpr unsigned long long kNoCrossing64 = 1ull << 58;  // beyond any crossing of the ray
constexpr double kFixScale = 72057594037927936.0;          // 2^56: fixed-point value of alpha = span

// Reciprocal of a double to ~1e-14 relative: an FP32 seed refined by one FP64
// Newton step (a full FP64 division costs several times more on the FP64 pipe,
// which is narrow on this GPU).  Exact division outside the FP32 seed's range.
__device__ __forceinline__ double rcp_fast(double x) {
  const float xf = static_cast<float>(x);
  const float ax = fabsf(xf);
  if (!(ax > 1e-30f && ax < 1e30f)) return 1.0 / x;
  const double r = static_cast<double>(__frcp_rn(xf));
  return fma(r, fma(-x, r, 1.0), r);
}

// floor of a double: in FP32 unless the value is within 2^-10 of an integer
// (or too large for FP32 to resolve that), where FP64 decides.
__device__ __forceinline__ int floor_fast(double x) {
  const float xf = static_cast<float>(x);
  const float fl = floorf(xf);
  const float fr = xf - fl;
  if (fabsf(xf) < 4096.f && fr > 9.765625e-4f && fr < 1.f - 9.765625e-4f) return static_cast<int>(fl);
  return static_cast<int>(floor(x));
}

// FP64 clip (Sec. 2.3, clamped to [0, 1]), entry/exit voxels and first
// crossings.  The faces the ray enters and leaves through are found in FP32
// (in FP64 where FP32 cannot tell them apart); alpha_min / alpha_max are then
// evaluated in FP64 on those faces.  Returns 1 for a hit, 0 when the ray
// misses, -1 for non-finite geometry.
// kEntry: also the entry point s + amin (p - s) in world coordinates (mm, from
// the FP64 entry) into e[3], for the pose Jacobian.
template <bool kEntry>
__device__ __forceinline__ int ray_setup(const VolumeDev& vd, const PoseGeom& pg, int h, int w, RaySetup& r,
                                         float* e = nullptr) {
  double g[3];
  float gf[3];
  bool finite = true;
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    g[a] = fma(static_cast<double>(h), pg.gh[a], fma(static_cast<double>(w), pg.gw[a], pg.g00[a]));
    gf[a] = static_cast<float>(g[a]);
    finite = finite && isfinite(gf[a]) && isfinite(pg.u0f[a]);
  }
  r.nseg = 0;
  if (!finite) return -1;
  // faces in FP32; a choice that FP32 cannot make safely -- the runner-up
  // crossing (or the clamp at alpha 0 / 1) within 2^-20 of the chosen one, four
  // times the FP32 error of these products, or a hit test that close -- is
  // made again in FP64.  That matters where the clipped span is a small part of
  // alpha (a small volume far from the source): there an FP32 tie moves the
  // entry by a visible share of the span.
  float lof = 0.f, hif = 1.f, lo2 = -1.f, hi2 = 2.f;  // chosen and runner-up entry / exit
  int ea = -1, xa = -1;
  bool hit = true;
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    if (g[a] != 0.0) {
      const float rf = __frcp_rn(gf[a]);
      const float t0 = -pg.u0f[a] * rf, t1 = pg.unf[a] * rf;
      const float lo = fminf(t0, t1), hi = fmaxf(t0, t1);
      if (lo > lof) { lo2 = lof; lof = lo; ea = a; } else lo2 = fmaxf(lo2, lo);
      if (hi < hif) { hi2 = hif; hif = hi; xa = a; } else hi2 = fminf(hi2, hi);
    } else if (!(pg.u0[a] >= 0.0 && pg.un[a] > 0.0)) {
      hit = false;
    }
  }
  if (!hit) return 0;
  const float tol = 9.5367431640625e-7f * fmaxf(fabsf(lof), fabsf(hif)) + 1e-30f;  // 2^-20
  const bool exact = lof - lo2 < tol || hi2 - hif < tol || fabsf(hif - lof) < tol;
  if (!exact && !(lof < hif)) return 0;
  double rg[3];
#pragma unroll
  for (int a = 0; a < 3; ++a) rg[a] = g[a] != 0.0 ? rcp_fast(g[a]) : 0.0;
  // entry / exit faces: plane 0 when the ray runs up the axis, plane n otherwise
  double amin = 0.0, amax = 1.0;
  if (exact) {
    ea = xa = -1;
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      if (g[a] != 0.0) {
        const double en = (g[a] > 0.0 ? -pg.u0[a] : pg.un[a]) * rg[a];
        const double ex = (g[a] > 0.0 ? pg.un[a] : -pg.u0[a]) * rg[a];
        if (en > amin) { amin = en; ea = a; }
        if (ex < amax) { amax = ex; xa = a; }
      }
    }
  } else {
#pragma unroll
    for (int a = 0; a < 3; ++a) {  // static indices: the arrays stay in registers
      if (a == ea) amin = (g[a] > 0.0 ? -pg.u0[a] : pg.un[a]) * rg[a];
      if (a == xa) amax = (g[a] > 0.0 ? pg.un[a] : -pg.u0[a]) * rg[a];
    }
  }
  if (!(amin < amax)) return 0;
  r.ea = ea;
  r.xa = xa;
  r.amin = amin;
  const double span = amax - amin;
  const double to_fix = kFixScale * rcp_fast(span);  // fixed-point units per unit of alpha
  r.unit = static_cast<float>(span) * (1.f / static_cast<float>(kExitUnits));
  int total = 0;
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    const int n = vd.n[a];
    r.d[a] = gf[a] * vd.delta[a];
    // entry position u_e (voxel units) and its world point (volume centred at
    // the origin); u_e lies in [0, n], so FP32 holds it to ~1e-7 voxel
    const double ue = fma(amin, g[a], pg.u0[a]);
    if (kEntry) e[a] = fmaf(static_cast<float>(ue), vd.delta[a], -0.5f * static_cast<float>(n) * vd.delta[a]);
    if (g[a] == 0.0) {
      r.ient[a] = min(max(static_cast<int>(floor(pg.u0[a])), 0), n - 1);
      r.cnt[a] = 0;
      r.A0[a] = kNoCrossing64;
      r.D[a] = 0ull;
      r.step[a] = vd.stride[a];
      continue;
    }
    const bool up = g[a] > 0.0;
    const double ux = fma(amax, g[a], pg.u0[a]);
    int i0, i1;
    if (a == ea) i0 = up ? 0 : n - 1;
    else i0 = up ? floor_fast(ue) : -floor_fast(-ue) - 1;
    if (a == xa) i1 = up ? n - 1 : 0;
    else i1 = up ? -floor_fast(-ux) - 1 : floor_fast(ux);
    i0 = min(max(i0, 0), n - 1);
    i1 = min(max(i1, 0), n - 1);
    r.ient[a] = i0;
    r.cnt[a] = max(up ? i1 - i0 : i0 - i1, 0);
    total += r.cnt[a];
    const double plane = static_cast<double>(up ? i0 + 1 : i0);
    // first crossing, kept within [0, span] (rounding can put it a hair outside)
    const double f = fmax((plane - ue) * rg[a], 0.0);
    r.A0[a] = r.cnt[a] > 0 ? min(__double2ull_rz(f * to_fix), kFixMax) : kNoCrossing64;
    // plane spacing, saturated at the span: an axis whose planes are farther
    // apart has at most one crossing, and one step past it stays below 2^57
    r.D[a] = min(__double2ull_rz(fabs(rg[a]) * to_fix), kFixMax);
    r.step[a] = up ? vd.stride[a] : -vd.stride[a];
  }
  r.nseg = total + 1;
  r.off = vd.origin + r.ient[0] * vd.stride[0] + r.ient[1] * vd.stride[1] + r.ient[2] * vd.stride[2];
  return 1;
}

// ---------------------------------------------------------------------------
// Chunked walk.  The exact fixed-point crossing positions are the reference
// frame, but the per-segment arithmetic runs in FP32 on positions measured from
// a nearby origin: at the start of every chunk of crossings the next crossing
// of each axis is recomputed exactly (first + k * delta in 64-bit) relative to
// the exact position of the current point, so local positions stay below
// ~chunk plane gaps and carry 2^-24 of the chunk instead of 2^-24 of the ray's
// alpha as a whole-ray FP32 walk would.  Positions are in fixed-point
// high-word units (span / 2^24).
// ---------------------------------------------------------------------------
#ifndef DRR_FWD_MINB
#define DRR_FWD_MINB 4
#endif
#ifndef DRR_JAC_MINB
#define DRR_JAC_MINB 4
#endif
constexpr float kTwoM32 = 2.3283064365386963e-10f;  // 2^-32

// Per-thread exact crossing parameters, kept in shared memory: they are read
// only when a chunk starts (and on the rare exact tie path).
struct WalkScratch {
  unsigned long long A0[3][kThreads];
  unsigned long long D[3][kThreads];
};
// The Jacobian walk also keeps the state at the start of the current chunk,
// for an exact re-walk of the chunk.  (Shared memory comes out of the same
// on-chip store as the L1 cache that serves the voxel gathers, so each kernel
// declares only what its walk uses.)
struct JacScratch : WalkScratch {
  int cnt[3][kThreads];  // crossings per slot (read only by the exact re-walk)
  float e[3][kThreads];  // the ray's entry point (read only by the Jacobian epilogue)
  int c_off[kThreads];
  float c_v[kThreads], c_vprev[kThreads];
  int c_pend[kThreads];
};

__device__ __forceinline__ unsigned long long fix_at(unsigned long long A0, unsigned long long D, unsigned int k) {
  return A0 + static_cast<unsigned long long>(k) * D;
}

// FP32 value (high-word units) of a signed 32.32 fixed-point number, from two
// 32-bit conversions (a 64-bit conversion would run on the FP64 pipe, which is
// narrow on this GPU).  For |d| < 2^56 -- every position within a ray, every
// plane spacing -- the high word converts exactly, so the result carries one
// rounding (2^-24 relative) plus at most 2^-25 units from the low word.
__device__ __forceinline__ float fix_to_float(long long d) {
  return fmaf(static_cast<float>(static_cast<unsigned int>(d)), kTwoM32, static_cast<float>(static_cast<int>(d >> 32)));
}

// Next crossings of two axes, l * delta + x0 each, in one packed two-lane FP32
// FMA (each lane rounded as fmaf rounds it, so the results are the same);
// -DDRR_PACKED_XY=0 issues two scalar FMAs.
#ifndef DRR_PACKED_XY
#define DRR_PACKED_XY 1
#endif
__device__ __forceinline__ void next_xy(float& tx, float& ty, float lx, float ly, float dx, float dy, float x0,
                                        float y0) {
#if DRR_PACKED_XY
  const float2 t = __ffma2_rn(make_float2(lx, ly), make_float2(dx, dy), make_float2(x0, y0));
  tx = t.x;
  ty = t.y;
#else
  tx = fmaf(lx, dx, x0);
  ty = fmaf(ly, dy, y0);
#endif
}

// One forward-walk step in predicated PTX: an = min(tx, ty, tz); the axis it
// belongs to (x before y before z on ties) steps: its crossing counter + 1 and
// the voxel offset by its stride, each as a guarded add, where the compiler's
// code for the same C++ (kept below, -DDRR_FWD_PTX=0) spends selects on the
// busier ALU pipe (forward 0.384 -> 0.377 ms on the CT batch, same DRR bits).
// The Jacobian walk keeps the C++ form: it carries each step's axis
// predicates to the next step's weight accounting, which an asm block cannot.
#ifndef DRR_FWD_PTX
#define DRR_FWD_PTX 1
#endif
__device__ __forceinline__ float walk_step(float tx, float ty, float tz, float& lx, float& ly, float& lz, int& off,
                                           int sx, int sy, int sz) {
  float an;
  asm("{\n\t"
      ".reg .pred px, py, pxy;\n\t"
      "min.f32 %0, %5, %6;\n\t"
      "min.f32 %0, %0, %7;\n\t"
      "setp.eq.f32 px, %5, %0;\n\t"
      "setp.eq.and.f32 py, %6, %0, !px;\n\t"
      "or.pred pxy, px, py;\n\t"
      "@px add.f32 %1, %1, 0f3F800000;\n\t"
      "@py add.f32 %2, %2, 0f3F800000;\n\t"
      "@!pxy add.f32 %3, %3, 0f3F800000;\n\t"
      "@px add.s32 %4, %4, %8;\n\t"
      "@py add.s32 %4, %4, %9;\n\t"
      "@!pxy add.s32 %4, %4, %10;\n\t"
      "}"
      : "=&f"(an), "+f"(lx), "+f"(ly), "+f"(lz), "+r"(off)
      : "f"(tx), "f"(ty), "f"(tz), "r"(sx), "r"(sy), "r"(sz));
  return an;
}

// Local FP32 position of an exact position relative to O.
__device__ __forceinline__ float local_pos(unsigned long long x, unsigned long long O) {
  return fix_to_float(static_cast<long long>(x - O));
}

// Both walks gather two crossings ahead: the first crossing of a chunk is
// peeled and the unrolled loop runs chunk - 1 times.  The three voxel registers
// of that pipeline rotate without register moves when the unroll is a multiple
// of 3.  The Jacobian walk's 6 divides chunk - 1 for every chunk length; the
// forward walk's 12 divides it for its long-ray chunks (121, 181) and for 13.
// (Measured on the CT batch: forward 6 / 12 / 24 at 0.376 / 0.371 / 0.375 ms,
// Jacobian 3 / 6 / 12 at 0.649 / 0.556 / 0.563 ms.)
#ifndef DRR_FWD_UNROLL
#define DRR_FWD_UNROLL 12
#endif
#ifndef DRR_JAC_UNROLL
#define DRR_JAC_UNROLL 6
#endif
constexpr int kFwdUnroll = DRR_FWD_UNROLL;
constexpr int kJacUnroll = DRR_JAC_UNROLL;
// Chunk length per ray.  The FP32 error of a local position grows with the
// chunk's share of the ray, so long rays take long chunks (fewer exact
// re-anchorings) and short rays short ones; 6k + 1 crossings.  The Jacobian
// walk stays at 61 for long rays: its tie test's threshold grows with the
// positions, so longer chunks are flagged (and walked twice) more often.  The
// forward walk has no tie test and takes 121 / 181 for rays of more than 512 /
// 1024 segments (on the CT workload: 3 % faster, worst pixel error unchanged).
#ifndef DRR_JAC_LONG
#define DRR_JAC_LONG 61
#endif
__device__ __forceinline__ int walk_chunk(int nseg) {
  return nseg > 512 ? DRR_JAC_LONG : nseg > 256 ? 31 : nseg > 128 ? 19 : 13;
}
__device__ __forceinline__ int fwd_chunk(int nseg) {
  return nseg > 1024 ? 181 : nseg > 512 ? 121 : walk_chunk(nseg);
}

// Forward walk (Eq. 2 with the crossings of Eq. 3 taken in order, Sec. 2.2).
// The gathers run two crossings ahead of the accumulation (the first crossing
// of a chunk is peeled); the segment that ends at a chunk's last crossing takes
// that crossing's exact position.
template <int DT>
__device__ __forceinline__ float walk_forward(const VolumeDev& vd, const RaySetup& r, WalkScratch* ws) {
  const int t = threadIdx.x;
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    ws->A0[a][t] = r.A0[a];
    ws->D[a][t] = r.D[a];
  }
  const float dx = fix_to_float(static_cast<long long>(r.D[0])), dy = fix_to_float(static_cast<long long>(r.D[1])),
              dz = fix_to_float(static_cast<long long>(r.D[2]));
  unsigned int kx = 0u, ky = 0u, kz = 0u;  // crossings consumed per axis before this chunk
  unsigned long long O = 0ull;              // exact position of the current point
  int off = r.off;
  float v = gather<DT>(vd, off);
  float acc = 0.f;
  int remaining = r.nseg - 1;
  const int chunk = fwd_chunk(r.nseg);
  while (remaining > 0) {
    const float x0 = local_pos(fix_at(ws->A0[0][t], ws->D[0][t], kx), O);
    const float y0 = local_pos(fix_at(ws->A0[1][t], ws->D[1][t], ky), O);
    const float z0 = local_pos(fix_at(ws->A0[2][t], ws->D[2][t], kz), O);
    float tx = x0, ty = y0, tz = z0;
    float lx = 0.f, ly = 0.f, lz = 0.f;
    const int n = min(remaining, chunk);
#if DRR_FWD_PTX
#define DRR_FSTEP(an)                                                                     \
  const float an = walk_step(tx, ty, tz, lx, ly, lz, off, r.step[0], r.step[1], r.step[2]); \
  {                                                                                       \
    next_xy(tx, ty, lx, ly, dx, dy, x0, y0);                                              \
    tz = fmaf(lz, dz, z0);                                                                \
  }
#else
#define DRR_FSTEP(an)                                       \
  const float an = fminf(fminf(tx, ty), tz);                \
  {                                                         \
    const bool bx = tx == an;                               \
    const bool by = !bx && ty == an;                        \
    const bool bz = !bx && !by;                             \
    off += bx ? r.step[0] : (by ? r.step[1] : r.step[2]);   \
    if (bx) lx += 1.f;                                      \
    if (by) ly += 1.f;                                      \
    if (bz) lz += 1.f;                                      \
    next_xy(tx, ty, lx, ly, dx, dy, x0, y0);                \
    tz = fmaf(lz, dz, z0);                                  \
  }
#endif
    DRR_FSTEP(a1)
    float an1 = a1;
    float v1 = gather<DT>(vd, off);
    float ac = 0.f;
#pragma unroll kFwdUnroll
    for (int m = 1; m < n; ++m) {
      DRR_FSTEP(an2)
      const float v2 = gather<DT>(vd, off);
      acc = fmaf(an1 - ac, v, acc);
      ac = an1;
      an1 = an2;
      v = v1;
      v1 = v2;
    }
#undef DRR_FSTEP
    remaining -= n;
    kx += static_cast<unsigned int>(lx);
    ky += static_cast<unsigned int>(ly);
    kz += static_cast<unsigned int>(lz);
    unsigned long long Onew = O;
    if (kx) Onew = max(Onew, fix_at(ws->A0[0][t], ws->D[0][t], kx - 1u));
    if (ky) Onew = max(Onew, fix_at(ws->A0[1][t], ws->D[1][t], ky - 1u));
    if (kz) Onew = max(Onew, fix_at(ws->A0[2][t], ws->D[2][t], kz - 1u));
    acc = fmaf(local_pos(Onew, O) - ac, v, acc);  // the segment ending at the chunk's last crossing, exact end
    v = v1;
    O = Onew;
  }
  acc = fmaf(local_pos(static_cast<unsigned long long>(kExitUnits) << 32, O), v, acc);
  return acc * r.unit;
}

// Walk with the pose-Jacobian bookkeeping (Sec. 2.4).  Crossing k with weight
// w_k = V_before - V_after adds to per-axis sums G_a = sum w, A_a = sum w alpha
// (alpha from the entry).  The axes are relabelled per ray so that slot 2 is the
// axis with most crossings; only slots 0 and 1 are summed and slot 2 follows
// from sum_k w_k = 0 and sum_k w_k alpha_k = F over all crossings, entry and
// exit included (end points clamped to alpha = 0 or 1 belong to no axis and are
// kept in Gc, Ac).
//
// The order of two crossings decides the voxel between them and hence both
// weights, so it must be exact.  A chunk's FP32 position t = l * dl + x0 (x0
// and dl each one rounding from exact values, see fix_to_float, then the FMA)
// is within 2^-24 (x0 + l dl + t) + (l + 1) 2^-25 = 2^-23 t + (l + 1) 2^-25
// units of the exact one, so the walk can only misorder two crossings less
// than 2^-22 t + 62 * 2^-24 apart, and then it takes a segment no longer than
// that at the misordered pair.  So each chunk tracks its shortest segment and
// the gap to the next crossing after it; if either is below kTieRel * position
// + kTieAbs (25 % and ~250x above those two terms), the chunk is walked again
// from its saved start state in exact fixed-point order (rare: about one lane
// in two thousand chunks).
// Sums are kept per chunk in local positions and moved to the anchor frame
// when the chunk ends, so a re-walk only discards the chunk's own sums.
struct JacSums {
  float F, G[3], A[3], Gc, Ac;
  int dom;
};

constexpr float kTieRel = 2.98023223876953125e-7f;  // 1.25 * 2^-22
constexpr float kTieAbs = 9.765625e-4f;             // 2^-10 high-word units

// Per-ray constants of the Jacobian walk: the slot relabelling (slot 2 is the
// axis with most crossings), each slot's signed stride and FP32 plane spacing,
// and the chunk length.  jac_prepare also stores each slot's exact sequence
// (first crossing, spacing, count) in the lane's shared-memory scratch.
struct JacRay {
  int dom, a0, a1;
  int step[3];
  float dl[3];
  int chunk;
};

// State of the Jacobian walk at a chunk boundary.
struct JacState {
  unsigned int k0, k1, k2;  // crossings taken per slot
  unsigned long long O;     // exact position of the last crossing taken (the anchor)
  int off;                  // voxel after it (padded offset)
  float v, vprev;           // voxel after and before it
  bool p0, p1;              // its slot (neither: slot 2 or a clamped entry), whose weight is not yet summed
};

// One chunk's contribution: the segment sum f (its last segment ending at the
// exact anchor of the next chunk) and the two slots' weight sums in local
// positions, with the chunk's anchor as FP32 (Of).
struct JacChunk {
  float f, g0, g1, h0, h1, Of;
};

__device__ __forceinline__ void jac_prepare(const RaySetup& r, JacScratch* ws, JacRay& jr) {
  const int t = threadIdx.x;
  int dom = 0;
  if (r.cnt[1] > r.cnt[dom]) dom = 1;
  if (r.cnt[2] > r.cnt[dom]) dom = 2;
  jr.dom = dom;
  jr.a0 = dom == 0 ? 1 : 0;  // real axis of slot 0
  jr.a1 = dom == 2 ? 1 : 2;  // real axis of slot 1
  const int ax_of[3] = {jr.a0, jr.a1, dom};
#pragma unroll
  for (int sl = 0; sl < 3; ++sl) {
    const int a = ax_of[sl];
    const unsigned long long D = pick3(a, r.D[0], r.D[1], r.D[2]);
    ws->A0[sl][t] = pick3(a, r.A0[0], r.A0[1], r.A0[2]);
    ws->D[sl][t] = D;
    jr.step[sl] = pick3(a, r.step[0], r.step[1], r.step[2]);
    ws->cnt[sl][t] = pick3(a, r.cnt[0], r.cnt[1], r.cnt[2]);
    jr.dl[sl] = fix_to_float(static_cast<long long>(D));
  }
  jr.chunk = walk_chunk(r.nseg);
}

// The state before the first crossing: the entry voxel, the entry crossing pending.
template <int DT>
__device__ __forceinline__ void jac_start(const VolumeDev& vd, const RaySetup& r, const JacRay& jr, JacState& s) {
  s.k0 = s.k1 = s.k2 = 0u;
  s.O = 0ull;
  s.off = r.off;
  s.v = gather<DT>(vd, s.off);
  s.vprev = 0.f;
  s.p0 = r.ea == jr.a0;
  s.p1 = r.ea == jr.a1;
}

// One chunk of n crossings from state s (more: crossings follow the chunk).
template <int DT>
__device__ __forceinline__ void jac_chunk(const VolumeDev& vd, const JacRay& jr, JacScratch* ws, JacState& s, int n,
                                          bool more, JacChunk& out) {
  const int t = threadIdx.x;
  const int* step = jr.step;
  const float* dl = jr.dl;
  unsigned long long O = s.O;
  int off = s.off;
  float v = s.v, vprev = s.vprev;
  bool p0 = s.p0, p1 = s.p1;
  ws->c_off[t] = off;
  ws->c_v[t] = v;
  ws->c_vprev[t] = vprev;
  ws->c_pend[t] = p0 ? 0 : (p1 ? 1 : 2);
  const float x0 = local_pos(fix_at(ws->A0[0][t], ws->D[0][t], s.k0), O);
  const float y0 = local_pos(fix_at(ws->A0[1][t], ws->D[1][t], s.k1), O);
  const float z0 = local_pos(fix_at(ws->A0[2][t], ws->D[2][t], s.k2), O);
  float tx = x0, ty = y0, tz = z0;
  float lx = 0.f, ly = 0.f, lz = 0.f;
  // chunk sums in local positions
  float ac = 0.f, f = 0.f, g0 = 0.f, g1 = 0.f, h0 = 0.f, h1 = 0.f;
#define DRR_JAC_STEP(an, bx, by)                           \
  const float an = fminf(fminf(tx, ty), tz);               \
  const bool bx = tx == an;                                \
  const bool by = !bx && ty == an;                         \
  {                                                        \
    const bool bz = !bx && !by;                            \
    off += bx ? step[0] : (by ? step[1] : step[2]);        \
    if (bx) lx += 1.f;                                     \
    if (by) ly += 1.f;                                     \
    if (bz) lz += 1.f;                                     \
    next_xy(tx, ty, lx, ly, dl[0], dl[1], x0, y0);         \
    tz = fmaf(lz, dl[2], z0);                              \
  }
#define DRR_JAC_ACCOUNT()                                  \
  {                                                        \
    const float wgt = vprev - v;                           \
    if (p0) { g0 += wgt; h0 = fmaf(wgt, ac, h0); }         \
    if (p1) { g1 += wgt; h1 = fmaf(wgt, ac, h1); }         \
  }
  // The gathers run two crossings ahead: crossing m+1 (an1, q0/q1, voxel v1
  // after it) is taken while segment m is summed, and a crossing's weight is
  // taken once the voxel after it has had one walk step to arrive.  First the
  // pending crossing at the anchor.
  DRR_JAC_ACCOUNT()
  DRR_JAC_STEP(a1st, b1x, b1y)
  float an1 = a1st;
  bool q0 = b1x, q1 = b1y;
  float v1 = gather<DT>(vd, off);
  float gmin = 3.0e38f;
#pragma unroll kJacUnroll
  for (int m = 1; m < n; ++m) {
    DRR_JAC_STEP(an2, bx, by)
    const float v2 = gather<DT>(vd, off);
    const float seg = an1 - ac;
    gmin = fminf(gmin, seg);
    f = fmaf(seg, v, f);
    {  // crossing m, at the end of the segment just summed
      const float wgt = v - v1;
      if (q0) { g0 += wgt; h0 = fmaf(wgt, an1, h0); }
      if (q1) { g1 += wgt; h1 = fmaf(wgt, an1, h1); }
    }
    ac = an1;
    q0 = bx;
    q1 = by;
    v = v1;
    v1 = v2;
    an1 = an2;
  }
  // drain: the segment that ends at the chunk's last crossing, which stays pending
  {
    const float seg = an1 - ac;
    gmin = fminf(gmin, seg);
    f = fmaf(seg, v, f);
  }
  ac = an1;
  p0 = q0;
  p1 = q1;
  vprev = v;
  v = v1;
  unsigned int c0 = static_cast<unsigned int>(lx), c1 = static_cast<unsigned int>(ly),
               c2 = static_cast<unsigned int>(lz);
  // The float order is exact unless two crossings came within the FP32 error
  // of the local positions: check the chunk's shortest segment and the gap to
  // the next crossing after it.
  const float next = fminf(fminf(tx, ty), tz);
  if (gmin < fmaf(ac, kTieRel, kTieAbs) || (more && next - ac < fmaf(next, kTieRel, kTieAbs))) {
    // exact re-walk of the chunk: the next crossing of each slot held as 64-bit
    // fixed point (all ones once the slot's crossings are used up), the
    // smallest taken each step (ties to the lower slot)
    off = ws->c_off[t];
    v = ws->c_v[t];
    vprev = ws->c_vprev[t];
    const int pend = ws->c_pend[t];
    p0 = pend == 0;
    p1 = pend == 1;
    ac = f = g0 = g1 = h0 = h1 = 0.f;
    c0 = c1 = c2 = 0u;
    int r0 = ws->cnt[0][t] - static_cast<int>(s.k0), r1 = ws->cnt[1][t] - static_cast<int>(s.k1),
        r2 = ws->cnt[2][t] - static_cast<int>(s.k2);
    unsigned long long e0 = r0 > 0 ? fix_at(ws->A0[0][t], ws->D[0][t], s.k0) : ~0ull;
    unsigned long long e1 = r1 > 0 ? fix_at(ws->A0[1][t], ws->D[1][t], s.k1) : ~0ull;
    unsigned long long e2 = r2 > 0 ? fix_at(ws->A0[2][t], ws->D[2][t], s.k2) : ~0ull;
    for (int m = 0; m < n; ++m) {
      DRR_JAC_ACCOUNT()
      const bool sx = e0 <= e1 && e0 <= e2;
      const bool sy = !sx && e1 <= e2;
      unsigned long long best;
      if (sx) {
        best = e0;
        off += step[0];
        ++c0;
        e0 = --r0 > 0 ? e0 + ws->D[0][t] : ~0ull;
      } else if (sy) {
        best = e1;
        off += step[1];
        ++c1;
        e1 = --r1 > 0 ? e1 + ws->D[1][t] : ~0ull;
      } else {
        best = e2;
        off += step[2];
        ++c2;
        e2 = --r2 > 0 ? e2 + ws->D[2][t] : ~0ull;
      }
      const float an = local_pos(best, O);
      const float vn = gather<DT>(vd, off);
      f = fmaf(an - ac, v, f);
      ac = an;
      p0 = sx;
      p1 = sy;
      vprev = v;
      v = vn;
    }
  }
#undef DRR_JAC_STEP
#undef DRR_JAC_ACCOUNT
  s.k0 += c0;
  s.k1 += c1;
  s.k2 += c2;
  // the chunk's last crossing (the largest one taken) is the next anchor; the
  // segment that ends there gets its exact end
  unsigned long long Onew = O;
  if (s.k0) Onew = max(Onew, fix_at(ws->A0[0][t], ws->D[0][t], s.k0 - 1u));
  if (s.k1) Onew = max(Onew, fix_at(ws->A0[1][t], ws->D[1][t], s.k1 - 1u));
  if (s.k2) Onew = max(Onew, fix_at(ws->A0[2][t], ws->D[2][t], s.k2 - 1u));
  out.f = fmaf(local_pos(Onew, O) - ac, vprev, f);
  out.g0 = g0;
  out.g1 = g1;
  out.h0 = h0;
  out.h1 = h1;
  out.Of = fix_to_float(static_cast<long long>(O));
  s.O = Onew;
  s.off = off;
  s.v = v;
  s.vprev = vprev;
  s.p0 = p0;
  s.p1 = p1;
}

// Running sums of the Jacobian walk over its chunks, in chunk order (chunk sums
// to absolute positions: alpha = O + local).
struct JacTotals {
  float F, G0, G1, A0, A1;
};

__device__ __forceinline__ void jac_add_chunk(JacTotals& T, const JacChunk& c) {
  T.F += c.f;
  T.G0 += c.g0;
  T.A0 += fmaf(c.Of, c.g0, c.h0);
  T.G1 += c.g1;
  T.A1 += fmaf(c.Of, c.g1, c.h1);
}

// After the last chunk: the last segment to the exit, the last crossing's
// weight at its absolute position, the exit crossing, and the sums moved back
// to alpha units and real axes.  Gc: the clamped entry's weight.
__device__ __forceinline__ void jac_finish(const RaySetup& r, const JacRay& jr, const JacState& s, JacTotals T,
                                           float Gc, JacSums& out) {
  float F = fmaf(local_pos(static_cast<unsigned long long>(kExitUnits) << 32, s.O), s.v, T.F);
  float G0 = T.G0, G1 = T.G1, A0 = T.A0, A1 = T.A1;
  {
    const float last = fix_to_float(static_cast<long long>(s.O));
    const float wgt = s.vprev - s.v;
    if (s.p0) { G0 += wgt; A0 = fmaf(wgt, last, A0); }
    if (s.p1) { G1 += wgt; A1 = fmaf(wgt, last, A1); }
  }
  // exit crossing: weight V_last - 0 at the exit
  const float v = s.v;
  const float ex = static_cast<float>(kExitUnits);
  float Ac = 0.f;
  if (r.xa < 0) { Gc += v; Ac = v * ex; }
  else if (r.xa == jr.a0) { G0 += v; A0 = fmaf(v, ex, A0); }
  else if (r.xa == jr.a1) { G1 += v; A1 = fmaf(v, ex, A1); }
  // back to alpha units and real axes (static indices)
  const float u = r.unit;
  out.F = F * u;
  out.dom = jr.dom;
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    out.G[a] = a == jr.a0 ? G0 : (a == jr.a1 ? G1 : -(G0 + G1 + Gc));  // sum of all crossing weights is 0
    out.A[a] = a == jr.a0 ? A0 * u : (a == jr.a1 ? A1 * u : 0.f);      // the dominant axis is handled through R
  }
  out.Gc = Gc;
  out.Ac = Ac * u;
}

template <int DT>
__device__ __forceinline__ void walk_jacobian(const VolumeDev& vd, const RaySetup& r, JacScratch* ws,
                                              JacSums& out) {
  JacRay jr;
  jac_prepare(r, ws, jr);
  JacState s;
  jac_start<DT>(vd, r, jr, s);
  const float Gc = r.ea < 0 ? -s.v : 0.f;  // entry clamped at alpha 0: weight -V_first
  JacTotals T{0.f, 0.f, 0.f, 0.f, 0.f};
  int remaining = r.nseg - 1;
  while (remaining > 0) {
    const int n = min(remaining, jr.chunk);
    JacChunk c;
    jac_chunk<DT>(vd, jr, ws, s, n, remaining > n, c);
    remaining -= n;
    jac_add_chunk(T, c);
  }
  jac_finish(r, jr, s, T, Gc, out);
}

// dE/d eta for one ray from the crossing sums (Sec. 2.4 with the voxel lookup
// held fixed).  With d = p - s, L = |d|, absolute alphas A_abs = A + amin G:
//   dE/dt_a = dE/ds_a + dE/dp_a = -L G_a / d_a
//   dE/dp_a = d_a F / L - L A_abs_a / d_a
// and for the dominant axis the second line is rearranged with
// A_abs = F - R (R = the other axes' and the clamped points' A_abs) into
//   dE/dp_a = (L R - F (L^2 - d_a^2) / L) / d_a,
// which has no cancellation for rays nearly along that axis.
//   dE/d eta_j = dE/dt . (dR_j s_c) + dE/dp . (dR_j (p_c - s_c)).
// gt = dE/dt, gp = dE/dp in world units.
__device__ __forceinline__ void ray_world_grads(const RaySetup& r, const JacSums& s, float gt[3], float q[3]) {
  const float L2 = fmaf(r.d[2], r.d[2], fmaf(r.d[1], r.d[1], r.d[0] * r.d[0]));
  const float L = sqrtf(L2);
  const float F = s.F;
  float R = s.Ac;  // position sums relative to the entry
#pragma unroll
  for (int a = 0; a < 3; ++a)
    if (a != s.dom) R += s.A[a];
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    if (r.d[a] != 0.f) {
      const float Ld = L / r.d[a];
      gt[a] = -s.G[a] * Ld;
      if (a == s.dom) {
        float D = 0.f;
#pragma unroll
        for (int b = 0; b < 3; ++b)
          if (b != a) D = fmaf(r.d[b], r.d[b], D);
        q[a] = (L * R - F * D / L) / r.d[a];
      } else {
        q[a] = r.d[a] * F / L - s.A[a] * Ld;
      }
    } else {
      gt[a] = 0.f;
      q[a] = 0.f;
    }
  }
}

__device__ __forceinline__ void pose_jacobian(const RaySetup& r, const JacSums& s, const PoseGeom& pg,
                                              const float e[3], int h, int w, float scale, float J[6]) {
  float gt[3], q[3];
  ray_world_grads(r, s, gt, q);
  // an angle moves the entry point e by omega_j x (e - t): its term is
  // gt . (omega_j x (e - t)) = omega_j . ((e - t) x gt)
  const float x0 = e[0] - pg.t[0], x1 = e[1] - pg.t[1], x2 = e[2] - pg.t[2];
  const float c0 = fmaf(x1, gt[2], -x2 * gt[1]), c1 = fmaf(x2, gt[0], -x0 * gt[2]), c2 = fmaf(x0, gt[1], -x1 * gt[0]);
  const float fw = static_cast<float>(w), fh = static_cast<float>(h);
#pragma unroll
  for (int j = 0; j < 3; ++j) {
    float acc = fmaf(pg.Om[j][0], c0, fmaf(pg.Om[j][1], c1, pg.Om[j][2] * c2));
#pragma unroll
    for (int a = 0; a < 3; ++a) acc = fmaf(q[a], fmaf(fh, pg.Hv[j][a], fmaf(fw, pg.Wv[j][a], pg.Q[j][a])), acc);
    J[j] = acc * scale;
  }
#pragma unroll
  for (int a = 0; a < 3; ++a) J[3 + a] = gt[a] * scale;
}

// dE/d(sdr, dh, dw) for one ray: the detector parameters (the paper notes the
// generator also differentiates with respect to the source-to-detector
// distance 2 rho and the pixel spacing, Sec. 3.2).  With s = R (rho,0,0) + t,
// rho = sdr / 2, p = R (-rho, (w - wc) dw, (h - hc) dh) + t and dE/ds = gt - gp:
//   dE/dsdr = (dE/ds - dE/dp) . R e_x / 2,
//   dE/ddh  = (h - hc) dE/dp . R e_z,   dE/ddw = (w - wc) dE/dp . R e_y.
__device__ __forceinline__ void geometry_jacobian(const RaySetup& r, const JacSums& s, const PoseGeom& pg, int h,
                                                  int w, float scale, float J[3]) {
  float gt[3], q[3];
  ray_world_grads(r, s, gt, q);
  // dE/dp = q + amin gt; dE/ds - dE/dp = gt - 2 dE/dp = (1 - 2 amin) gt - 2 q
  const float am = static_cast<float>(r.amin), c = static_cast<float>(1.0 - 2.0 * r.amin);
  float a0 = 0.f, a1 = 0.f, a2 = 0.f;
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    const float gp = fmaf(am, gt[a], q[a]);
    a0 = fmaf(fmaf(c, gt[a], -2.f * q[a]), pg.Rc[0][a], a0);
    a1 = fmaf(gp, pg.Rc[2][a], a1);
    a2 = fmaf(gp, pg.Rc[1][a], a2);
  }
  J[0] = 0.5f * a0 * scale;
  J[1] = (static_cast<float>(h) - pg.hc) * a1 * scale;
  J[2] = (static_cast<float>(w) - pg.wc) * a2 * scale;
}

// Back-projection adds of one warp step, merged down each column of the warp's
// TW x (32 / TW) pixel tile: the lanes of one column (pixels h, h+1, ... at the
// same w) whose rays are in the same voxel at this step add once, through the
// first lane of each run of equal addresses, the run's sum found by a segmented
// suffix scan over the column.  The L2 serves every lane's atomic as its own
// sector operation, so each lane merged away is one L2 operation less; rays a
// pixel apart along h often share a voxel (2.5 mm CT slices against 0.7 mm
// pixels at the isocentre).  Addresses at or beyond nvox add nothing.
#ifndef DRR_BP_MERGE_ROWS
#define DRR_BP_MERGE_ROWS 8  // runs are merged within aligned groups of this many rows (a power of two)
#endif
template <int TW>
__device__ __forceinline__ void red_column_merged(float* __restrict__ gvol, unsigned int addr, float v,
                                                  unsigned int nvox, int lane) {
  constexpr unsigned int kAll = 0xffffffffu;
  constexpr int TH = 32 / TW;
  constexpr int kRows = DRR_BP_MERGE_ROWS < TH ? DRR_BP_MERGE_ROWS : TH;
  const int hrow = lane / TW;
  const unsigned int a_dn = __shfl_down_sync(kAll, addr, TW);
  bool lk = (hrow + 1) % kRows != 0 && a_dn == addr;  // the pixel below adds to the same voxel
  const unsigned int first = __ballot_sync(kAll, lk);
  unsigned int lkm = first;
  float s = v;
#pragma unroll
  for (int d = 1; d < kRows; d *= 2) {
    // s: the run's sum over rows hrow .. hrow + d - 1; lk: the run goes on past them
    const float s_dn = __shfl_down_sync(kAll, s, d * TW);
    if (lk) s += s_dn;
    if (2 * d < kRows) {
      lk = lk && ((lkm >> ((lane + d * TW) & 31)) & 1u);
      lkm = __ballot_sync(kAll, lk);
    }
  }
  // the first row of each run within its group adds
  const bool head = hrow % kRows == 0 || !((first >> ((lane - TW) & 31)) & 1u);
  if (head && addr < nvox) atomicAdd(gvol + addr, s);
}

// Back-projection walk: grad_V[voxel] += g L (a_{m+1} - a_m), the transpose of
// the forward map V -> E (Eq. 2 is linear in V), into an unpadded (nz, ny, nx)
// FP32 volume.  The crossings are those of the forward walk: FP32 positions
// local to an exact fixed-point anchor, re-anchored every kBpChunk steps.  All
// 32 lanes step together (to the warp's longest ray) and re-anchor at the same
// steps, since their adds are merged across lanes; a lane whose pixel has no
// ray to walk passes nseg = 0 and adds nothing.
constexpr int kBpChunk = 64;
__device__ __forceinline__ void walk_backproject(const VolumeDev& vd, const RaySetup& r, int nseg, float gL,
                                                 float* __restrict__ gvol, WalkScratch* ws, int lane) {
  const int t = threadIdx.x;
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    ws->A0[a][t] = r.A0[a];
    ws->D[a][t] = r.D[a];
  }
  const float dx = fix_to_float(static_cast<long long>(r.D[0])), dy = fix_to_float(static_cast<long long>(r.D[1])),
              dz = fix_to_float(static_cast<long long>(r.D[2]));
  // unsigned index arithmetic: a lane past its exit keeps stepping (wrapping) without adding
  const unsigned int nx = static_cast<unsigned int>(vd.n[0]), nxy = nx * static_cast<unsigned int>(vd.n[1]);
  const unsigned int sx = r.step[0] > 0 ? 1u : 0u - 1u;
  const unsigned int sy = r.step[1] > 0 ? nx : 0u - nx;
  const unsigned int sz = r.step[2] > 0 ? nxy : 0u - nxy;
  const unsigned int nvox = static_cast<unsigned int>(vd.n[0] * vd.n[1] * vd.n[2]);
  unsigned int lin = static_cast<unsigned int>(r.ient[0] + vd.n[0] * (r.ient[1] + vd.n[1] * r.ient[2]));
  const float s = gL * r.unit;  // gradient per high-word unit of segment length
  const int nmax = __reduce_max_sync(0xffffffffu, nseg);
  unsigned int kx = 0u, ky = 0u, kz = 0u;
  unsigned long long O = 0ull;  // exact position of the last crossing taken (the anchor)
  float ac = 0.f;               // local position where the current segment starts
  for (int m = 0; m < nmax;) {  // warp-uniform
    const int n = min(nmax - m, kBpChunk);
    const float x0 = local_pos(fix_at(ws->A0[0][t], ws->D[0][t], kx), O);
    const float y0 = local_pos(fix_at(ws->A0[1][t], ws->D[1][t], ky), O);
    const float z0 = local_pos(fix_at(ws->A0[2][t], ws->D[2][t], kz), O);
    const float xe = local_pos(static_cast<unsigned long long>(kExitUnits) << 32, O);
    float tx = x0, ty = y0, tz = z0;
    float cx = 0.f, cy = 0.f, cz = 0.f;
#pragma unroll 4
    for (int j = 1; j <= n; ++j) {
      const int step = m + j;  // this step ends segment step - 1 (the exit segment at step nseg)
      const float an = fminf(fminf(tx, ty), tz);
      const float val = s * ((step < nseg ? an : xe) - ac);
#if DRR_CHECK_BOUNDS
      if (step <= nseg && lin >= nvox) atomicOr(&g_fault_word, kFaultBackproject);
#endif
      red_column_merged<kBpTileW>(gvol, step <= nseg ? lin : 0xffffffffu, val, nvox, lane);
      ac = an;
      const bool bx = tx == an;
      const bool by = !bx && ty == an;
      const bool bz = !bx && !by;
      lin += bx ? sx : (by ? sy : sz);
      if (bx) cx += 1.f;
      if (by) cy += 1.f;
      if (bz) cz += 1.f;
      next_xy(tx, ty, cx, cy, dx, dy, x0, y0);
      tz = fmaf(cz, dz, z0);
    }
    m += n;
    kx += static_cast<unsigned int>(cx);
    ky += static_cast<unsigned int>(cy);
    kz += static_cast<unsigned int>(cz);
    // re-anchor at the last crossing taken: the current segment starts there
    unsigned long long Onew = O;
    if (kx) Onew = max(Onew, fix_at(ws->A0[0][t], ws->D[0][t], kx - 1u));
    if (ky) Onew = max(Onew, fix_at(ws->A0[1][t], ws->D[1][t], ky - 1u));
    if (kz) Onew = max(Onew, fix_at(ws->A0[2][t], ws->D[2][t], kz - 1u));
    ac = 0.f;
    O = Onew;
  }
}

// One warp's back-projection of its tile: every lane takes part in the walk,
// with nseg = 0 where its pixel is outside the detector, its upstream gradient
// is zero, the ray misses the volume or the geometry is not finite.
__device__ __forceinline__ void backproject_tile_ray(const VolumeDev& vd, const PoseGeom& pg, int h, int w, bool active,
                                                     float g, float* __restrict__ gvol, WalkScratch* ws, int lane) {
  RaySetup r{};
  int nseg = 0;
  float gL = 0.f;
  if (active && ray_setup<false>(vd, pg, h, w, r) > 0) {
    nseg = r.nseg;
    gL = g * sqrtf(fmaf(r.d[2], r.d[2], fmaf(r.d[1], r.d[1], r.d[0] * r.d[0])));
  }
  walk_backproject(vd, r, nseg, gL, gvol, ws, lane);
}

template <int MODE>
struct ScratchFor {
  using type = WalkScratch;
};
template <>
struct ScratchFor<kFwdJac> {
  using type = JacScratch;
};
template <>
struct ScratchFor<kPoseGrad> {
  using type = JacScratch;
};
template <>
struct ScratchFor<kGeoGrad> {
  using type = JacScratch;
};

template <int MODE, int DT>
__device__ __forceinline__ void trace_ray(const VolumeDev& vd, const PoseGeom& pg, int h, int w, float gscale,
                                          float* __restrict__ gvol, WalkScratch* ws, RayResult& res) {
  res.F = 0.f;
  res.nseg = 0;
#pragma unroll
  for (int k = 0; k < 6; ++k) res.J[k] = 0.f;
  constexpr bool kJac = MODE == kFwdJac || MODE == kPoseGrad || MODE == kGeoGrad;
  RaySetup r;
  float e[3];
  const int rs = ray_setup<kJac>(vd, pg, h, w, r, e);
  if (kJac && rs > 0) {  // parked in shared memory until the epilogue
    JacScratch* js = static_cast<JacScratch*>(ws);
#pragma unroll
    for (int a = 0; a < 3; ++a) js->e[a][threadIdx.x] = e[a];
  }
  if (rs < 0) {  // non-finite geometry (e.g. a NaN pose): NaN out, no walk
    res.F = __int_as_float(0x7fffffff);
#pragma unroll
    for (int k = 0; k < 6; ++k) res.J[k] = res.F;
    return;
  }
  if (rs == 0) return;
  res.nseg = r.nseg;
  if (MODE == kCount) return;
  const float L = sqrtf(fmaf(r.d[2], r.d[2], fmaf(r.d[1], r.d[1], r.d[0] * r.d[0])));
  if (MODE == kFwd) {
    res.F = walk_forward<DT>(vd, r, ws) * L * vd.out_scale;
  } else if (MODE == kFwdJac || MODE == kPoseGrad || MODE == kGeoGrad) {
    JacSums s;
    walk_jacobian<DT>(vd, r, static_cast<JacScratch*>(ws), s);
    res.F = s.F * L * vd.out_scale;
    if (MODE == kGeoGrad) {
      geometry_jacobian(r, s, pg, h, w, vd.out_scale, res.J);
      res.J[3] = res.J[4] = res.J[5] = 0.f;
    } else {
      const JacScratch* js = static_cast<const JacScratch*>(ws);
      const float ep[3] = {js->e[0][threadIdx.x], js->e[1][threadIdx.x], js->e[2][threadIdx.x]};
      pose_jacobian(r, s, pg, ep, h, w, vd.out_scale, res.J);
    }
  }
}

// Persistent walk kernel: each warp claims 8x4-pixel tiles (pose-major order)
// from a per-launch counter until the batch runs out, so no warp slot idles
// while a slower warp of its block finishes, and the grid is exactly what the
// GPU holds at once.  A warp copies its pose's geometry to its own shared slot
// when the pose changes.  Pose-gradient mode writes one partial sum of g . J
// per tile, so the result does not depend on which warp took which tile.
template <int MODE, int DT>
__global__ void __launch_bounds__(kThreads, (MODE == kFwdJac || MODE == kPoseGrad || MODE == kGeoGrad) ? DRR_JAC_MINB
                                                                                                : DRR_FWD_MINB)
    siddon_kernel(VolumeDev vd, DetDev det, const PoseGeom* __restrict__ pgs, int B, unsigned int* __restrict__ counter,
                  float* __restrict__ out, float* __restrict__ jac, const float* __restrict__ gin,
                  float* __restrict__ partials, float* __restrict__ gvol) {
  __shared__ PoseGeom spg[kThreads / 32];
  __shared__ typename ScratchFor<MODE>::type ws;
  grid_dep_wait();
  grid_dep_release();
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  constexpr bool kBp = MODE == kBackproject;
  constexpr int TW = kBp ? kBpTileW : kWarpTileW, TH = 32 / TW;
  const int twx = (det.W + TW - 1) / TW;
  const int per_pose = twx * ((det.H + TH - 1) / TH);
  const unsigned int total = static_cast<unsigned int>(per_pose) * static_cast<unsigned int>(B);
  const size_t npix = static_cast<size_t>(det.H) * det.W;
  PoseGeom& pg = spg[warp];
  int cur = -1;
  for (;;) {
    unsigned int tile = 0u;
    if (lane == 0) tile = atomicAdd(counter, 1u);
    tile = __shfl_sync(0xffffffffu, tile, 0);  // also: every lane is done with the previous tile
    if (tile >= total) break;
    const int b = static_cast<int>(tile / static_cast<unsigned int>(per_pose));
    const int tin = static_cast<int>(tile) - b * per_pose;
    if (b != cur) {
      const unsigned int* src = reinterpret_cast<const unsigned int*>(pgs + b);
      unsigned int* dst = reinterpret_cast<unsigned int*>(&pg);
      for (int i = lane; i < static_cast<int>(sizeof(PoseGeom) / 4); i += 32) dst[i] = src[i];
      __syncwarp();
      cur = b;
    }
    const int ty = tin / twx, tx = tin - ty * twx;
    const int h = ty * TH + lane / TW, w = tx * TW + lane % TW;
    const bool valid = (w < det.W) && (h < det.H);
    const size_t pix = static_cast<size_t>(h) * det.W + w;
    RayResult r;
    r.nseg = 0;
    float gsc = 0.f;
    if (valid && (MODE == kPoseGrad || MODE == kGeoGrad || kBp)) gsc = gin[b * npix + pix];
    if (kBp) {
      backproject_tile_ray(vd, pg, h, w, valid && gsc != 0.f, gsc, gvol, &ws, lane);
      continue;
    }
    if (valid) {
      trace_ray<MODE, DT>(vd, pg, h, w, gsc, gvol, &ws, r);
    } else {
      r.F = 0.f;
#pragma unroll
      for (int k = 0; k < 6; ++k) r.J[k] = 0.f;
    }
    if (MODE == kCount) {
      if (valid) reinterpret_cast<int*>(out)[b * npix + pix] = r.nseg;
    } else if (MODE == kFwd || MODE == kFwdJac) {
      if (valid) {
        out[b * npix + pix] = r.F;
        if (MODE == kFwdJac) {
#pragma unroll
          for (int k = 0; k < 6; ++k) jac[(static_cast<size_t>(b) * 6 + k) * npix + pix] = r.J[k];
        }
      }
    } else if (MODE == kPoseGrad || MODE == kGeoGrad) {
      constexpr int nc = MODE == kPoseGrad ? 6 : 3;  // pose or detector parameters
      float c[nc];
#pragma unroll
      for (int k = 0; k < nc; ++k) {
        c[k] = gsc * r.J[k];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) c[k] += __shfl_xor_sync(0xffffffffu, c[k], o);
      }
      if (lane == 0) {
#pragma unroll
        for (int k = 0; k < nc; ++k) partials[(static_cast<size_t>(b) * per_pose + tin) * nc + k] = c[k];
      }
    }
  }
}

// ---------------------------------------------------------------------------
// Split walk for launches too small to fill the GPU (the fused forward +
// pose-Jacobian mode): each ray is walked by K lanes, lane j taking the j-th
// of K runs of whole chunks.  A lane rebuilds the exact walk state at its first
// chunk boundary, walks its chunks with the same code as the whole-ray walk and
// parks each chunk's sums in shared memory; the ray's first lane then adds all
// chunk sums in chunk order and finishes the ray.  Every arithmetic step is the
// whole-ray walk's, in the same order, so the results are the same bits.
// ---------------------------------------------------------------------------
constexpr int kSplitMaxChunks = 32;  // rays with more chunks are not split (longer than ~1950 segments)

// Exact walk state after c crossings in the walk's order (by exact position,
// ties to the lower slot, which is the order every chunk of the whole-ray walk
// takes: its tie test sends any chunk whose FP32 order could differ to the
// exact re-walk).  The crossings of each slot before a position X are counted
// from the arithmetic sequence (Eq. 3) by one 64-bit division, X is pulled back
// until at most c crossings precede it, and the rest are taken exactly.
template <int DT>
__device__ __forceinline__ void jac_state_at(const VolumeDev& vd, const RaySetup& r, const JacRay& jr,
                                             const JacScratch* ws, int c, JacState& s) {
  const int t = threadIdx.x;
  unsigned long long A[3], D[3];
  unsigned int cnt[3];
#pragma unroll
  for (int sl = 0; sl < 3; ++sl) {
    A[sl] = ws->A0[sl][t];
    D[sl] = ws->D[sl][t];
    cnt[sl] = static_cast<unsigned int>(max(ws->cnt[sl][t], 0));
  }
  unsigned int n[3] = {0u, 0u, 0u};
  const unsigned int total = static_cast<unsigned int>(r.nseg - 1);
  unsigned long long X = static_cast<unsigned long long>(static_cast<double>(c) / total * 0.98 * kFixScale);
  for (int it = 0; it < 16; ++it) {
    unsigned int sum = 0u;
#pragma unroll
    for (int sl = 0; sl < 3; ++sl) {
      n[sl] = (cnt[sl] == 0u || X <= A[sl]) ? 0u
                                            : static_cast<unsigned int>(min((X - A[sl] - 1ull) / D[sl] + 1ull,
                                                                            static_cast<unsigned long long>(cnt[sl])));
      sum += n[sl];
    }
    if (sum <= static_cast<unsigned int>(c)) break;
    X = it < 14 ? X / (sum + 1u) * static_cast<unsigned int>(c) : 0ull;  // the last pass counts from the entry
  }
  unsigned long long e[3];
#pragma unroll
  for (int sl = 0; sl < 3; ++sl) e[sl] = n[sl] < cnt[sl] ? fix_at(A[sl], D[sl], n[sl]) : ~0ull;
  for (unsigned int m = n[0] + n[1] + n[2]; m < static_cast<unsigned int>(c); ++m) {
    const bool sx = e[0] <= e[1] && e[0] <= e[2];
    const bool sy = !sx && e[1] <= e[2];
    if (sx) { ++n[0]; e[0] = n[0] < cnt[0] ? e[0] + D[0] : ~0ull; }
    else if (sy) { ++n[1]; e[1] = n[1] < cnt[1] ? e[1] + D[1] : ~0ull; }
    else { ++n[2]; e[2] = n[2] < cnt[2] ? e[2] + D[2] : ~0ull; }
  }
  // the last crossing taken: the largest position (ties: the higher slot, taken later)
  unsigned long long O = 0ull;
  int last = -1;
#pragma unroll
  for (int sl = 0; sl < 3; ++sl) {
    if (n[sl] > 0u) {
      const unsigned long long q = fix_at(A[sl], D[sl], n[sl] - 1u);
      if (last < 0 || q >= O) { O = q; last = sl; }
    }
  }
  s.k0 = n[0];
  s.k1 = n[1];
  s.k2 = n[2];
  s.O = O;
  s.off = r.off + static_cast<int>(n[0]) * jr.step[0] + static_cast<int>(n[1]) * jr.step[1] +
          static_cast<int>(n[2]) * jr.step[2];
  s.v = gather<DT>(vd, s.off);
  s.vprev = gather<DT>(vd, s.off - pick3(last, jr.step[0], jr.step[1], jr.step[2]));
  s.p0 = last == 0;
  s.p1 = last == 1;
}

// Persistent split kernel (mode kFwdJac): a block of K warps claims one warp
// tile (8x4 pixels, pose-major) at a time; warp j walks the j-th run of chunks
// of all 32 rays (so a warp's lanes are neighbouring rays, as in the whole-ray
// kernel, and share cache lines); then the first warp adds each ray's chunk
// sums in chunk order and finishes the rays.
template <int DT, int K>
__global__ void __launch_bounds__(32 * K) siddon_split_kernel(VolumeDev vd, DetDev det, const PoseGeom* __restrict__ pgs,
                                                              int B, unsigned int* __restrict__ counter,
                                                              float* __restrict__ out, float* __restrict__ jac) {
  __shared__ PoseGeom pg;
  __shared__ JacScratch ws;  // indexed by threadIdx.x (< 32 K)
  __shared__ JacState fin[32];
  __shared__ float gcs[32];
  __shared__ unsigned int tile_s;
  extern __shared__ JacChunk split_chunks[];  // [kSplitMaxChunks][32]: chunk k of ray i at k * 32 + i
  grid_dep_wait();
  grid_dep_release();
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, piece = warp;
  const int twx = (det.W + kWarpTileW - 1) / kWarpTileW;
  const int per_pose = twx * ((det.H + kWarpTileH - 1) / kWarpTileH);
  const unsigned int total = static_cast<unsigned int>(per_pose) * static_cast<unsigned int>(B);
  const size_t npix = static_cast<size_t>(det.H) * det.W;
  int cur = -1;
  for (;;) {
    if (threadIdx.x == 0) tile_s = atomicAdd(counter, 1u);
    __syncthreads();  // also: the block is done with the previous tile
    const unsigned int tile = tile_s;
    if (tile >= total) break;
    const int b = static_cast<int>(tile / static_cast<unsigned int>(per_pose));
    const int tin = static_cast<int>(tile) - b * per_pose;
    if (b != cur) {
      const unsigned int* src = reinterpret_cast<const unsigned int*>(pgs + b);
      unsigned int* dst = reinterpret_cast<unsigned int*>(&pg);
      for (int i = threadIdx.x; i < static_cast<int>(sizeof(PoseGeom) / 4); i += 32 * K) dst[i] = src[i];
      cur = b;
    }
    __syncthreads();
    const int ty = tin / twx, tx = tin - ty * twx;
    const int h = ty * kWarpTileH + lane / kWarpTileW, w = tx * kWarpTileW + lane % kWarpTileW;
    const bool valid = (w < det.W) && (h < det.H);
    RaySetup r;
    float e[3];
    const int rs = valid ? ray_setup<true>(vd, pg, h, w, r, e) : 0;
    JacRay jr;
    JacState s{};
    int nch = 0;
    if (rs > 0) {
      jac_prepare(r, &ws, jr);
      const int ncross = r.nseg - 1;
      nch = (ncross + jr.chunk - 1) / jr.chunk;  // at most kSplitMaxChunks (checked on the host)
      const int cb = nch * piece / K, ce = nch * (piece + 1) / K;
      if (cb == 0) {  // the first run, or no crossing at all: from the entry
        jac_start<DT>(vd, r, jr, s);
        if (piece == 0) gcs[lane] = r.ea < 0 ? -s.v : 0.f;  // entry clamped at alpha 0: weight -V_first
      } else if (cb < ce) {
        jac_state_at<DT>(vd, r, jr, &ws, cb * jr.chunk, s);
      }
      for (int k = cb; k < ce; ++k) {
        const int remaining = ncross - k * jr.chunk;
        const int n = min(remaining, jr.chunk);
        jac_chunk<DT>(vd, jr, &ws, s, n, remaining > n, split_chunks[k * 32 + lane]);
      }
      // the final state: the last run's (piece K - 1 walks the ray's last
      // chunk), or piece 0's when the ray has no crossing
      if (piece == (nch > 0 ? K - 1 : 0)) fin[lane] = s;
    }
    __syncthreads();
    if (warp == 0 && valid) {
      const size_t pix = static_cast<size_t>(h) * det.W + w;
      float F = 0.f, J[6] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
      if (rs < 0) {
        F = __int_as_float(0x7fffffff);
#pragma unroll
        for (int k = 0; k < 6; ++k) J[k] = F;
      } else if (rs > 0) {
        JacTotals T{0.f, 0.f, 0.f, 0.f, 0.f};
        for (int k = 0; k < nch; ++k) jac_add_chunk(T, split_chunks[k * 32 + lane]);
        JacSums js;
        jac_finish(r, jr, fin[lane], T, gcs[lane], js);
        const float L = sqrtf(fmaf(r.d[2], r.d[2], fmaf(r.d[1], r.d[1], r.d[0] * r.d[0])));
        F = js.F * L * vd.out_scale;
        pose_jacobian(r, js, pg, e, h, w, vd.out_scale, J);
      }
      out[b * npix + pix] = F;
#pragma unroll
      for (int k = 0; k < 6; ++k) jac[(static_cast<size_t>(b) * 6 + k) * npix + pix] = J[k];
    }
  }
}

// Pose gradient from a stored Jacobian in one launch (Sec. 2.4, chain rule:
// dL/d eta = sum over pixels of dL/dE * dE/d eta).  One thread-block cluster
// per pose: block r of the cluster sums g * J over the r-th of kJacCluster
// contiguous shares of the pose's pixels (in FP32: FP64 arithmetic is narrow
// on this GPU), writes its six sums into a row of block 0's shared memory
// through the cluster's distributed shared memory, and block 0 adds the rows
// in rank order in FP64.  Every sum has a fixed order, so the result is
// bitwise reproducible, and no partial sums leave the chip.
constexpr int kJacCluster = 8;  // blocks per pose (the portable cluster size)
#ifndef DRR_JAC_THREADS
#define DRR_JAC_THREADS 512
#endif
// Threads per block: two 512-thread blocks share an SM, so a cluster spans 4
// SMs and ~38 clusters run at once (1024-thread blocks allowed 15 at once: a
// 16-pose batch took two waves, 16.8 us).
constexpr int kJacThreads = DRR_JAC_THREADS;

__device__ __forceinline__ void jac_fma4(float c[6], const float4 gv, const float* __restrict__ jb, int npix, int i) {
#pragma unroll
  for (int k = 0; k < 6; ++k) {
    const float4 jv = __ldcs(reinterpret_cast<const float4*>(jb + static_cast<size_t>(k) * npix) + i);
    c[k] = fmaf(gv.x, jv.x, c[k]);
    c[k] = fmaf(gv.y, jv.y, c[k]);
    c[k] = fmaf(gv.z, jv.z, c[k]);
    c[k] = fmaf(gv.w, jv.w, c[k]);
  }
}

__global__ void __cluster_dims__(kJacCluster, 1, 1) __launch_bounds__(kJacThreads)
    jac_grad_kernel(const float* __restrict__ gin, const float* __restrict__ jac, int npix, int vec,
                    float* __restrict__ grad) {
  static_assert(kJacThreads % 32 == 0 && kJacThreads <= 32 * 32, "the block sum takes one warp sum per lane");
  __shared__ float wsum[kJacThreads / 32][6];
  __shared__ double rows[kJacCluster][6];  // filled in block 0 only
  namespace cg = cooperative_groups;
  cg::cluster_group cluster = cg::this_cluster();
  const unsigned int rank = cluster.block_rank();
  const int b = blockIdx.y;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  grid_dep_wait();
  grid_dep_release();
  const float* gb = gin + static_cast<size_t>(b) * npix;
  const float* jb = jac + static_cast<size_t>(b) * 6 * npix;
  float c[6] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
  if (vec) {  // npix % 4 == 0 and 16-byte aligned planes: float4 loads
    const int nv = npix >> 2;
    const int lo = static_cast<int>(static_cast<int64_t>(nv) * rank / kJacCluster);
    const int hi = static_cast<int>(static_cast<int64_t>(nv) * (rank + 1) / kJacCluster);
#pragma unroll 1
    for (int i = lo + threadIdx.x; i < hi; i += kJacThreads)
      jac_fma4(c, __ldcs(reinterpret_cast<const float4*>(gb) + i), jb, npix, i);
  } else {
    const int lo = static_cast<int>(static_cast<int64_t>(npix) * rank / kJacCluster);
    const int hi = static_cast<int>(static_cast<int64_t>(npix) * (rank + 1) / kJacCluster);
#pragma unroll 1
    for (int p = lo + threadIdx.x; p < hi; p += kJacThreads) {
      const float gv = __ldcs(gb + p);
#pragma unroll
      for (int k = 0; k < 6; ++k) c[k] = fmaf(gv, __ldcs(jb + static_cast<size_t>(k) * npix + p), c[k]);
    }
  }
#pragma unroll
  for (int k = 0; k < 6; ++k) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) c[k] += __shfl_xor_sync(0xffffffffu, c[k], o);
  }
  if (lane == 0) {
#pragma unroll
    for (int k = 0; k < 6; ++k) wsum[warp][k] = c[k];
  }
  __syncthreads();
  // every block of the cluster is running (its shared memory exists) before any
  // block writes into block 0's
  cluster.sync();
  if (warp == 0) {  // lane q holds warp q's sums; a fixed butterfly adds them
    float t[6];
#pragma unroll
    for (int k = 0; k < 6; ++k) {
      t[k] = lane < kJacThreads / 32 ? wsum[lane][k] : 0.f;
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) t[k] += __shfl_xor_sync(0xffffffffu, t[k], o);
    }
    float mine = t[0];
#pragma unroll
    for (int k = 1; k < 6; ++k)
      if (lane == k) mine = t[k];
    if (lane < 6) cluster.map_shared_rank(&rows[0][0], 0)[rank * 6 + lane] = static_cast<double>(mine);
  }
  cluster.sync();  // rows complete; no block exits while its row is still being written
  if (rank == 0 && threadIdx.x < 6) {
    double t = 0.0;
    for (int r = 0; r < kJacCluster; ++r) t += rows[r][threadIdx.x];
    grad[6 * b + threadIdx.x] = static_cast<float>(t);
  }
}

// Fixed-order FP64 sum of one pose's per-tile partial sums (nt tiles, ncol
// values each, tile-major): thread t adds tiles t, t + kFinThreads, ... in
// order (one coalesced pass for all columns), each warp's sums are combined by
// a fixed shuffle tree, and thread k adds the warps' sums of column k in warp
// order.  The order depends only on nt, so the result is bitwise reproducible,
// and the server and the direct calls, which both finish through here, agree
// bit for bit.  Called by all threads of the block.
constexpr int kFinThreads = 256;

__device__ __forceinline__ void sum_pose_partials(const float* __restrict__ p, int nt, int ncol,
                                                  float* __restrict__ out) {
  __shared__ double wsum[kFinThreads / 32][6];
  const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
  double s[6] = {0.0, 0.0, 0.0, 0.0, 0.0, 0.0};
  for (int c = t; c < nt; c += kFinThreads) {
    const float* row = p + static_cast<size_t>(c) * ncol;
#pragma unroll
    for (int k = 0; k < 6; ++k)
      if (k < ncol) s[k] += static_cast<double>(row[k]);
  }
#pragma unroll
  for (int k = 0; k < 6; ++k) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s[k] += __shfl_xor_sync(0xffffffffu, s[k], o);
  }
  if (lane == 0) {
#pragma unroll
    for (int k = 0; k < 6; ++k) wsum[warp][k] = s[k];
  }
  __syncthreads();
  if (t < ncol) {
    double a = 0.0;
#pragma unroll
    for (int w = 0; w < kFinThreads / 32; ++w) a += wsum[w][t];
    out[t] = static_cast<float>(a);
  }
  __syncthreads();  // wsum is reused by the block's next pose
}

__global__ void __launch_bounds__(kFinThreads) pose_grad_finalize_kernel(const float* __restrict__ partials, int nblk,
                                                                         int ncol, float* __restrict__ grad) {
  grid_dep_wait();
  const int b = blockIdx.x;
  sum_pose_partials(partials + static_cast<size_t>(b) * nblk * ncol, nblk, ncol, grad + static_cast<size_t>(ncol) * b);
}

// ---------------------------------------------------------------------------
// Volume ingest: HU -> attenuation, storage conversion, padded layout.
// ---------------------------------------------------------------------------
__device__ __forceinline__ float source_value(const void* src, int src_dtype, int64_t i, float mu_water) {
  if (src_dtype == 3) {  // int16 HU: mu = max(0, mu_water (1 + HU/1000))
    const float hu = static_cast<float>(static_cast<const short*>(src)[i]);
    return fmaxf(0.f, mu_water * (1.f + hu / 1000.f));
  }
  return static_cast<const float*>(src)[i];
}

__global__ void abs_max_kernel(const void* __restrict__ src, int src_dtype, int64_t count, float mu_water,
                               unsigned int* __restrict__ out_bits) {
  float m = 0.f;
  for (int64_t i = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x; i < count;
       i += static_cast<int64_t>(gridDim.x) * blockDim.x)
    m = fmaxf(m, fabsf(source_value(src, src_dtype, i, mu_water)));
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
  if ((threadIdx.x & 31) == 0) atomicMax(out_bits, __float_as_uint(m));
}

// One thread per padded voxel (pi, pj, pk): x across the threads of a block,
// y and z over the grid (grid-stride), written at pi stride_x + pj stride_y +
// pk stride_z, whichever axis the layout makes fastest; the padding is zero.
__global__ void ingest_kernel(const void* __restrict__ src, int src_dtype, float mu_water, VolumeDev vd,
                              void* __restrict__ dst, float scale) {
  const int px = vd.n[0] + 2, py = vd.n[1] + 2, pz = vd.n[2] + 2;
  const int pi = blockIdx.x * blockDim.x + threadIdx.x;
  if (pi >= px) return;
  for (int pk = blockIdx.z; pk < pz; pk += gridDim.z) {
    for (int pj = blockIdx.y; pj < py; pj += gridDim.y) {
      const int i = pi - 1, j = pj - 1, k = pk - 1;
      float v = 0.f;
      if (i >= 0 && j >= 0 && k >= 0 && i < vd.n[0] && j < vd.n[1] && k < vd.n[2])
        v = source_value(src, src_dtype, (static_cast<int64_t>(k) * vd.n[1] + j) * vd.n[0] + i, mu_water);
      const int64_t e = static_cast<int64_t>(pi) * vd.stride[0] + static_cast<int64_t>(pj) * vd.stride[1] +
                        static_cast<int64_t>(pk) * vd.stride[2];
      if (vd.dtype == kF32) {
        static_cast<float*>(dst)[e] = v;
      } else if (vd.dtype == kBF16) {
        static_cast<__nv_bfloat16*>(dst)[e] = __float2bfloat16_rn(v);
      } else {
        static_cast<__half*>(dst)[e] = __float2half_rn(v * scale);
      }
    }
  }
}

// ---------------------------------------------------------------------------
// Serving tick kernels: one launch each covers every admitted request.
// ---------------------------------------------------------------------------
// Index of the request whose [start, next start) range holds `i` (starts ascending).
__device__ __forceinline__ int find_request(const ServeRequest* reqs, int nreq, int i, bool by_tile) {
  int lo = 0, hi = nreq - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    const int st = by_tile ? reqs[mid].tile_start : reqs[mid].pose_start;
    if (st <= i) lo = mid;
    else hi = mid - 1;
  }
  return lo;
}

// One warp (block) per pose, grid-stride over the tick's poses.  A pose index
// that decodes outside its request (an inconsistent tick table) sets the
// request's status word and is skipped.
__global__ void __launch_bounds__(32) serve_setup_kernel(const ServeHeader* __restrict__ hdr,
                                                         const ServeRequest* __restrict__ reqs,
                                                         unsigned int* __restrict__ status) {
  const int nreq = hdr->nreq, total = hdr->total_poses;
  for (int i = blockIdx.x; i < total; i += gridDim.x) {
    const int r = find_request(reqs, nreq, i, false);
    const int b = i - reqs[r].pose_start;
    if (b < 0 || b >= reqs[r].B) {  // uniform in the warp
      if (threadIdx.x == 0) atomicOr(status + r, kServePoseRange);
      continue;
    }
    warp_pose_geom(reqs[r].poses + 6 * b, reqs[r].det, reqs[r].vd, reqs[r].geom + b);
  }
}

template <int MODE>
__device__ __forceinline__ void serve_trace(const VolumeDev& vd, const PoseGeom& pg, int h, int w, float gsc,
                                            WalkScratch* ws, RayResult& r) {
  switch (vd.dtype) {
    case kF32: trace_ray<MODE, kF32>(vd, pg, h, w, gsc, nullptr, ws, r); break;
    case kBF16: trace_ray<MODE, kBF16>(vd, pg, h, w, gsc, nullptr, ws, r); break;
    default: trace_ray<MODE, kF16>(vd, pg, h, w, gsc, nullptr, ws, r); break;
  }
}

// Persistent walk: warps claim 8x4-pixel tiles of any request (numbered per
// request as in siddon_kernel, pose-major) until the tick's tiles run out, so
// a small request spreads over many SMs.  Render-only tiles run the forward
// walk, gradient tiles the Jacobian walk with the warp's sum of g . J written
// per tile; a warp copies its request's record and pose geometry to its own
// shared slots when they change.
__global__ void __launch_bounds__(kThreads, 4) serve_walk_kernel(const ServeHeader* __restrict__ hdr,
                                                                 const ServeRequest* __restrict__ reqs,
                                                                 unsigned int* __restrict__ status,
                                                                 int* __restrict__ counter) {
  __shared__ PoseGeom spg[kThreads / 32];
  __shared__ ServeRequest sreq[kThreads / 32];
  __shared__ JacScratch ws;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int nreq = hdr->nreq, total = hdr->total_tiles;
  ServeRequest& sr = sreq[warp];
  PoseGeom& pg = spg[warp];
  int cur_r = -1, cur_b = -1;
  for (;;) {
    int t = 0;
    if (lane == 0) t = atomicAdd(counter, 1);
    t = __shfl_sync(0xffffffffu, t, 0);  // also: every lane is done with the previous tile
    if (t >= total) break;
    const int r = find_request(reqs, nreq, t, true);
    if (r != cur_r) {
      const unsigned int* src = reinterpret_cast<const unsigned int*>(reqs + r);
      unsigned int* dst = reinterpret_cast<unsigned int*>(&sr);
      for (int i = lane; i < static_cast<int>(sizeof(ServeRequest) / 4); i += 32) dst[i] = src[i];
      __syncwarp();
      cur_r = r;
      cur_b = -1;
    }
    const int per_pose = pose_tiles(sr.det);
    const int local = t - sr.tile_start;
    const int b = local / per_pose;
    if (b < 0 || b >= sr.B) {  // the tick table's tile ranges, checked (uniform in the warp)
      if (lane == 0) atomicOr(status + r, kServeTileRange);
      continue;
    }
    const int tin = local - b * per_pose;
    if (b != cur_b) {
      const unsigned int* src = reinterpret_cast<const unsigned int*>(sr.geom + b);
      unsigned int* dst = reinterpret_cast<unsigned int*>(&pg);
      for (int i = lane; i < static_cast<int>(sizeof(PoseGeom) / 4); i += 32) dst[i] = src[i];
      __syncwarp();
      cur_b = b;
    }
    const int twx = (sr.det.W + kWarpTileW - 1) / kWarpTileW;
    const int ty = tin / twx, tx = tin - ty * twx;
    const int h = ty * kWarpTileH + lane / kWarpTileW, w = tx * kWarpTileW + lane % kWarpTileW;
    const bool valid = (w < sr.det.W) && (h < sr.det.H);
    const size_t npix = static_cast<size_t>(sr.det.H) * sr.det.W;
    const size_t pix = static_cast<size_t>(h) * sr.det.W + w;
    const bool want_grad = sr.grad != nullptr;
    RayResult res;
    res.F = 0.f;
#pragma unroll
    for (int k = 0; k < 6; ++k) res.J[k] = 0.f;
    float gsc = 0.f;
    if (valid) {
      if (want_grad) {
        gsc = sr.grad[b * npix + pix];
        serve_trace<kPoseGrad>(sr.vd, pg, h, w, gsc, &ws, res);
      } else {
        serve_trace<kFwd>(sr.vd, pg, h, w, 0.f, &ws, res);
      }
      sr.out[b * npix + pix] = res.F;
    }
    if (want_grad) {  // uniform across the warp: one partial per tile, as a direct render_backward
      float c[6];
#pragma unroll
      for (int k = 0; k < 6; ++k) {
        c[k] = gsc * res.J[k];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) c[k] += __shfl_xor_sync(0xffffffffu, c[k], o);
      }
      if (lane == 0) {
        const size_t slot = static_cast<size_t>(b) * per_pose + tin;
#pragma unroll
        for (int k = 0; k < 6; ++k) sr.partials[slot * 6 + k] = c[k];
      }
    }
  }
}

// Each gradient request's pose gradients from its per-tile partials: one block
// per pose, summed in the fixed order of sum_pose_partials.
__global__ void __launch_bounds__(kFinThreads) serve_finalize_kernel(const ServeHeader* __restrict__ hdr,
                                                                     const ServeRequest* __restrict__ reqs) {
  const int nreq = hdr->nreq, total = hdr->total_poses;
  for (int i = blockIdx.x; i < total; i += gridDim.x) {
    const int r = find_request(reqs, nreq, i, false);
    const ServeRequest& q = reqs[r];
    if (q.grad == nullptr) continue;  // uniform across the block
    const int b = i - q.pose_start;
    if (b < 0 || b >= q.B) continue;  // flagged by serve_setup_kernel (same decode)
    const int nt = pose_tiles(q.det);
    sum_pose_partials(q.partials + static_cast<size_t>(b) * nt * 6, nt, 6, q.grad_pose + 6 * b);
  }
}

// Launch with programmatic stream serialization (the kernel must begin with
// grid_dep_wait()); -DDRR_PDL=0 launches plainly.
#ifndef DRR_PDL
#define DRR_PDL 1
#endif
template <typename... KArgs, typename... Args>
cudaError_t launch_pdl_smem(void (*kernel)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t stream,
                            Args... args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = grid;
  cfg.blockDim = block;
  cfg.dynamicSmemBytes = smem;
  cfg.stream = stream;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = DRR_PDL ? 1 : 0;
  return cudaLaunchKernelEx(&cfg, kernel, static_cast<KArgs>(args)...);
}

template <typename... KArgs, typename... Args>
cudaError_t launch_pdl(void (*kernel)(KArgs...), dim3 grid, dim3 block, cudaStream_t stream, Args... args) {
  return launch_pdl_smem(kernel, grid, block, 0, stream, args...);
}

int grid_for(int64_t n, int threads) {
  int64_t g = (n + threads - 1) / threads;
  if (g > 152 * 64) g = 152 * 64;
  return static_cast<int>(g < 1 ? 1 : g);
}

// Blocks of one walk-kernel instance that fit on the device at once (cached per device).
template <int MODE, int DT>
int resident_blocks() {
  constexpr int kMaxDev = 64;
  static std::atomic<int> cache[kMaxDev] = {};  // calls from several host threads may race to fill it
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDev) dev = 0;
  int v = cache[dev].load(std::memory_order_relaxed);
  if (v == 0) {
    int sms = 0, per_sm = 0;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, siddon_kernel<MODE, DT>, kThreads, 0);
    v = (sms > 0 ? sms : 1) * (per_sm > 0 ? per_sm : 1);
    cache[dev].store(v, std::memory_order_relaxed);
  }
  return v;
}

// The split kernel with K warps per tile: its dynamic shared memory (the chunk
// sums of one tile's rays) and the blocks of it the device holds at once
// (cached per device; 0 if it cannot be configured).
constexpr size_t kSplitSmem = static_cast<size_t>(kSplitMaxChunks) * 32 * sizeof(JacChunk);
template <int DT, int K>
int split_resident_blocks() {
  constexpr int kMaxDev = 64;
  static std::atomic<int> cache[kMaxDev] = {};  // calls from several host threads may race to fill it
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDev) return 0;
  int v = cache[dev].load(std::memory_order_relaxed);
  if (v == 0) {
    int sms = 0, per_sm = 0;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (cudaFuncSetAttribute(siddon_split_kernel<DT, K>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             static_cast<int>(kSplitSmem)) != cudaSuccess ||
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, siddon_split_kernel<DT, K>, 32 * K, kSplitSmem) !=
            cudaSuccess) {
      cudaGetLastError();
      v = -1;
    } else {
      v = per_sm > 0 ? sms * per_sm : -1;
    }
    cache[dev].store(v, std::memory_order_relaxed);
  }
  return v > 0 ? v : 0;
}

template <int DT, int K>
cudaError_t launch_split(const VolumeDev& vd, const DetDev& det, const PoseGeom* pg, int B, unsigned int* counter,
                         float* out, float* jac, cudaStream_t stream) {
  const int64_t tiles = static_cast<int64_t>(pose_tiles(det)) * B;
  const int grid = static_cast<int>(std::min<int64_t>(tiles, split_resident_blocks<DT, K>()));
  return launch_pdl_smem(siddon_split_kernel<DT, K>, dim3(grid), dim3(32 * K), kSplitSmem, stream, vd, det, pg, B,
                         counter, out, jac);
}

// Warps per ray (per warp tile) for a fused forward + Jacobian launch: 8 or 4
// when the split kernel's resident blocks can take every tile of the launch at
// once (the whole-ray walk would leave most of the GPU idle, latency-bound on
// few warps), 1 otherwise.  Rays are split only where every ray fits the split
// kernel's chunk table (nx + ny + nz <= 61 * kSplitMaxChunks).
#ifndef DRR_SPLIT
#define DRR_SPLIT 1
#endif
template <int DT>
int split_lanes(const VolumeDev& vd, const DetDev& det, int B) {
  if (!DRR_SPLIT) return 1;
  if (static_cast<int64_t>(vd.n[0]) + vd.n[1] + vd.n[2] > static_cast<int64_t>(DRR_JAC_LONG) * kSplitMaxChunks) return 1;
  const int64_t tiles = static_cast<int64_t>(pose_tiles(det)) * B;
  if (tiles <= split_resident_blocks<DT, 8>()) return 8;
  if (tiles <= split_resident_blocks<DT, 4>()) return 4;
  return 1;
}

template <int MODE, int DT>
cudaError_t launch_siddon_dt(const VolumeDev& vd, const DetDev& det, const PoseGeom* pg, int B, unsigned int* counter,
                             float* out, float* jac, const float* gin, float* partials, float* gvol,
                             cudaStream_t stream, int lanes = 1) {
  if (MODE == kFwdJac) {
    if (lanes == 8) return launch_split<DT, 8>(vd, det, pg, B, counter, out, jac, stream);
    if (lanes == 4) return launch_split<DT, 4>(vd, det, pg, B, counter, out, jac, stream);
  }
  const int64_t tiles = static_cast<int64_t>(pose_tiles(det)) * B;
  const int64_t want = (tiles + kThreads / 32 - 1) / (kThreads / 32);
  const int grid = static_cast<int>(std::min<int64_t>(want, resident_blocks<MODE, DT>()));
  return launch_pdl(siddon_kernel<MODE, DT>, dim3(grid), dim3(kThreads), stream, vd, det, pg, B, counter, out, jac, gin,
                    partials, gvol);
}

template <int MODE>
cudaError_t launch_siddon(const VolumeDev& vd, const DetDev& det, const PoseGeom* pg, int B, float* out, float* jac,
                          const float* gin, float* partials, float* gvol, cudaStream_t stream, int lanes = 1) {
  // one counter per walk kind, so a geometry can serve one launch of each
  const int slot = MODE == kPoseGrad ? 1 : (MODE == kBackproject ? 2 : (MODE == kGeoGrad ? 3 : 0));
  unsigned int* counter = reinterpret_cast<unsigned int*>(const_cast<PoseGeom*>(pg) + B) + slot;
  switch (vd.dtype) {
    case kF32:
      return launch_siddon_dt<MODE, kF32>(vd, det, pg, B, counter, out, jac, gin, partials, gvol, stream, lanes);
    case kBF16:
      return launch_siddon_dt<MODE, kBF16>(vd, det, pg, B, counter, out, jac, gin, partials, gvol, stream, lanes);
    default:
      return launch_siddon_dt<MODE, kF16>(vd, det, pg, B, counter, out, jac, gin, partials, gvol, stream, lanes);
  }
}

// ---------------------------------------------------------------------------
// Comparison baseline: the plain FP32 forward path.  The textbook incremental
// Siddon-Jacobs walk (Sec. 2.2, Eq. 2-3) entirely in FP32: one thread per ray
// in 16x16 blocks, FP32 clip (Sec. 2.3), each axis' next crossing advanced by
// repeated FP32 addition, the voxel of the first segment from its midpoint.
// It is what the product walk is measured against; its rounding drift is
// why the product walk anchors its crossings in fixed point.
// ---------------------------------------------------------------------------
template <int DT>
__global__ void __launch_bounds__(256) plain_fp32_kernel(VolumeDev vd, DetDev det, const PoseGeom* __restrict__ pgs,
                                                         float* __restrict__ out) {
  const int w = blockIdx.x * 16 + (threadIdx.x & 15), h = blockIdx.y * 16 + (threadIdx.x >> 4), b = blockIdx.z;
  if (w >= det.W || h >= det.H) return;
  const PoseGeom& pg = pgs[b];
  float u0[3], g[3], amin = 0.f, amax = 1.f;
  bool hit = true;
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    u0[a] = pg.u0f[a];
    g[a] = static_cast<float>(pg.g00[a]) + static_cast<float>(w) * static_cast<float>(pg.gw[a]) +
           static_cast<float>(h) * static_cast<float>(pg.gh[a]);
    if (g[a] != 0.f) {
      const float t0 = -u0[a] / g[a], t1 = (static_cast<float>(vd.n[a]) - u0[a]) / g[a];
      amin = fmaxf(amin, fminf(t0, t1));
      amax = fminf(amax, fmaxf(t0, t1));
    } else if (!(u0[a] >= 0.f && u0[a] < static_cast<float>(vd.n[a]))) {
      hit = false;
    }
  }
  float acc = 0.f;
  if (hit && amin < amax) {
    float an[3], da[3];
    int idx[3], st[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      const float ue = u0[a] + amin * g[a];
      if (g[a] > 0.f) {
        an[a] = (floorf(ue) + 1.f - u0[a]) / g[a];
        da[a] = 1.f / g[a];
        st[a] = 1;
      } else if (g[a] < 0.f) {
        an[a] = (ceilf(ue) - 1.f - u0[a]) / g[a];
        da[a] = -1.f / g[a];
        st[a] = -1;
      } else {
        an[a] = 2.f;
        da[a] = 0.f;
        st[a] = 0;
      }
    }
    const float first = fminf(fminf(fminf(an[0], an[1]), an[2]), amax);
    const float am = 0.5f * (amin + first);
#pragma unroll
    for (int a = 0; a < 3; ++a) idx[a] = static_cast<int>(floorf(u0[a] + am * g[a]));
    // scalar copies: the walk indexes no register array
    float ax = an[0], ay = an[1], az = an[2];
    int ix = idx[0], iy = idx[1], iz = idx[2];
    float al = amin;
    for (int guard = 0; guard < 4 * (vd.n[0] + vd.n[1] + vd.n[2]) + 8 && al < amax; ++guard) {
      const float nx = fminf(fminf(fminf(ax, ay), az), amax);
      if (ix >= 0 && ix < vd.n[0] && iy >= 0 && iy < vd.n[1] && iz >= 0 && iz < vd.n[2])
        acc += (nx - al) * Voxel<DT>::load(vd.data, vd.origin + ix * vd.stride[0] + iy * vd.stride[1] +
                                                         iz * vd.stride[2]);
      al = nx;
      const bool sx = ax == nx, sy = !sx && ay == nx, sz = !sx && !sy;
      if (sx) { ix += st[0]; ax += da[0]; }
      if (sy) { iy += st[1]; ay += da[1]; }
      if (sz) { iz += st[2]; az += da[2]; }
    }
  }
#pragma unroll
  for (int a = 0; a < 3; ++a) g[a] *= vd.delta[a];
  out[(static_cast<size_t>(b) * det.H + h) * det.W + w] = acc * sqrtf(g[0] * g[0] + g[1] * g[1] + g[2] * g[2]) *
                                                          vd.out_scale;
}

// The comparison server's central differences (see launch_plain_fd_finish).
__global__ void plain_fd_finish_kernel(const float* __restrict__ E13, int B, int npix, float h_rot, float h_trans,
                                       float* __restrict__ out, float* __restrict__ jac) {
  const int64_t n = static_cast<int64_t>(B) * npix;
  for (int64_t i = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x; i < n;
       i += static_cast<int64_t>(gridDim.x) * blockDim.x) {
    const int b = static_cast<int>(i / npix);
    const int p = static_cast<int>(i - static_cast<int64_t>(b) * npix);
    const float* e = E13 + static_cast<size_t>(b) * 13 * npix + p;
    out[i] = e[0];
#pragma unroll
    for (int k = 0; k < 6; ++k) {
      const float h2 = 2.f * (k < 3 ? h_rot : h_trans);
      jac[(static_cast<size_t>(b) * 6 + k) * npix + p] = (e[static_cast<size_t>(1 + 2 * k) * npix] -
                                                          e[static_cast<size_t>(2 + 2 * k) * npix]) / h2;
    }
  }
}

}  // namespace

cudaError_t read_and_clear_fault(unsigned int* bits) {
  *bits = 0u;
#if DRR_CHECK_BOUNDS
  cudaError_t e = cudaMemcpyFromSymbol(bits, g_fault_word, sizeof(unsigned int));
  if (e != cudaSuccess) return e;
  const unsigned int zero = 0u;
  if (*bits) e = cudaMemcpyToSymbol(g_fault_word, &zero, sizeof(unsigned int));
  return e;
#else
  return cudaSuccess;
#endif
}

bool bounds_checked() { return DRR_CHECK_BOUNDS != 0; }

cudaError_t launch_plain_fd_finish(const float* E13, int B, int npix, float h_rot, float h_trans, float* out,
                                   float* jac, cudaStream_t stream) {
  plain_fd_finish_kernel<<<grid_for(static_cast<int64_t>(B) * npix, 256), 256, 0, stream>>>(E13, B, npix, h_rot,
                                                                                          h_trans, out, jac);
  return cudaGetLastError();
}

cudaError_t launch_render_plain_fp32(const VolumeDev& vd, const DetDev& det, const PoseGeom* pg, int B, float* out,
                                     cudaStream_t stream) {
  dim3 grid((det.W + 15) / 16, (det.H + 15) / 16, B);
  switch (vd.dtype) {
    case kF32: plain_fp32_kernel<kF32><<<grid, 256, 0, stream>>>(vd, det, pg, out); break;
    case kBF16: plain_fp32_kernel<kBF16><<<grid, 256, 0, stream>>>(vd, det, pg, out); break;
    default: plain_fp32_kernel<kF16><<<grid, 256, 0, stream>>>(vd, det, pg, out); break;
  }
  return cudaGetLastError();
}

cudaError_t launch_pose_setup(const float* poses, int B, const DetDev& det, const VolumeDev* vd, PoseGeom* out,
                              cudaStream_t stream) {
  return launch_pdl(pose_setup_kernel, dim3(B), dim3(32), stream, poses, B, det, *vd, out);
}

cudaError_t launch_ray_setup(const float* poses, int B, const DetDev& det, float* rays, cudaStream_t stream) {
  const int64_t n = static_cast<int64_t>(B) * det.H * det.W;
  ray_setup_kernel<<<static_cast<unsigned int>((n + 255) / 256), 256, 0, stream>>>(poses, B, det, rays);
  return cudaGetLastError();
}

int render_split_lanes(const VolumeDev& vd, const DetDev& det, int B) {
  switch (vd.dtype) {
    case kF32: return split_lanes<kF32>(vd, det, B);
    case kBF16: return split_lanes<kBF16>(vd, det, B);
    default: return split_lanes<kF16>(vd, det, B);
  }
}

cudaError_t launch_render(const VolumeDev& vd, const DetDev& det, const PoseGeom* pg, int B, float* out, float* jac,
                          cudaStream_t stream, int lanes) {
  if (jac) return launch_siddon<kFwdJac>(vd, det, pg, B, out, jac, nullptr, nullptr, nullptr, stream, lanes);
  return launch_siddon<kFwd>(vd, det, pg, B, out, nullptr, nullptr, nullptr, nullptr, stream);
}

cudaError_t launch_pose_grad_walk(const VolumeDev& vd, const DetDev& det, const PoseGeom* pg, int B,
                                  const float* grad_drr, float* partials, cudaStream_t stream) {
  return launch_siddon<kPoseGrad>(vd, det, pg, B, nullptr, nullptr, grad_drr, partials, nullptr, stream);
}

cudaError_t launch_pose_grad_from_jacobian(const DetDev& det, int B, const float* grad_drr, const float* jac,
                                           float* grad_pose, cudaStream_t stream) {
  const int npix = det.H * det.W;
  const int vec = (npix % 4 == 0) && (reinterpret_cast<uintptr_t>(grad_drr) % 16 == 0) &&
                  (reinterpret_cast<uintptr_t>(jac) % 16 == 0);
  return launch_pdl(jac_grad_kernel, dim3(kJacCluster, B), dim3(kJacThreads), stream, grad_drr, jac, npix, vec,
                    grad_pose);
}

cudaError_t launch_count_segments(const VolumeDev& vd, const DetDev& det, const PoseGeom* pg, int B, int* counts,
                                  cudaStream_t stream) {
  return launch_siddon<kCount>(vd, det, pg, B, reinterpret_cast<float*>(counts), nullptr, nullptr, nullptr, nullptr,
                               stream);
}

cudaError_t launch_pose_grad_finalize(const float* partials, int B, int nblk, float* grad_pose, cudaStream_t stream) {
  return launch_pdl(pose_grad_finalize_kernel, dim3(B), dim3(kFinThreads), stream, partials, nblk, 6, grad_pose);
}

cudaError_t launch_geometry_grad(const VolumeDev& vd, const DetDev& det, const PoseGeom* pg, int B,
                                 const float* grad_drr, float* partials, float* grad_geometry, cudaStream_t stream) {
  cudaError_t e = launch_siddon<kGeoGrad>(vd, det, pg, B, nullptr, nullptr, grad_drr, partials, nullptr, stream);
  if (e != cudaSuccess) return e;
  return launch_pdl(pose_grad_finalize_kernel, dim3(B), dim3(kFinThreads), stream, static_cast<const float*>(partials),
                    pose_tiles(det), 3, grad_geometry);
}

cudaError_t launch_backproject(const VolumeDev& vd, const DetDev& det, const PoseGeom* pg, int B,
                               const float* grad_drr, float* grad_vol, cudaStream_t stream) {
  return launch_siddon<kBackproject>(vd, det, pg, B, nullptr, nullptr, grad_drr, nullptr, grad_vol, stream);
}

int serve_walk_grid(int device) {
  int sms = 0, per_sm = 0;
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device);
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, serve_walk_kernel, kThreads, 0);
  return max(1, sms * max(per_sm, 1));
}

cudaError_t launch_serve_tick(const ServeHeader* hdr, const ServeRequest* reqs, unsigned int* status, int* counter,
                              int max_poses, int walk_grid, cudaStream_t stream) {
  cudaError_t e = cudaMemsetAsync(counter, 0, sizeof(int), stream);
  if (e != cudaSuccess) return e;
  // setup and finalize stride over the tick's poses: one block per pose up to
  // the walk's grid, so that a small tick does not pay for thousands of idle blocks
  const int aux = max(1, min(max_poses, walk_grid));
  serve_setup_kernel<<<aux, 32, 0, stream>>>(hdr, reqs, status);
  serve_walk_kernel<<<walk_grid, kThreads, 0, stream>>>(hdr, reqs, status, counter);
  serve_finalize_kernel<<<aux, kFinThreads, 0, stream>>>(hdr, reqs);
  return cudaGetLastError();
}

cudaError_t launch_abs_max(const void* src, int src_dtype, int64_t count, float mu_water, unsigned int* out_bits,
                           cudaStream_t stream) {
  abs_max_kernel<<<grid_for(count, 256), 256, 0, stream>>>(src, src_dtype, count, mu_water, out_bits);
  return cudaGetLastError();
}

cudaError_t launch_ingest(const void* src, int src_dtype, float mu_water, const VolumeDev& vd, void* dst, float scale,
                          cudaStream_t stream) {
  const dim3 grid((vd.n[0] + 2 + 255) / 256, std::min(vd.n[1] + 2, 65535), std::min(vd.n[2] + 2, 65535));
  ingest_kernel<<<grid, 256, 0, stream>>>(src, src_dtype, mu_water, vd, dst, scale);
  return cudaGetLastError();
}

}  // namespace drr
