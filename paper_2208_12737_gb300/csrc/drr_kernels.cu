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
#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include "drr_internal.cuh"

namespace drr {
namespace {

constexpr float kNoCrossing = 4.0f;  // relative alpha never exceeds 1

enum Mode : int { kFwd = 0, kFwdJac = 1, kPoseGrad = 2, kBackproject = 3, kCount = 4 };

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

// ---------------------------------------------------------------------------
// Pose -> frame (Sec. 2.4), FP64.  R = Rz(eta0) Ry(eta1) Rx(eta2).
// ---------------------------------------------------------------------------
__device__ void mul3(const double* A, const double* B, double* C) {
#pragma unroll
  for (int r = 0; r < 3; ++r)
#pragma unroll
    for (int c = 0; c < 3; ++c) C[3 * r + c] = A[3 * r] * B[c] + A[3 * r + 1] * B[3 + c] + A[3 * r + 2] * B[6 + c];
}

__device__ void apply3(const double* A, const double* x, double* y) {
#pragma unroll
  for (int r = 0; r < 3; ++r) y[r] = A[3 * r] * x[0] + A[3 * r + 1] * x[1] + A[3 * r + 2] * x[2];
}

// World-space frame of one pose: source s, pixel (0,0) centre p00, the
// per-column and per-row pixel steps ew, eh, and optionally dR/d eta_j.
__device__ void pose_frame(const float* pose, const DetDev& det, double s[3], double p00[3], double ew[3],
                           double eh[3], double sc_out[3], double pc00_out[3], double* dR /*27 or null*/) {
  double sz, cz, sy, cy, sx, cx;
  sincos(static_cast<double>(pose[0]), &sz, &cz);
  sincos(static_cast<double>(pose[1]), &sy, &cy);
  sincos(static_cast<double>(pose[2]), &sx, &cx);
  const double Rz[9] = {cz, -sz, 0, sz, cz, 0, 0, 0, 1};
  const double Ry[9] = {cy, 0, sy, 0, 1, 0, -sy, 0, cy};
  const double Rx[9] = {1, 0, 0, 0, cx, -sx, 0, sx, cx};
  double T[9], R[9];
  mul3(Rz, Ry, T);
  mul3(T, Rx, R);
  if (dR) {
    const double dRz[9] = {-sz, -cz, 0, cz, -sz, 0, 0, 0, 0};
    const double dRy[9] = {-sy, 0, cy, 0, 0, 0, -cy, 0, -sy};
    const double dRx[9] = {0, 0, 0, 0, -sx, -cx, 0, cx, -sx};
    double U[9];
    mul3(dRz, Ry, U);
    mul3(U, Rx, dR);
    mul3(Rz, dRy, U);
    mul3(U, Rx, dR + 9);
    mul3(T, dRx, dR + 18);
  }
  const double rho = 0.5 * static_cast<double>(det.sdr);
  const double sc[3] = {rho, 0.0, 0.0};
  const double pc00[3] = {-rho, -0.5 * static_cast<double>(det.W - 1) * static_cast<double>(det.dw),
                          -0.5 * static_cast<double>(det.H - 1) * static_cast<double>(det.dh)};
  const double vw[3] = {0.0, static_cast<double>(det.dw), 0.0};
  const double vh[3] = {0.0, 0.0, static_cast<double>(det.dh)};
  apply3(R, sc, s);
  apply3(R, pc00, p00);
  apply3(R, vw, ew);
  apply3(R, vh, eh);
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    s[a] += static_cast<double>(pose[3 + a]);
    p00[a] += static_cast<double>(pose[3 + a]);
    sc_out[a] = sc[a];
    pc00_out[a] = pc00[a];
  }
}

__global__ void pose_setup_kernel(const float* __restrict__ poses, int B, DetDev det, VolumeDev vd,
                                  PoseGeom* __restrict__ out) {
  const int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= B) return;
  double s[3], p00[3], ew[3], eh[3], sc[3], pc00[3], dR[27];
  pose_frame(poses + 6 * b, det, s, p00, ew, eh, sc, pc00, dR);
  PoseGeom g;
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    const double dl = static_cast<double>(vd.delta[a]);
    const double lo = -0.5 * static_cast<double>(vd.n[a]) * dl;  // b_a: volume centred at the origin
    g.u0[a] = (s[a] - lo) / dl;
    g.un[a] = static_cast<double>(vd.n[a]) - g.u0[a];
    g.g00[a] = (p00[a] - s[a]) / dl;
    g.gw[a] = ew[a] / dl;
    g.gh[a] = eh[a] / dl;
  }
  const double q[3] = {pc00[0] - sc[0], pc00[1] - sc[1], pc00[2] - sc[2]};
  const double vw[3] = {0.0, static_cast<double>(det.dw), 0.0};
  const double vh[3] = {0.0, 0.0, static_cast<double>(det.dh)};
#pragma unroll
  for (int j = 0; j < 3; ++j) {
    double t[3];
    apply3(dR + 9 * j, sc, t);
    for (int a = 0; a < 3; ++a) g.S[j][a] = static_cast<float>(t[a]);
    apply3(dR + 9 * j, q, t);
    for (int a = 0; a < 3; ++a) g.Q[j][a] = static_cast<float>(t[a]);
    apply3(dR + 9 * j, vw, t);
    for (int a = 0; a < 3; ++a) g.Wv[j][a] = static_cast<float>(t[a]);
    apply3(dR + 9 * j, vh, t);
    for (int a = 0; a < 3; ++a) g.Hv[j][a] = static_cast<float>(t[a]);
  }
  out[b] = g;
}

__global__ void ray_setup_kernel(const float* __restrict__ poses, int B, DetDev det, float* __restrict__ rays) {
  const int64_t i = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
  const int64_t npix = static_cast<int64_t>(det.H) * det.W;
  if (i >= npix * B) return;
  const int b = static_cast<int>(i / npix);
  const int q = static_cast<int>(i % npix);
  const int h = q / det.W, w = q % det.W;
  double s[3], p00[3], ew[3], eh[3], sc[3], pc00[3];
  pose_frame(poses + 6 * b, det, s, p00, ew, eh, sc, pc00, nullptr);
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

// Block-wide sum of 6 floats per thread; thread 0 gets the totals.
__device__ __forceinline__ void block_sum6(float v[6], float (*sm)[6]) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int k = 0; k < 6; ++k) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v[k] += __shfl_xor_sync(0xffffffffu, v[k], o);
  }
  if (lane == 0) {
#pragma unroll
    for (int k = 0; k < 6; ++k) sm[warp][k] = v[k];
  }
  __syncthreads();
  if (threadIdx.x == 0) {
#pragma unroll
    for (int k = 0; k < 6; ++k) {
      float t = 0.f;
      for (int q = 0; q < kThreads / 32; ++q) t += sm[q][k];
      v[k] = t;
    }
  }
}

template <int MODE, int DT>
__device__ __forceinline__ void trace_ray(const VolumeDev& vd, const PoseGeom& pg, int h, int w, float gscale,
                                          float* __restrict__ gvol, RayResult& res) {
  res.F = 0.f;
  res.nseg = 0;
#pragma unroll
  for (int k = 0; k < 6; ++k) res.J[k] = 0.f;

  // Direction p - s in voxel units for this pixel (FP64).
  double g[3];
#pragma unroll
  for (int a = 0; a < 3; ++a) g[a] = fma(static_cast<double>(h), pg.gh[a], fma(static_cast<double>(w), pg.gw[a], pg.g00[a]));

  // Clip to the volume box: a_min = max of per-axis entries, a_max = min of
  // exits (Sec. 2.3), clamped to [0, 1].  An axis with g == 0 constrains
  // nothing if the ray lies inside its slab [0, n), else the ray misses.
  double amin = 0.0, amax = 1.0, rg[3];
  int ea = -1, xa = -1;
  bool hit = true;
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    if (g[a] != 0.0) {
      rg[a] = 1.0 / g[a];
      const double t0 = -pg.u0[a] * rg[a], t1 = pg.un[a] * rg[a];
      const double lo = fmin(t0, t1), hi = fmax(t0, t1);
      if (lo > amin) { amin = lo; ea = a; }
      if (hi < amax) { amax = hi; xa = a; }
    } else {
      rg[a] = 0.0;
      if (!(pg.u0[a] >= 0.0 && pg.un[a] > 0.0)) hit = false;
    }
  }
  if (!hit || !(amin < amax)) return;

  // Entry and exit voxels, crossing counts and the first crossing of each
  // axis measured from the entry point (FP64, then FP32).
  int ient[3], cnt[3];
  float a_first[3], a_step[3];
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    const int n = vd.n[a];
    if (g[a] == 0.0) {
      ient[a] = min(max(static_cast<int>(floor(pg.u0[a])), 0), n - 1);
      cnt[a] = 0;
      a_first[a] = kNoCrossing;
      a_step[a] = 0.f;
      continue;
    }
    const bool up = g[a] > 0.0;
    const double ue = fma(amin, g[a], pg.u0[a]);
    const double ux = fma(amax, g[a], pg.u0[a]);
    int i0, i1;
    if (a == ea) i0 = up ? 0 : n - 1;
    else i0 = up ? static_cast<int>(floor(ue)) : static_cast<int>(ceil(ue)) - 1;
    if (a == xa) i1 = up ? n - 1 : 0;
    else i1 = up ? static_cast<int>(ceil(ux)) - 1 : static_cast<int>(floor(ux));
    i0 = min(max(i0, 0), n - 1);
    i1 = min(max(i1, 0), n - 1);
    ient[a] = i0;
    cnt[a] = max(up ? i1 - i0 : i0 - i1, 0);
    const double plane = static_cast<double>(up ? i0 + 1 : i0);
    a_first[a] = cnt[a] > 0 ? static_cast<float>((plane - ue) * rg[a]) : kNoCrossing;
    a_step[a] = static_cast<float>(fabs(rg[a]));
  }
  const float span = static_cast<float>(amax - amin);
  const int nseg = cnt[0] + cnt[1] + cnt[2] + 1;
  res.nseg = nseg;
  if (MODE == kCount) return;

  int off = vd.origin + ient[0] * vd.stride[0] + ient[1] * vd.stride[1] + ient[2] * vd.stride[2];
  const int sx = g[0] > 0.0 ? vd.stride[0] : -vd.stride[0];
  const int sy = g[1] > 0.0 ? vd.stride[1] : -vd.stride[1];
  const int sz = g[2] > 0.0 ? vd.stride[2] : -vd.stride[2];

  // Linear index into an unpadded (nz, ny, nx) gradient volume (back-projection).
  int lin = 0, lx = 0, ly = 0, lz = 0;
  unsigned int nvox = 0;
  float gL = 0.f;
  if (MODE == kBackproject) {
    lin = ient[0] + vd.n[0] * (ient[1] + vd.n[1] * ient[2]);
    lx = g[0] > 0.0 ? 1 : -1;
    ly = g[1] > 0.0 ? vd.n[0] : -vd.n[0];
    lz = g[2] > 0.0 ? vd.n[0] * vd.n[1] : -(vd.n[0] * vd.n[1]);
    nvox = static_cast<unsigned int>(vd.n[0] * vd.n[1] * vd.n[2]);
    const float dx = static_cast<float>(g[0]) * vd.delta[0], dy = static_cast<float>(g[1]) * vd.delta[1],
                dz = static_cast<float>(g[2]) * vd.delta[2];
    gL = gscale * sqrtf(dx * dx + dy * dy + dz * dz);
  }

  float ax = a_first[0], ay = a_first[1], az = a_first[2];
  float kx = 0.f, ky = 0.f, kz = 0.f;
  float acc = 0.f, ac = 0.f;
  // Jacobian bookkeeping: each plane crossing with weight w = V_before - V_after
  // contributes d alpha / d(s, p) (Sec. 2.4); sums are kept per axis:
  //   Gs[a] = sum w,   As[a] = sum w * alpha_rel.
  float vprev = 0.f;
  int pa = ea;  // axis of the crossing that starts the current segment (-1: none)
  float Gs0 = 0.f, Gs1 = 0.f, Gs2 = 0.f, As0 = 0.f, As1 = 0.f, As2 = 0.f;

  for (int m = 0; m < nseg; ++m) {
    const float an = fminf(fminf(ax, ay), fminf(az, span));
    const float len = an - ac;
    if (MODE != kBackproject) {
      const float v = Voxel<DT>::load(vd.data, off);
      acc = fmaf(len, v, acc);
      if (MODE == kFwdJac || MODE == kPoseGrad) {
        const float wgt = vprev - v;
        const float wa = wgt * ac;
        if (pa == 0) { Gs0 += wgt; As0 += wa; }
        else if (pa == 1) { Gs1 += wgt; As1 += wa; }
        else if (pa == 2) { Gs2 += wgt; As2 += wa; }
        vprev = v;
      }
    } else {
      if (static_cast<unsigned int>(lin) < nvox) atomicAdd(gvol + lin, gL * len);
    }
    ac = an;
    if (ax <= an) {
      off += sx; kx += 1.f; ax = fmaf(kx, a_step[0], a_first[0]); pa = 0;
      if (MODE == kBackproject) lin += lx;
    } else if (ay <= an) {
      off += sy; ky += 1.f; ay = fmaf(ky, a_step[1], a_first[1]); pa = 1;
      if (MODE == kBackproject) lin += ly;
    } else {
      off += sz; kz += 1.f; az = fmaf(kz, a_step[2], a_first[2]); pa = 2;
      if (MODE == kBackproject) lin += lz;
    }
  }
  res.F = acc;

  if (MODE == kFwdJac || MODE == kPoseGrad) {
    // Exit crossing (weight V_last - 0) unless the exit is the clamp a = 1.
    if (xa == 0) { Gs0 += vprev; As0 += vprev * span; }
    else if (xa == 1) { Gs1 += vprev; As1 += vprev * span; }
    else if (xa == 2) { Gs2 += vprev; As2 += vprev * span; }
    const float Gv[3] = {Gs0, Gs1, Gs2};
    const float Av[3] = {As0, As1, As2};
    float d[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) d[a] = static_cast<float>(g[a]) * vd.delta[a];
    const float L = sqrtf(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]);
    const float FoL = acc / L;
    const float am = static_cast<float>(amin);
    float gt[3], gp[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      if (d[a] != 0.f) {
        const float rd = L / d[a];
        const float Aabs = fmaf(am, Gv[a], Av[a]);  // sum w * alpha (absolute alpha)
        gt[a] = -Gv[a] * rd;                        // dE/dt_a = dE/ds_a + dE/dp_a
        gp[a] = d[a] * FoL - Aabs * rd;             // dE/dp_a
      } else {
        gt[a] = 0.f;
        gp[a] = 0.f;
      }
    }
    const float fw = static_cast<float>(w), fh = static_cast<float>(h);
#pragma unroll
    for (int j = 0; j < 3; ++j) {
      float acc_j = 0.f;
#pragma unroll
      for (int a = 0; a < 3; ++a) {
        const float Dja = fmaf(fh, pg.Hv[j][a], fmaf(fw, pg.Wv[j][a], pg.Q[j][a]));
        acc_j = fmaf(gt[a], pg.S[j][a], acc_j);
        acc_j = fmaf(gp[a], Dja, acc_j);
      }
      res.J[j] = acc_j * vd.out_scale;
    }
#pragma unroll
    for (int a = 0; a < 3; ++a) res.J[3 + a] = gt[a] * vd.out_scale;
  }
  if (MODE == kFwd) {
    float d[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) d[a] = static_cast<float>(g[a]) * vd.delta[a];
    res.F = acc * sqrtf(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]) * vd.out_scale;  // E
  } else if (MODE == kFwdJac || MODE == kPoseGrad) {
    float d[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) d[a] = static_cast<float>(g[a]) * vd.delta[a];
    res.F = acc * sqrtf(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]) * vd.out_scale;
  }
}

template <int MODE, int DT>
__global__ void __launch_bounds__(kThreads) siddon_kernel(VolumeDev vd, DetDev det, const PoseGeom* __restrict__ pgs,
                                                          float* __restrict__ out, float* __restrict__ jac,
                                                          const float* __restrict__ gin,
                                                          float* __restrict__ partials, float* __restrict__ gvol) {
  __shared__ PoseGeom spg;
  __shared__ float red[kThreads / 32][6];
  const int b = blockIdx.z;
  {
    const unsigned int* src = reinterpret_cast<const unsigned int*>(pgs + b);
    unsigned int* dst = reinterpret_cast<unsigned int*>(&spg);
    for (int i = threadIdx.x; i < static_cast<int>(sizeof(PoseGeom) / 4); i += kThreads) dst[i] = src[i];
  }
  __syncthreads();
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int w = blockIdx.x * kTileW + (warp & 3) * kWarpTileW + (lane & 7);
  const int h = blockIdx.y * kTileH + (warp >> 2) * kWarpTileH + (lane >> 3);
  const bool valid = (w < det.W) && (h < det.H);
  const size_t npix = static_cast<size_t>(det.H) * det.W;
  const size_t pix = static_cast<size_t>(h) * det.W + w;

  RayResult r;
  r.nseg = 0;
  float gsc = 0.f;
  if (valid && (MODE == kPoseGrad || MODE == kBackproject)) gsc = gin[b * npix + pix];
  if (valid && !(MODE == kBackproject && gsc == 0.f)) {
    trace_ray<MODE, DT>(vd, spg, h, w, gsc, gvol, r);
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
  } else if (MODE == kPoseGrad) {
    float c[6];
#pragma unroll
    for (int k = 0; k < 6; ++k) c[k] = gsc * r.J[k];
    block_sum6(c, red);
    if (threadIdx.x == 0) {
      const int blk = blockIdx.y * gridDim.x + blockIdx.x;
      const int nblk = gridDim.x * gridDim.y;
#pragma unroll
      for (int k = 0; k < 6; ++k) partials[(static_cast<size_t>(b) * nblk + blk) * 6 + k] = c[k];
    }
  }
}

// Pose gradient from a stored Jacobian: sum g * J over each chunk of pixels.
constexpr int kJacPixPerThread = 8;
__global__ void __launch_bounds__(kThreads) jac_reduce_kernel(const float* __restrict__ gin,
                                                              const float* __restrict__ jac, int npix,
                                                              float* __restrict__ partials) {
  __shared__ float red[kThreads / 32][6];
  const int b = blockIdx.y;
  float c[6] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
  const int base = blockIdx.x * (kThreads * kJacPixPerThread);
  for (int i = 0; i < kJacPixPerThread; ++i) {
    const int p = base + i * kThreads + threadIdx.x;
    if (p < npix) {
      const float gv = __ldg(gin + static_cast<size_t>(b) * npix + p);
#pragma unroll
      for (int k = 0; k < 6; ++k) c[k] = fmaf(gv, __ldg(jac + (static_cast<size_t>(b) * 6 + k) * npix + p), c[k]);
    }
  }
  block_sum6(c, red);
  if (threadIdx.x == 0) {
#pragma unroll
    for (int k = 0; k < 6; ++k) partials[(static_cast<size_t>(b) * gridDim.x + blockIdx.x) * 6 + k] = c[k];
  }
}

// Fixed-order FP64 sum of the per-block partials: one warp per pose.
__global__ void pose_grad_finalize_kernel(const float* __restrict__ partials, int nblk, float* __restrict__ grad) {
  const int b = blockIdx.x, lane = threadIdx.x;
  for (int k = 0; k < 6; ++k) {
    double s = 0.0;
    for (int c = lane; c < nblk; c += 32) s += static_cast<double>(partials[(static_cast<size_t>(b) * nblk + c) * 6 + k]);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (lane == 0) grad[6 * b + k] = static_cast<float>(s);
  }
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

__global__ void ingest_kernel(const void* __restrict__ src, int src_dtype, float mu_water, VolumeDev vd,
                              void* __restrict__ dst, float scale) {
  const int px = vd.n[0] + 2, py = vd.n[1] + 2;
  for (int64_t e = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x; e < vd.elems;
       e += static_cast<int64_t>(gridDim.x) * blockDim.x) {
    const int pk = static_cast<int>(e / (static_cast<int64_t>(px) * py));
    const int rem = static_cast<int>(e - static_cast<int64_t>(pk) * px * py);
    const int pj = rem / px, pi = rem - pj * px;
    const int i = pi - 1, j = pj - 1, k = pk - 1;
    float v = 0.f;
    if (i >= 0 && j >= 0 && k >= 0 && i < vd.n[0] && j < vd.n[1] && k < vd.n[2])
      v = source_value(src, src_dtype, (static_cast<int64_t>(k) * vd.n[1] + j) * vd.n[0] + i, mu_water);
    if (vd.dtype == kF32) {
      static_cast<float*>(dst)[e] = v;
    } else if (vd.dtype == kBF16) {
      static_cast<__nv_bfloat16*>(dst)[e] = __float2bfloat16_rn(v);
    } else {
      static_cast<__half*>(dst)[e] = __float2half_rn(v * scale);
    }
  }
}

int grid_for(int64_t n, int threads) {
  int64_t g = (n + threads - 1) / threads;
  if (g > 152 * 64) g = 152 * 64;
  return static_cast<int>(g < 1 ? 1 : g);
}

template <int MODE>
cudaError_t launch_siddon(const VolumeDev& vd, const DetDev& det, const PoseGeom* pg, int B, float* out, float* jac,
                          const float* gin, float* partials, float* gvol, cudaStream_t stream) {
  dim3 grid((det.W + kTileW - 1) / kTileW, (det.H + kTileH - 1) / kTileH, B);
  switch (vd.dtype) {
    case kF32:
      siddon_kernel<MODE, kF32><<<grid, kThreads, 0, stream>>>(vd, det, pg, out, jac, gin, partials, gvol);
      break;
    case kBF16:
      siddon_kernel<MODE, kBF16><<<grid, kThreads, 0, stream>>>(vd, det, pg, out, jac, gin, partials, gvol);
      break;
    default:
      siddon_kernel<MODE, kF16><<<grid, kThreads, 0, stream>>>(vd, det, pg, out, jac, gin, partials, gvol);
      break;
  }
  return cudaGetLastError();
}

}  // namespace

cudaError_t launch_pose_setup(const float* poses, int B, const DetDev& det, const VolumeDev* vd, PoseGeom* out,
                              cudaStream_t stream) {
  pose_setup_kernel<<<(B + 63) / 64, 64, 0, stream>>>(poses, B, det, *vd, out);
  return cudaGetLastError();
}

cudaError_t launch_ray_setup(const float* poses, int B, const DetDev& det, float* rays, cudaStream_t stream) {
  const int64_t n = static_cast<int64_t>(B) * det.H * det.W;
  ray_setup_kernel<<<static_cast<unsigned int>((n + 255) / 256), 256, 0, stream>>>(poses, B, det, rays);
  return cudaGetLastError();
}

cudaError_t launch_render(const VolumeDev& vd, const DetDev& det, const PoseGeom* pg, int B, float* out, float* jac,
                          cudaStream_t stream) {
  if (jac) return launch_siddon<kFwdJac>(vd, det, pg, B, out, jac, nullptr, nullptr, nullptr, stream);
  return launch_siddon<kFwd>(vd, det, pg, B, out, nullptr, nullptr, nullptr, nullptr, stream);
}

int pose_grad_blocks(const DetDev& det, bool from_jacobian) {
  if (from_jacobian) {
    const int npix = det.H * det.W;
    return (npix + kThreads * kJacPixPerThread - 1) / (kThreads * kJacPixPerThread);
  }
  return ((det.W + kTileW - 1) / kTileW) * ((det.H + kTileH - 1) / kTileH);
}

cudaError_t launch_pose_grad_partials(const VolumeDev& vd, const DetDev& det, const PoseGeom* pg, int B,
                                      const float* grad_drr, const float* jac, float* partials, cudaStream_t stream) {
  if (jac) {
    dim3 grid(pose_grad_blocks(det, true), B);
    jac_reduce_kernel<<<grid, kThreads, 0, stream>>>(grad_drr, jac, det.H * det.W, partials);
    return cudaGetLastError();
  }
  return launch_siddon<kPoseGrad>(vd, det, pg, B, nullptr, nullptr, grad_drr, partials, nullptr, stream);
}

cudaError_t launch_count_segments(const VolumeDev& vd, const DetDev& det, const PoseGeom* pg, int B, int* counts,
                                  cudaStream_t stream) {
  return launch_siddon<kCount>(vd, det, pg, B, reinterpret_cast<float*>(counts), nullptr, nullptr, nullptr, nullptr,
                               stream);
}

cudaError_t launch_pose_grad_finalize(const float* partials, int B, int nblk, float* grad_pose, cudaStream_t stream) {
  pose_grad_finalize_kernel<<<B, 32, 0, stream>>>(partials, nblk, grad_pose);
  return cudaGetLastError();
}

cudaError_t launch_backproject(const VolumeDev& vd, const DetDev& det, const PoseGeom* pg, int B,
                               const float* grad_drr, float* grad_vol, cudaStream_t stream) {
  return launch_siddon<kBackproject>(vd, det, pg, B, nullptr, nullptr, grad_drr, nullptr, grad_vol, stream);
}

cudaError_t launch_abs_max(const void* src, int src_dtype, int64_t count, float mu_water, unsigned int* out_bits,
                           cudaStream_t stream) {
  abs_max_kernel<<<grid_for(count, 256), 256, 0, stream>>>(src, src_dtype, count, mu_water, out_bits);
  return cudaGetLastError();
}

cudaError_t launch_ingest(const void* src, int src_dtype, float mu_water, const VolumeDev& vd, void* dst, float scale,
                          cudaStream_t stream) {
  ingest_kernel<<<grid_for(vd.elems, 256), 256, 0, stream>>>(src, src_dtype, mu_water, vd, dst, scale);
  return cudaGetLastError();
}

}  // namespace drr
