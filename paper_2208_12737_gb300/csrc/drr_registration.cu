// Registration support (Sec. 3.2 of the paper: slice-to-volume registration by
// gradient descent on the negative zero-normalised cross-correlation between a
// moving DRR and a fixed image): the ZNCC loss with its image gradient, and an
// Adam step on the pose parameters.
#include <cuda_runtime.h>

#include "drr.h"
#include "drr_internal.cuh"

namespace {

constexpr int kZThreads = 512;

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Block-wide sums of n doubles; every thread gets the totals.
template <int N>
__device__ __forceinline__ void block_sums(double (&v)[N], double (*sm)[N]) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int k = 0; k < N; ++k) v[k] = warp_sum(v[k]);
  if (lane == 0) {
#pragma unroll
    for (int k = 0; k < N; ++k) sm[warp][k] = v[k];
  }
  __syncthreads();
#pragma unroll
  for (int k = 0; k < N; ++k) {
    double t = 0.0;
    for (int q = 0; q < kZThreads / 32; ++q) t += sm[q][k];
    v[k] = t;
  }
  __syncthreads();
}

// One block per image pair.  With population statistics and c = I - mean(I),
// s = sqrt(mean(c^2)), I^ = c / (s + eps) (same for the fixed image F):
//   zncc = mean(I^ F^),  loss = -zncc,
//   d zncc / dI_j = (F^_j - zncc c_j / s) / (N (s + eps)).
// fixed_stride: elements between consecutive fixed images (0: one fixed image for all).
__global__ void __launch_bounds__(kZThreads) zncc_kernel(const float* __restrict__ moving,
                                                         const float* __restrict__ fixed, size_t fixed_stride,
                                                         int npix, float eps, float* __restrict__ loss,
                                                         float* __restrict__ grad) {
  __shared__ double sm[kZThreads / 32][5];
  const size_t base = static_cast<size_t>(blockIdx.x) * npix;
  const float* I = moving + base;
  const float* F = fixed + static_cast<size_t>(blockIdx.x) * fixed_stride;
  double v[5] = {0.0, 0.0, 0.0, 0.0, 0.0};  // sum I, sum I^2, sum F, sum F^2, sum I F
  for (int i = threadIdx.x; i < npix; i += kZThreads) {
    const double a = I[i], b = F[i];
    v[0] += a;
    v[1] += a * a;
    v[2] += b;
    v[3] += b * b;
    v[4] += a * b;
  }
  block_sums<5>(v, sm);
  const double n = static_cast<double>(npix);
  const double mi = v[0] / n, mf = v[2] / n;
  const double si = sqrt(fmax(v[1] / n - mi * mi, 0.0)), sf = sqrt(fmax(v[3] / n - mf * mf, 0.0));
  const double cov = v[4] / n - mi * mf;
  const double zncc = cov / ((si + eps) * (sf + eps));
  if (threadIdx.x == 0 && loss) loss[blockIdx.x] = static_cast<float>(-zncc);
  if (!grad) return;
  const double a_f = 1.0 / (sf + eps);
  const double k1 = -1.0 / (n * (si + eps));            // d loss = -d zncc
  const double k2 = si > 0.0 ? zncc / si : 0.0;
  for (int i = threadIdx.x; i < npix; i += kZThreads) {
    const double fh = (static_cast<double>(F[i]) - mf) * a_f;
    const double c = static_cast<double>(I[i]) - mi;
    grad[base + i] = static_cast<float>(k1 * (fh - k2 * c));
  }
}

// Adam on the six pose parameters of each of B poses (rotations and
// translations have separate step sizes, Sec. 3.2 uses separate rates too).
__global__ void adam_kernel(float* __restrict__ params, const float* __restrict__ grads, float* __restrict__ m,
                            float* __restrict__ v, int n, int step, float lr_rot, float lr_trans, float b1, float b2,
                            float eps) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const float g = grads[i];
  const float mi = b1 * m[i] + (1.f - b1) * g;
  const float vi = b2 * v[i] + (1.f - b2) * g * g;
  m[i] = mi;
  v[i] = vi;
  const float mh = mi / (1.f - powf(b1, static_cast<float>(step)));
  const float vh = vi / (1.f - powf(b2, static_cast<float>(step)));
  const float lr = (i % 6) < 3 ? lr_rot : lr_trans;
  params[i] -= lr * mh / (sqrtf(vh) + eps);
}

}  // namespace

cudaError_t drr::launch_zncc(const float* moving, const float* fixed, size_t fixed_stride, int B, int npix, float eps,
                             float* loss, float* grad, cudaStream_t stream) {
  zncc_kernel<<<B, kZThreads, 0, stream>>>(moving, fixed, fixed_stride, npix, eps, loss, grad);
  return cudaGetLastError();
}

extern "C" drr_status drr_zncc(const float* moving_dev, const float* fixed_dev, int32_t B, int32_t npix,
                               float eps, float* loss_dev, float* grad_dev, void* cuda_stream) {
  if (B <= 0 || npix <= 0) return drr::set_error(DRR_ERR_INVALID, "B and npix must be positive");
  if (!moving_dev || !fixed_dev || (!loss_dev && !grad_dev)) return drr::set_error(DRR_ERR_INVALID, "NULL pointer");
  if (!(eps >= 0.f)) return drr::set_error(DRR_ERR_INVALID, "eps must be >= 0");
  const int dev = drr::current_device();
  if (drr_status s = drr::device_view(moving_dev, dev, true, "moving", &moving_dev)) return s;
  if (drr_status s = drr::device_view(fixed_dev, dev, true, "fixed", &fixed_dev)) return s;
  if (loss_dev) {
    if (drr_status s = drr::device_view(loss_dev, dev, true, "loss", &loss_dev)) return s;
  }
  if (grad_dev) {
    if (drr_status s = drr::device_view(grad_dev, dev, true, "grad", &grad_dev)) return s;
  }
  cudaError_t e = drr::launch_zncc(moving_dev, fixed_dev, static_cast<size_t>(npix), B, npix, eps, loss_dev, grad_dev,
                                   static_cast<cudaStream_t>(cuda_stream));
  if (e != cudaSuccess) return drr::cuda_error(e, "zncc launch");
  drr::count_launches(1);
  return DRR_OK;
}

extern "C" drr_status drr_adam_step(float* params_dev, const float* grads_dev, float* m_dev, float* v_dev, int32_t B,
                                    int32_t step, float lr_rot, float lr_trans, float beta1, float beta2, float eps,
                                    void* cuda_stream) {
  if (B <= 0 || step <= 0) return drr::set_error(DRR_ERR_INVALID, "B and step must be positive");
  if (!params_dev || !grads_dev || !m_dev || !v_dev) return drr::set_error(DRR_ERR_INVALID, "NULL pointer");
  const int dev = drr::current_device();
  if (drr_status s = drr::device_view(params_dev, dev, true, "params", &params_dev)) return s;
  if (drr_status s = drr::device_view(grads_dev, dev, true, "grads", &grads_dev)) return s;
  if (drr_status s = drr::device_view(m_dev, dev, true, "m", &m_dev)) return s;
  if (drr_status s = drr::device_view(v_dev, dev, true, "v", &v_dev)) return s;
  const int n = 6 * B;
  adam_kernel<<<(n + 255) / 256, 256, 0, static_cast<cudaStream_t>(cuda_stream)>>>(
      params_dev, grads_dev, m_dev, v_dev, n, step, lr_rot, lr_trans, beta1, beta2, eps);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return drr::cuda_error(e, "adam launch");
  drr::count_launches(1);
  return DRR_OK;
}
