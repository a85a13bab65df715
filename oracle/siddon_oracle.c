/*
 * FP64 CPU oracle for digitally reconstructed radiographs by Siddon's method
 * (Gopalakrishnan & Golland, "Fast Auto-Differentiable Digitally Reconstructed
 * Radiographs", arXiv 2208.12737).
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the slow, plain reference that the
 * CUDA path is checked against.  Only the test-suite, the smoke check and the
 * CPU-baseline leg of the benchmark may load it.  It shares no code, header,
 * table or helper with the CUDA library, and the library never calls it.
 *
 * Everything here is double precision and follows the paper's definitions
 * literally, with no blocking, fusion or reordering:
 *   - Eq. (1)/(2): E = |p - s| * sum_m (alpha_{m+1} - alpha_m) V[voxel at midpoint]
 *   - Eq. (3):     alpha_x(i) = (b_x + i dX - s_x) / (p_x - s_x)   (same for y, z)
 *   - Sec. 2.3:    alpha_min / alpha_max = max of per-axis minima / min of maxima
 *   - Eq. (4):     alpha = sort(alpha_x, alpha_y, alpha_z)
 *   - Sec. 2.4:    source on a sphere of radius rho = SDR/2, detector tangent
 *                  at the antipode, roll about the x axis, translation added
 *                  to source and detector; gradient = derivative of the above
 *                  with the voxel lookup held fixed (what autograd through
 *                  Eq. 2-4 yields).
 * Readings where the paper is silent (all listed in the design notes):
 *   - volume centred at the world origin: b = -(n * delta) / 2 per axis;
 *   - voxel (i,j,k) is the half-open box [b + i delta, b + (i+1) delta);
 *   - alpha_min / alpha_max are clamped to [0, 1] (Siddon's original);
 *   - an axis with p_a == s_a contributes no crossings and no clip bound when
 *     b_a <= s_a < b_a + n_a delta_a, otherwise the ray misses;
 *   - pose eta = (rz, ry, rx, tx, ty, tz), R = Rz(rz) Ry(ry) Rx(rx),
 *     s = R (rho,0,0) + t, p = R (-rho, (w-(W-1)/2) dw, (h-(H-1)/2) dh) + t;
 *   - HU -> attenuation: mu = max(0, mu_water (1 + HU/1000)).
 *
 * Volumes are float32 arrays of shape (nz, ny, nx), x fastest.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

/* ------------------------------------------------------------------------- */
/* Pose -> rotation (Sec. 2.4).                                              */
/* ------------------------------------------------------------------------- */

static void mat3_mul(const double A[9], const double B[9], double C[9]) {
  for (int r = 0; r < 3; ++r)
    for (int c = 0; c < 3; ++c) {
      double acc = 0.0;
      for (int k = 0; k < 3; ++k) acc += A[3 * r + k] * B[3 * k + c];
      C[3 * r + c] = acc;
    }
}

static void mat3_vec(const double A[9], const double x[3], double y[3]) {
  for (int r = 0; r < 3; ++r) y[r] = A[3 * r] * x[0] + A[3 * r + 1] * x[1] + A[3 * r + 2] * x[2];
}

/* R = Rz(eta0) Ry(eta1) Rx(eta2) (row-major), and dR[j] = dR / d eta_j. */
void oracle_pose_matrix(const double eta[3], double R[9], double dR[27]) {
  double cz = cos(eta[0]), sz = sin(eta[0]);
  double cy = cos(eta[1]), sy = sin(eta[1]);
  double cx = cos(eta[2]), sx = sin(eta[2]);
  double Rz[9] = {cz, -sz, 0, sz, cz, 0, 0, 0, 1};
  double Ry[9] = {cy, 0, sy, 0, 1, 0, -sy, 0, cy};
  double Rx[9] = {1, 0, 0, 0, cx, -sx, 0, sx, cx};
  double dRz[9] = {-sz, -cz, 0, cz, -sz, 0, 0, 0, 0};
  double dRy[9] = {-sy, 0, cy, 0, 0, 0, -cy, 0, -sy};
  double dRx[9] = {0, 0, 0, 0, -sx, -cx, 0, cx, -sx};
  double T[9];
  mat3_mul(Rz, Ry, T);
  mat3_mul(T, Rx, R);
  if (dR) {
    double U[9];
    mat3_mul(dRz, Ry, U);
    mat3_mul(U, Rx, dR + 0);
    mat3_mul(Rz, dRy, U);
    mat3_mul(U, Rx, dR + 9);
    mat3_mul(T, dRx, dR + 18);
  }
}

/* Canonical (pose-free) source and pixel centre, Sec. 2.4. */
static void canonical_points(double sdr, int32_t H, int32_t W, double dh, double dw, int32_t h,
                             int32_t w, double sc[3], double pc[3]) {
  double rho = 0.5 * sdr;
  sc[0] = rho;
  sc[1] = 0.0;
  sc[2] = 0.0;
  pc[0] = -rho;
  pc[1] = ((double)w - 0.5 * (double)(W - 1)) * dw;
  pc[2] = ((double)h - 0.5 * (double)(H - 1)) * dh;
}

/* Source s and pixel centre p in world coordinates for one pose. */
void oracle_ray_endpoints(const double pose[6], double sdr, int32_t H, int32_t W, double dh,
                          double dw, int32_t h, int32_t w, double s[3], double p[3]) {
  double R[9], sc[3], pc[3];
  oracle_pose_matrix(pose, R, NULL);
  canonical_points(sdr, H, W, dh, dw, h, w, sc, pc);
  mat3_vec(R, sc, s);
  mat3_vec(R, pc, p);
  for (int a = 0; a < 3; ++a) {
    s[a] += pose[3 + a];
    p[a] += pose[3 + a];
  }
}

/* ------------------------------------------------------------------------- */
/* Siddon's method, Eq. (2)-(4).                                             */
/* ------------------------------------------------------------------------- */

typedef struct {
  double alpha;
  int axis; /* axis whose plane this is, or -1 for a clamp at alpha = 0 or 1 */
} crossing_t;

static int cmp_crossing(const void* a, const void* b) {
  double x = ((const crossing_t*)a)->alpha, y = ((const crossing_t*)b)->alpha;
  return (x < y) ? -1 : (x > y) ? 1 : 0;
}

static double voxel_value(const int32_t n[3], const float* vol, const int64_t idx[3]) {
  if (!vol) return 0.0;
  for (int a = 0; a < 3; ++a)
    if (idx[a] < 0 || idx[a] >= n[a]) return 0.0;
  return (double)vol[(idx[2] * n[1] + idx[1]) * (int64_t)n[0] + idx[0]];
}

/*
 * Line integral E for the segment s -> p, and optionally dE/ds, dE/dp.
 * scratch must hold n[0] + n[1] + n[2] + 5 crossings.
 * If seg_cb is non-NULL it is called for every segment with (voxel index,
 * segment length in alpha) -- used by the back-projector.
 */
typedef void (*seg_cb_t)(void* ctx, const int64_t idx[3], double len_alpha);

static double siddon_ray(const int32_t n[3], const double delta[3], const float* vol,
                         const double s[3], const double p[3], double gs[3], double gp[3],
                         crossing_t* list, seg_cb_t cb, void* cb_ctx) {
  double b[3], d[3];
  if (gs)
    for (int a = 0; a < 3; ++a) gs[a] = gp[a] = 0.0;
  for (int a = 0; a < 3; ++a) {
    b[a] = -0.5 * (double)n[a] * delta[a];
    d[a] = p[a] - s[a];
  }
  /* alpha_min / alpha_max (Sec. 2.3), clamped to [0, 1]. */
  double amin = 0.0, amax = 1.0;
  int ax_min = -1, ax_max = -1;
  for (int a = 0; a < 3; ++a) {
    if (d[a] != 0.0) {
      double a0 = (b[a] - s[a]) / d[a];
      double an = (b[a] + (double)n[a] * delta[a] - s[a]) / d[a];
      double lo = fmin(a0, an), hi = fmax(a0, an);
      if (lo > amin) {
        amin = lo;
        ax_min = a;
      }
      if (hi < amax) {
        amax = hi;
        ax_max = a;
      }
    } else if (!(s[a] >= b[a] && s[a] < b[a] + (double)n[a] * delta[a])) {
      return 0.0;
    }
  }
  if (!(amin < amax)) return 0.0;

  /* All plane crossings strictly inside (alpha_min, alpha_max), Eq. (3). */
  int M = 0;
  list[M].alpha = amin;
  list[M++].axis = ax_min;
  for (int a = 0; a < 3; ++a) {
    if (d[a] == 0.0) continue;
    for (int32_t i = 0; i <= n[a]; ++i) {
      double al = (b[a] + (double)i * delta[a] - s[a]) / d[a];
      if (al > amin && al < amax) {
        list[M].alpha = al;
        list[M++].axis = a;
      }
    }
  }
  list[M].alpha = amax;
  list[M++].axis = ax_max;
  /* Eq. (4): sort. */
  qsort(list, (size_t)M, sizeof(crossing_t), cmp_crossing);

  /* Eq. (2): sum of segment length times the voxel at the segment midpoint. */
  double F = 0.0;
  double v_prev = 0.0;
  double L = sqrt(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]);
  double dFds[3] = {0, 0, 0}, dFdp[3] = {0, 0, 0};
  for (int m = 0; m + 1 < M; ++m) {
    double a0 = list[m].alpha, a1 = list[m + 1].alpha;
    double mid = 0.5 * (a0 + a1);
    int64_t idx[3];
    for (int a = 0; a < 3; ++a) idx[a] = (int64_t)floor((s[a] + mid * d[a] - b[a]) / delta[a]);
    double v = voxel_value(n, vol, idx);
    F += (a1 - a0) * v;
    if (cb) cb(cb_ctx, idx, a1 - a0);
    if (gs) {
      /* crossing m separates segment m-1 (value v_prev) from segment m (v). */
      int ax = list[m].axis;
      if (ax >= 0) {
        double wk = v_prev - v;
        dFds[ax] += wk * (a0 - 1.0) / d[ax];
        dFdp[ax] += -wk * a0 / d[ax];
      }
    }
    v_prev = v;
  }
  if (gs) {
    int ax = list[M - 1].axis;
    if (ax >= 0) {
      double wk = v_prev; /* exit: value before minus zero after */
      double a0 = list[M - 1].alpha;
      dFds[ax] += wk * (a0 - 1.0) / d[ax];
      dFdp[ax] += -wk * a0 / d[ax];
    }
    for (int a = 0; a < 3; ++a) {
      gs[a] = -d[a] * F / L + L * dFds[a];
      gp[a] = d[a] * F / L + L * dFdp[a];
    }
  }
  return L * F;
}

static crossing_t* alloc_list(const int32_t n[3]) {
  return (crossing_t*)malloc(sizeof(crossing_t) * (size_t)(n[0] + n[1] + n[2] + 8));
}

/* Single ray: E and (optionally) dE/ds, dE/dp. */
double oracle_siddon_ray(const int32_t n[3], const double delta[3], const float* vol,
                         const double s[3], const double p[3], double gs[3], double gp[3]) {
  crossing_t* list = alloc_list(n);
  double E = siddon_ray(n, delta, vol, s, p, gs, gp, list, NULL, NULL);
  free(list);
  return E;
}

/* Sum of segment lengths (alpha units) along the ray, for the sum-of-lengths pin. */
static void add_len(void* ctx, const int64_t idx[3], double len) {
  (void)idx;
  *(double*)ctx += len;
}
double oracle_siddon_total_length(const int32_t n[3], const double delta[3], const float* vol,
                                  const double s[3], const double p[3]) {
  crossing_t* list = alloc_list(n);
  double total = 0.0;
  siddon_ray(n, delta, vol, s, p, NULL, NULL, list, add_len, &total);
  free(list);
  double d2 = 0.0;
  for (int a = 0; a < 3; ++a) d2 += (p[a] - s[a]) * (p[a] - s[a]);
  return total * sqrt(d2);
}

/* ------------------------------------------------------------------------- */
/* Independent checks of the line integral (used to pin the oracle).         */
/* ------------------------------------------------------------------------- */

/* Exact brute force: sum over every voxel of V times the length of the
 * segment s->p clipped to that voxel's box (slab method per voxel). */
double oracle_brute_ray(const int32_t n[3], const double delta[3], const float* vol,
                        const double s[3], const double p[3]) {
  double b[3], d[3];
  for (int a = 0; a < 3; ++a) {
    b[a] = -0.5 * (double)n[a] * delta[a];
    d[a] = p[a] - s[a];
  }
  double L = sqrt(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]);
  double acc = 0.0;
  for (int32_t k = 0; k < n[2]; ++k)
    for (int32_t j = 0; j < n[1]; ++j)
      for (int32_t i = 0; i < n[0]; ++i) {
        double v = vol[((int64_t)k * n[1] + j) * n[0] + i];
        if (v == 0.0) continue;
        int32_t id[3] = {i, j, k};
        double t_lo = 0.0, t_hi = 1.0;
        int empty = 0;
        for (int a = 0; a < 3 && !empty; ++a) {
          double lo = b[a] + id[a] * delta[a], hi = b[a] + (id[a] + 1) * delta[a];
          if (d[a] == 0.0) {
            if (!(s[a] >= lo && s[a] < hi)) empty = 1;
          } else {
            double t0 = (lo - s[a]) / d[a], t1 = (hi - s[a]) / d[a];
            t_lo = fmax(t_lo, fmin(t0, t1));
            t_hi = fmin(t_hi, fmax(t0, t1));
          }
        }
        if (!empty && t_hi > t_lo) acc += v * (t_hi - t_lo);
      }
  return L * acc;
}

/* Midpoint-rule sampling of Eq. (1) with N samples (converges as O(1/N)). */
double oracle_sample_ray(const int32_t n[3], const double delta[3], const float* vol,
                         const double s[3], const double p[3], int64_t N) {
  double b[3], d[3];
  for (int a = 0; a < 3; ++a) {
    b[a] = -0.5 * (double)n[a] * delta[a];
    d[a] = p[a] - s[a];
  }
  double L = sqrt(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]);
  double acc = 0.0;
  for (int64_t q = 0; q < N; ++q) {
    double al = ((double)q + 0.5) / (double)N;
    int64_t idx[3];
    for (int a = 0; a < 3; ++a) idx[a] = (int64_t)floor((s[a] + al * d[a] - b[a]) / delta[a]);
    acc += voxel_value(n, vol, idx);
  }
  return L * acc / (double)N;
}

/* ------------------------------------------------------------------------- */
/* Whole-detector rendering and the pose gradient.                           */
/* ------------------------------------------------------------------------- */

/*
 * out[b][q] = E for pose b and pixel pix[q] (flat h*W + w); pix == NULL means
 * every pixel (npix = H*W).  jac (optional) [b][q][6] = dE/d(rz, ry, rx, tx, ty, tz).
 * geo (optional) [b][q][3] = dE/d(sdr, dh, dw), the detector parameters (Sec. 3.2
 * notes the generator also differentiates with respect to the source-to-detector
 * distance 2 rho and the pixel spacing): with s = R (rho,0,0) + t, rho = sdr/2, and
 * p = R (-rho, (w-(W-1)/2) dw, (h-(H-1)/2) dh) + t, by the chain rule through s and p.
 */
int oracle_render(const int32_t n[3], const double delta[3], const float* vol, double sdr,
                  int32_t H, int32_t W, double dh, double dw, const float* poses, int32_t B,
                  const int64_t* pix, int64_t npix, double* out, double* jac, double* geo,
                  int32_t nthreads) {
  if (!pix) npix = (int64_t)H * W;
  int64_t total = (int64_t)B * npix;
#ifdef _OPENMP
  if (nthreads > 0) omp_set_num_threads(nthreads);
#else
  (void)nthreads;
#endif
#pragma omp parallel
  {
    crossing_t* list = alloc_list(n);
#pragma omp for schedule(dynamic, 64)
    for (int64_t r = 0; r < total; ++r) {
      int32_t bi = (int32_t)(r / npix);
      int64_t q = r % npix;
      int64_t flat = pix ? pix[q] : q;
      int32_t h = (int32_t)(flat / W), w = (int32_t)(flat % W);
      double pose[6];
      for (int k = 0; k < 6; ++k) pose[k] = (double)poses[6 * bi + k];
      double R[9], dR[27], sc[3], pc[3], s[3], p[3];
      oracle_pose_matrix(pose, R, dR);
      canonical_points(sdr, H, W, dh, dw, h, w, sc, pc);
      mat3_vec(R, sc, s);
      mat3_vec(R, pc, p);
      for (int a = 0; a < 3; ++a) {
        s[a] += pose[3 + a];
        p[a] += pose[3 + a];
      }
      double gs[3], gp[3];
      const int want = jac || geo;
      double E = siddon_ray(n, delta, vol, s, p, want ? gs : NULL, want ? gp : NULL, list, NULL,
                            NULL);
      out[r] = E;
      if (geo) {
        /* ds/dsdr = R (1/2, 0, 0); dp/dsdr = R (-1/2, 0, 0); dp/ddh = R (0, 0, h-(H-1)/2);
           dp/ddw = R (0, w-(W-1)/2, 0) */
        const double e_sdr_s[3] = {0.5, 0.0, 0.0}, e_sdr_p[3] = {-0.5, 0.0, 0.0};
        const double e_dh[3] = {0.0, 0.0, (double)h - 0.5 * (double)(H - 1)};
        const double e_dw[3] = {0.0, (double)w - 0.5 * (double)(W - 1), 0.0};
        double vs[3], vp[3], vh[3], vw[3];
        mat3_vec(R, e_sdr_s, vs);
        mat3_vec(R, e_sdr_p, vp);
        mat3_vec(R, e_dh, vh);
        mat3_vec(R, e_dw, vw);
        double* G = geo + 3 * r;
        G[0] = gs[0] * vs[0] + gs[1] * vs[1] + gs[2] * vs[2] + gp[0] * vp[0] + gp[1] * vp[1] +
               gp[2] * vp[2];
        G[1] = gp[0] * vh[0] + gp[1] * vh[1] + gp[2] * vh[2];
        G[2] = gp[0] * vw[0] + gp[1] * vw[1] + gp[2] * vw[2];
      }
      if (jac) {
        double* J = jac + 6 * r;
        for (int j = 0; j < 3; ++j) {
          double vs[3], vp[3];
          mat3_vec(dR + 9 * j, sc, vs);
          mat3_vec(dR + 9 * j, pc, vp);
          J[j] = gs[0] * vs[0] + gs[1] * vs[1] + gs[2] * vs[2] + gp[0] * vp[0] +
                 gp[1] * vp[1] + gp[2] * vp[2];
        }
        for (int a = 0; a < 3; ++a) J[3 + a] = gs[a] + gp[a];
      }
    }
    free(list);
  }
  return 0;
}

/* grad_pose[b][k] = sum over all pixels of grad_out[b][h][w] * dE/d eta_k. */
int oracle_pose_grad(const int32_t n[3], const double delta[3], const float* vol, double sdr,
                     int32_t H, int32_t W, double dh, double dw, const float* poses, int32_t B,
                     const double* grad_out, double* grad_pose, int32_t nthreads) {
  int64_t npix = (int64_t)H * W;
  double* E = (double*)malloc(sizeof(double) * (size_t)(B * npix));
  double* J = (double*)malloc(sizeof(double) * 6 * (size_t)(B * npix));
  if (!E || !J) {
    free(E);
    free(J);
    return 1;
  }
  oracle_render(n, delta, vol, sdr, H, W, dh, dw, poses, B, NULL, npix, E, J, NULL, nthreads);
  for (int32_t b = 0; b < B; ++b)
    for (int k = 0; k < 6; ++k) {
      double acc = 0.0;
      for (int64_t q = 0; q < npix; ++q)
        acc += grad_out[b * npix + q] * J[6 * (b * npix + q) + k];
      grad_pose[6 * b + k] = acc;
    }
  free(E);
  free(J);
  return 0;
}

/* Number of segments (consecutive pairs of the sorted list of Eq. 4) per ray,
 * zero-length ones included; 0 when the ray misses. out[b][q] like oracle_render. */
static void count_one(void* ctx, const int64_t idx[3], double len) {
  (void)idx;
  (void)len;
  *(int32_t*)ctx += 1;
}
int oracle_count_segments(const int32_t n[3], const double delta[3], double sdr, int32_t H, int32_t W, double dh,
                          double dw, const float* poses, int32_t B, const int64_t* pix, int64_t npix, int32_t* out) {
  if (!pix) npix = (int64_t)H * W;
  crossing_t* list = alloc_list(n);
  for (int32_t bi = 0; bi < B; ++bi) {
    double pose[6];
    for (int k = 0; k < 6; ++k) pose[k] = (double)poses[6 * bi + k];
    for (int64_t q = 0; q < npix; ++q) {
      int64_t flat = pix ? pix[q] : q;
      double s[3], p[3];
      oracle_ray_endpoints(pose, sdr, H, W, dh, dw, (int32_t)(flat / W), (int32_t)(flat % W), s, p);
      int32_t c = 0;
      siddon_ray(n, delta, NULL, s, p, NULL, NULL, list, count_one, &c);
      out[(int64_t)bi * npix + q] = c;
    }
  }
  free(list);
  return 0;
}

/* ------------------------------------------------------------------------- */
/* Volume adjoint: the transpose of the linear map V -> E (back-projection). */
/* ------------------------------------------------------------------------- */

typedef struct {
  const int32_t* n;
  double* grad;
  double weight;
} bp_ctx_t;

static void bp_add(void* ctx, const int64_t idx[3], double len) {
  bp_ctx_t* c = (bp_ctx_t*)ctx;
  for (int a = 0; a < 3; ++a)
    if (idx[a] < 0 || idx[a] >= c->n[a]) return;
  c->grad[(idx[2] * c->n[1] + idx[1]) * (int64_t)c->n[0] + idx[0]] += c->weight * len;
}

/* grad_vol[z][y][x] += sum over rays of grad_out * |p - s| * segment length. Serial. */
int oracle_backproject(const int32_t n[3], const double delta[3], double sdr, int32_t H,
                       int32_t W, double dh, double dw, const float* poses, int32_t B,
                       const double* grad_out, double* grad_vol) {
  crossing_t* list = alloc_list(n);
  int64_t nvox = (int64_t)n[0] * n[1] * n[2];
  float* ones = (float*)malloc(sizeof(float) * (size_t)nvox);
  for (int64_t i = 0; i < nvox; ++i) ones[i] = 1.0f;
  for (int32_t bi = 0; bi < B; ++bi) {
    double pose[6];
    for (int k = 0; k < 6; ++k) pose[k] = (double)poses[6 * bi + k];
    for (int32_t h = 0; h < H; ++h)
      for (int32_t w = 0; w < W; ++w) {
        double s[3], p[3];
        oracle_ray_endpoints(pose, sdr, H, W, dh, dw, h, w, s, p);
        double L = sqrt((p[0] - s[0]) * (p[0] - s[0]) + (p[1] - s[1]) * (p[1] - s[1]) +
                        (p[2] - s[2]) * (p[2] - s[2]));
        bp_ctx_t ctx = {n, grad_vol, grad_out[((int64_t)bi * H + h) * W + w] * L};
        siddon_ray(n, delta, ones, s, p, NULL, NULL, list, bp_add, &ctx);
      }
  }
  free(ones);
  free(list);
  return 0;
}

/* The transpose of V -> E for one ray s -> p: grad_vol[z][y][x] += g * |p - s| *
 * (length in alpha of each Siddon segment in that voxel). */
int oracle_backproject_ray(const int32_t n[3], const double delta[3], const double s[3], const double p[3],
                           double g, double* grad_vol) {
  crossing_t* list = alloc_list(n);
  const double L = sqrt((p[0] - s[0]) * (p[0] - s[0]) + (p[1] - s[1]) * (p[1] - s[1]) + (p[2] - s[2]) * (p[2] - s[2]));
  bp_ctx_t ctx = {n, grad_vol, g * L};
  siddon_ray(n, delta, NULL, s, p, NULL, NULL, list, bp_add, &ctx);
  free(list);
  return 0;
}

/* The transpose of V -> E at selected voxels, straight from its definition
 * (Eq. 1 with a piecewise-constant volume is linear in V): the adjoint at voxel
 * v is the sum over all rays of g * |p - s| * (the length, in alpha, of the
 * segment s->p clipped to v's box), the clip by the slab method as in
 * oracle_brute_ray.  Also returns, per voxel, the same sum with |g|: the scale
 * of the rounding error of any sum of these terms.  vox holds linear indices
 * i + nx (j + ny k).  OpenMP over the selected voxels. */
int oracle_voxel_adjoint(const int32_t n[3], const double delta[3], double sdr, int32_t H, int32_t W,
                         double dh, double dw, const float* poses, int32_t B, const double* grad_out,
                         const int64_t* vox, int64_t nsel, double* out, double* out_abs) {
  const int64_t nray = (int64_t)B * H * W;
  double* S = (double*)malloc(sizeof(double) * 3 * (size_t)nray);
  double* Dv = (double*)malloc(sizeof(double) * 3 * (size_t)nray);
  double* L = (double*)malloc(sizeof(double) * (size_t)nray);
  if (!S || !Dv || !L) {
    free(S);
    free(Dv);
    free(L);
    return -1;
  }
  for (int32_t bi = 0; bi < B; ++bi) {
    double pose[6];
    for (int k = 0; k < 6; ++k) pose[k] = (double)poses[6 * bi + k];
    for (int32_t h = 0; h < H; ++h)
      for (int32_t w = 0; w < W; ++w) {
        const int64_t r = ((int64_t)bi * H + h) * W + w;
        double s[3], p[3];
        oracle_ray_endpoints(pose, sdr, H, W, dh, dw, h, w, s, p);
        for (int a = 0; a < 3; ++a) {
          S[3 * r + a] = s[a];
          Dv[3 * r + a] = p[a] - s[a];
        }
        L[r] = sqrt(Dv[3 * r] * Dv[3 * r] + Dv[3 * r + 1] * Dv[3 * r + 1] + Dv[3 * r + 2] * Dv[3 * r + 2]);
      }
  }
#pragma omp parallel for schedule(dynamic, 1)
  for (int64_t q = 0; q < nsel; ++q) {
    const int64_t v = vox[q];
    const int64_t id[3] = {v % n[0], (v / n[0]) % n[1], v / ((int64_t)n[0] * n[1])};
    double lo[3], hi[3];
    for (int a = 0; a < 3; ++a) {
      const double b = -0.5 * (double)n[a] * delta[a];
      lo[a] = b + (double)id[a] * delta[a];
      hi[a] = b + (double)(id[a] + 1) * delta[a];
    }
    double acc = 0.0, acc_abs = 0.0;
    for (int64_t r = 0; r < nray; ++r) {
      const double* s = S + 3 * r;
      const double* d = Dv + 3 * r;
      double t_lo = 0.0, t_hi = 1.0;
      int empty = 0;
      for (int a = 0; a < 3 && !empty; ++a) {
        if (d[a] == 0.0) {
          if (!(s[a] >= lo[a] && s[a] < hi[a])) empty = 1;
        } else {
          const double t0 = (lo[a] - s[a]) / d[a], t1 = (hi[a] - s[a]) / d[a];
          t_lo = fmax(t_lo, fmin(t0, t1));
          t_hi = fmin(t_hi, fmax(t0, t1));
        }
      }
      if (!empty && t_hi > t_lo) {
        const double term = L[r] * (t_hi - t_lo);
        acc += grad_out[r] * term;
        acc_abs += fabs(grad_out[r]) * term;
      }
    }
    out[q] = acc;
    out_abs[q] = acc_abs;
  }
  free(S);
  free(Dv);
  free(L);
  return 0;
}

/* ------------------------------------------------------------------------- */
/* Volume ingest: HU -> attenuation, and 16-bit storage rounding.            */
/* ------------------------------------------------------------------------- */

/* mu = max(0, mu_water * (1 + HU / 1000)). */
void oracle_hu_to_mu(const int16_t* hu, int64_t count, double mu_water, double* out) {
  for (int64_t i = 0; i < count; ++i) {
    double mu = mu_water * (1.0 + (double)hu[i] / 1000.0);
    out[i] = mu > 0.0 ? mu : 0.0;
  }
}

/* Round float32 values to bfloat16 (round to nearest, ties to even), returned as float32. */
void oracle_round_bf16(const float* in, int64_t count, float* out) {
  for (int64_t i = 0; i < count; ++i) {
    uint32_t u;
    memcpy(&u, &in[i], 4);
    if ((u & 0x7F800000u) == 0x7F800000u) { /* inf / nan: truncate */
      u &= 0xFFFF0000u;
    } else {
      uint32_t lower = u & 0xFFFFu, upper = u & 0xFFFF0000u;
      uint32_t lsb = (u >> 16) & 1u;
      if (lower > 0x8000u || (lower == 0x8000u && lsb)) upper += 0x10000u;
      u = upper;
    }
    memcpy(&out[i], &u, 4);
  }
}

/* Round values to IEEE binary16 (round to nearest, ties to even, with
 * subnormals), returned as float32.  Values past the largest finite half
 * become +-inf. */
void oracle_round_f16(const float* in, int64_t count, float* out) {
  for (int64_t i = 0; i < count; ++i) {
    double x = (double)in[i];
    double ax = fabs(x);
    double r;
    if (ax != ax) {
      r = x;
    } else if (ax == 0.0) {
      r = x;
    } else {
      int e;
      frexp(ax, &e); /* ax = f * 2^e, f in [0.5, 1) -> exponent of leading bit is e-1 */
      int lead = e - 1;
      if (lead < -14) lead = -14;        /* subnormal range: fixed quantum 2^-24 */
      double q = ldexp(1.0, lead - 10);  /* 10 fraction bits */
      double m = ax / q;                 /* exact: power-of-two scaling */
      double fl = floor(m), fr = m - fl;
      double rm = fl;
      if (fr > 0.5 || (fr == 0.5 && fmod(fl, 2.0) != 0.0)) rm = fl + 1.0;
      r = rm * q;
      if (r > 65504.0) r = INFINITY;
      if (x < 0) r = -r;
    }
    out[i] = (float)r;
  }
}
