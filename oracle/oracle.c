/*
 * oracle.c -- plain FP64 reference of the CT augmentation hot path.
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the checker the CUDA library is
 * compared against: it is compiled into liboracle.so and called from the test
 * suite, from __graft_entry__.smoke() and from the benchmark's CPU-baseline
 * leg, never from the product path.  It shares no code, header, table or
 * constant generator with the CUDA library.
 *
 * Everything is single threaded, unblocked and computed in double precision
 * directly from the definitions:
 *
 *   coordinate   s = A o + b                          (Sec. 4, x' = Ax + b)
 *   image        trilinear interpolation of the input,
 *                every tap outside the volume reads the fill value
 *                                                     (Sec. 4, texture sampling)
 *   label        nearest voxel, floor(s + 1/2), fill label outside
 *                                                     (Sec. 4, nearest neighbour)
 *   intensity    y = a v + beta + sigma n,  n ~ N(0, 1) (Sec. 4, additive noise)
 *   occlusion    optional: output voxels with z0 <= k <= z0 + dz (output z index)
 *                are 0 and skip every later step (Sec. 4, random occlusion)
 *   window       optional: y <- min(max(y, 0), 1) after the noise; with
 *                a = 1/(hi - lo), beta = -lo/(hi - lo) and sigma scaled by a
 *                this is the window/level map clamp((I - lo)/(hi - lo), 0, 1)
 *                applied to the noisy image (Sec. 4, window/level)
 *   noise        Philox4x32-10 (Salmon et al., SC'11) + Box-Muller
 *   adjoint      d(out)/d(input) and d(out)/d(T) of the above
 *   IOU loss     1 - |py|_1 / (|p|_1 + |y|_1 - |py|_1), per class
 *                                                     (Sec. 5.C, IOU loss)
 *
 * Conventions: volumes are [nz][ny][nx], x fastest.  An output index
 * o = (i, j, k) maps to the input coordinate s_r = T[r][0] i + T[r][1] j +
 * T[r][2] k + T[r][3] (r = x, y, z; T row-major 3x4, float32 promoted exactly
 * to double).  Voxel centres sit at integer coordinates.
 *
 * Noise: output voxels are grouped in quads of four z-consecutive voxels,
 * quad index Q = ((k >> 2) * ony + j) * onx + i, lane l = k & 3.  One
 * Philox4x32-10 call with key (lo32(seed), hi32(seed)) and counter
 * (lo32(Q), hi32(Q), noise_id, 0) gives words r0..r3; lanes 0,1 use the pair
 * (r0, r1), lanes 2,3 the pair (r2, r3).  With u1 = ((ra >> 8) + 1) 2^-24 in
 * (0, 1] and u2 = (rb >> 8) 2^-24 in [0, 1) (both exact in float32),
 * R = sqrt(-2 ln u1); even lanes take R cos(2 pi u2), odd lanes R sin(2 pi u2).
 */
#include <math.h>
#include <stddef.h>
#include <stdlib.h>
#include <stdint.h>
#include <string.h>

#define ORACLE_EXPORT __attribute__((visibility("default")))

/* ------------------------------------------------------------------------ */
/* Philox4x32-10, from the published round function:                         */
/*   (hi0, lo0) = M0 * c0,  (hi1, lo1) = M1 * c2   (32x32 -> 64 bit)        */
/*   c <- (hi1 ^ c1 ^ k0, lo1, hi0 ^ c3 ^ k1, lo0)                            */
/* with the key advanced by the Weyl constants between rounds.               */
/* ------------------------------------------------------------------------ */
ORACLE_EXPORT void oracle_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2],
                                        uint32_t out[4]) {
  const uint32_t M0 = 0xD2511F53u, M1 = 0xCD9E8D57u;
  const uint32_t W0 = 0x9E3779B9u, W1 = 0xBB67AE85u;
  uint32_t c0 = ctr[0], c1 = ctr[1], c2 = ctr[2], c3 = ctr[3];
  uint32_t k0 = key[0], k1 = key[1];
  for (int round = 0; round < 10; ++round) {
    if (round > 0) {
      k0 += W0;
      k1 += W1;
    }
    uint64_t p0 = (uint64_t)M0 * (uint64_t)c0;
    uint64_t p1 = (uint64_t)M1 * (uint64_t)c2;
    uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
    uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
    uint32_t n0 = hi1 ^ c1 ^ k0;
    uint32_t n2 = hi0 ^ c3 ^ k1;
    c0 = n0;
    c1 = lo1;
    c2 = n2;
    c3 = lo0;
  }
  out[0] = c0;
  out[1] = c1;
  out[2] = c2;
  out[3] = c3;
}

/* Philox words for n counters (n x 4 words in, n x 4 words out). */
ORACLE_EXPORT void oracle_philox_many(uint64_t seed, const uint32_t* ctrs, int64_t n,
                                      uint32_t* out) {
  uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
  for (int64_t q = 0; q < n; ++q) oracle_philox4x32_10(ctrs + 4 * q, key, out + 4 * q);
}

/* Standard normal for output voxel (i, j, k) of a volume (see header). */
static double noise_normal(uint64_t seed, uint32_t noise_id, int64_t onx, int64_t ony,
                           int64_t i, int64_t j, int64_t k) {
  const double two_m24 = 1.0 / 16777216.0;
  const double pi = 3.14159265358979323846;
  uint64_t quad = (uint64_t)(((k >> 2) * ony + j) * onx + i);
  uint32_t ctr[4] = {(uint32_t)quad, (uint32_t)(quad >> 32), noise_id, 0u};
  uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
  uint32_t r[4];
  oracle_philox4x32_10(ctr, key, r);
  int lane = (int)(k & 3);
  uint32_t ra = (lane < 2) ? r[0] : r[2];
  uint32_t rb = (lane < 2) ? r[1] : r[3];
  double u1 = ((double)(ra >> 8) + 1.0) * two_m24;
  double u2 = (double)(rb >> 8) * two_m24;
  double radius = sqrt(-2.0 * log(u1));
  return (lane & 1) ? radius * sin(2.0 * pi * u2) : radius * cos(2.0 * pi * u2);
}

/* Standard normals for a list of flattened output indices q = (k*ony+j)*onx+i. */
ORACLE_EXPORT void oracle_noise(uint64_t seed, uint32_t noise_id, int64_t onx, int64_t ony,
                                const int64_t* q, int64_t n, double* z) {
  for (int64_t m = 0; m < n; ++m) {
    int64_t i = q[m] % onx, j = (q[m] / onx) % ony, k = q[m] / (onx * ony);
    z[m] = noise_normal(seed, noise_id, onx, ony, i, j, k);
  }
}

/* ------------------------------------------------------------------------ */
/* Sampling                                                                  */
/* ------------------------------------------------------------------------ */
typedef struct {
  const void* image;
  int image_is_i16;
  const uint8_t* label;
  int64_t nx, ny, nz;
  int64_t onx, ony, onz;
  double T[3][4];
  double a, beta, sigma, fill;
  int fill_label;
  uint64_t seed;
  uint32_t noise_id;
  int flags;  /* 1: clamp to [0, 1] (window/level), 2: occlusion */
  double occ_z0, occ_dz;
} volume;

#define ORACLE_CLAMP01 1
#define ORACLE_OCCLUDE 2

static void load_volume(volume* v, const void* image, int image_is_i16, const uint8_t* label,
                        int64_t nx, int64_t ny, int64_t nz, int64_t onx, int64_t ony,
                        int64_t onz, const float* T12, float a, float beta, float sigma,
                        float fill, int fill_label, uint64_t seed, uint32_t noise_id, int flags,
                        float occ_z0, float occ_dz) {
  v->flags = flags;
  v->occ_z0 = occ_z0;
  v->occ_dz = occ_dz;
  v->image = image;
  v->image_is_i16 = image_is_i16;
  v->label = label;
  v->nx = nx;
  v->ny = ny;
  v->nz = nz;
  v->onx = onx;
  v->ony = ony;
  v->onz = onz;
  for (int r = 0; r < 3; ++r)
    for (int c = 0; c < 4; ++c) v->T[r][c] = (double)T12[4 * r + c];
  v->a = a;
  v->beta = beta;
  v->sigma = sigma;
  v->fill = fill;
  v->fill_label = fill_label;
  v->seed = seed;
  v->noise_id = noise_id;
}

static int in_volume(const volume* v, int64_t x, int64_t y, int64_t z) {
  return x >= 0 && y >= 0 && z >= 0 && x < v->nx && y < v->ny && z < v->nz;
}

/* V(n): input value at integer position n, or the fill value outside. */
static double image_at(const volume* v, int64_t x, int64_t y, int64_t z) {
  if (!in_volume(v, x, y, z)) return v->fill;
  size_t idx = ((size_t)z * (size_t)v->ny + (size_t)y) * (size_t)v->nx + (size_t)x;
  if (v->image_is_i16) return (double)((const int16_t*)v->image)[idx];
  return (double)((const float*)v->image)[idx];
}

static void coordinate(const volume* v, int64_t i, int64_t j, int64_t k, double s[3]) {
  for (int r = 0; r < 3; ++r)
    s[r] = v->T[r][0] * (double)i + v->T[r][1] * (double)j + v->T[r][2] * (double)k +
           v->T[r][3];
}

/* Trilinear interpolation: sum over the 8 corners d of the cell floor(s) of
 * prod_r (d_r ? t_r : 1 - t_r) * V(floor(s) + d). */
static double trilinear(const volume* v, const double s[3]) {
  double f[3], t[3];
  for (int r = 0; r < 3; ++r) {
    f[r] = floor(s[r]);
    t[r] = s[r] - f[r];
  }
  double acc = 0.0;
  for (int d = 0; d < 8; ++d) {
    int dx = d & 1, dy = (d >> 1) & 1, dz = (d >> 2) & 1;
    double w = (dx ? t[0] : 1.0 - t[0]) * (dy ? t[1] : 1.0 - t[1]) * (dz ? t[2] : 1.0 - t[2]);
    acc += w * image_at(v, (int64_t)f[0] + dx, (int64_t)f[1] + dy, (int64_t)f[2] + dz);
  }
  return acc;
}

static int nearest_label(const volume* v, const double s[3]) {
  int64_t n[3];
  for (int r = 0; r < 3; ++r) n[r] = (int64_t)floor(s[r] + 0.5);
  if (!in_volume(v, n[0], n[1], n[2])) return v->fill_label;
  size_t idx = ((size_t)n[2] * (size_t)v->ny + (size_t)n[1]) * (size_t)v->nx + (size_t)n[0];
  return v->label[idx];
}

static int near_tie(const double s[3]) {
  for (int r = 0; r < 3; ++r)
    if (fabs(s[r] - floor(s[r]) - 0.5) < 1e-5) return 1;
  return 0;
}

static int occluded(const volume* v, int64_t k) {
  return (v->flags & ORACLE_OCCLUDE) && (double)k >= v->occ_z0 &&
         (double)k <= v->occ_z0 + v->occ_dz;
}

static void one_voxel(const volume* v, int64_t i, int64_t j, int64_t k, double* out_val,
                      uint8_t* out_lab, uint8_t* tie) {
  double s[3];
  coordinate(v, i, j, k, s);
  if (out_val) {
    if (occluded(v, k)) {
      *out_val = 0.0;
    } else {
      double val = v->a * trilinear(v, s) + v->beta;
      if (v->sigma != 0.0)
        val += v->sigma * noise_normal(v->seed, v->noise_id, v->onx, v->ony, i, j, k);
      if (v->flags & ORACLE_CLAMP01) val = val < 0.0 ? 0.0 : (val > 1.0 ? 1.0 : val);
      *out_val = val;
    }
  }
  if (out_lab) *out_lab = (uint8_t)nearest_label(v, s);
  if (tie) *tie = (uint8_t)near_tie(s);
}

/* Forward warp of one volume over its whole output grid.  Any of out_image,
 * out_label, tie may be NULL.  Returns the number of label-tie voxels (source
 * coordinate within 1e-5 of a rounding tie on some axis). */
ORACLE_EXPORT int64_t oracle_warp_fwd(const void* image, int image_is_i16,
                                      const uint8_t* label, int64_t nx, int64_t ny,
                                      int64_t nz, int64_t onx, int64_t ony, int64_t onz,
                                      const float* T12, float a, float beta, float sigma,
                                      float fill, int fill_label, uint64_t seed,
                                      uint32_t noise_id, int flags, float occ_z0, float occ_dz,
                                      double* out_image, uint8_t* out_label, uint8_t* tie) {
  volume v;
  load_volume(&v, image, image_is_i16, label, nx, ny, nz, onx, ony, onz, T12, a, beta, sigma,
              fill, fill_label, seed, noise_id, flags, occ_z0, occ_dz);
  int64_t ties = 0;
  size_t q = 0;
  for (int64_t k = 0; k < onz; ++k)
    for (int64_t j = 0; j < ony; ++j)
      for (int64_t i = 0; i < onx; ++i, ++q) {
        uint8_t tflag = 0;
        one_voxel(&v, i, j, k, out_image ? out_image + q : NULL,
                  (out_label && label) ? out_label + q : NULL, &tflag);
        if (tie) tie[q] = tflag;
        ties += tflag;
      }
  return ties;
}

/* Forward warp evaluated only at the listed flattened output indices. */
ORACLE_EXPORT void oracle_warp_fwd_points(const void* image, int image_is_i16,
                                          const uint8_t* label, int64_t nx, int64_t ny,
                                          int64_t nz, int64_t onx, int64_t ony, int64_t onz,
                                          const float* T12, float a, float beta, float sigma,
                                          float fill, int fill_label, uint64_t seed,
                                          uint32_t noise_id, int flags, float occ_z0,
                                          float occ_dz, const int64_t* q, int64_t n,
                                          double* out_image, uint8_t* out_label,
                                          uint8_t* tie) {
  volume v;
  load_volume(&v, image, image_is_i16, label, nx, ny, nz, onx, ony, onz, T12, a, beta, sigma,
              fill, fill_label, seed, noise_id, flags, occ_z0, occ_dz);
  for (int64_t m = 0; m < n; ++m) {
    int64_t i = q[m] % onx, j = (q[m] / onx) % ony, k = q[m] / (onx * ony);
    one_voxel(&v, i, j, k, out_image ? out_image + m : NULL,
              (out_label && label) ? out_label + m : NULL, tie ? tie + m : NULL);
  }
}

/* ------------------------------------------------------------------------ */
/* Adjoint of the image warp.                                                */
/*   out(o) = a * sum_d w_d(o) V(f(o) + d) + beta (+ noise, independent of   */
/*   the input and of T).  With g the upstream gradient:                     */
/*   grad_in[n]  = sum_o a g(o) w_d(o)      over in-volume taps n = f(o) + d */
/*   dv/ds_r     = sum_d (d_r ? +1 : -1) prod_{q != r} (d_q ? t_q : 1 - t_q)  */
/*                 V(f + d)     (right derivative where s_r is an integer)   */
/*   grad_T[r][c] = sum_o a g(o) dv/ds_r(o) obar_c(o), obar = (i, j, k, 1).  */
/* Fill taps contribute to dv/ds but not to grad_in.  Occluded output voxels  */
/* (flags & 2) contribute nothing.  The clamp of flags & 1 is not modelled:    */
/* the adjoint is defined for unclamped outputs.                              */
/* grad_in (input shape, overwritten), grad_T (12) and dvds (3 per output     */
/* voxel) may each be NULL.                                                  */
/* ------------------------------------------------------------------------ */
ORACLE_EXPORT void oracle_warp_bwd(const void* image, int image_is_i16, int64_t nx,
                                   int64_t ny, int64_t nz, int64_t onx, int64_t ony,
                                   int64_t onz, const float* T12, float a, float fill, int flags,
                                   float occ_z0, float occ_dz, const float* g, double* grad_in,
                                   double* grad_T, double* dvds) {
  volume v;
  load_volume(&v, image, image_is_i16, NULL, nx, ny, nz, onx, ony, onz, T12, a, 0.0f, 0.0f,
              fill, 0, 0, 0, flags, occ_z0, occ_dz);
  if (grad_in) memset(grad_in, 0, sizeof(double) * (size_t)(nx * ny * nz));
  double gt[3][4] = {{0}};
  size_t q = 0;
  for (int64_t k = 0; k < onz; ++k)
    for (int64_t j = 0; j < ony; ++j)
      for (int64_t i = 0; i < onx; ++i, ++q) {
        double s[3], f[3], t[3];
        coordinate(&v, i, j, k, s);
        for (int r = 0; r < 3; ++r) {
          f[r] = floor(s[r]);
          t[r] = s[r] - f[r];
        }
        /* An occluded voxel is the constant 0: no gradient flows through it. */
        double ga = occluded(&v, k) ? 0.0 : v.a * (double)g[q];
        double dv[3] = {0.0, 0.0, 0.0};
        for (int d = 0; d < 8; ++d) {
          int dd[3] = {d & 1, (d >> 1) & 1, (d >> 2) & 1};
          double wt[3];
          for (int r = 0; r < 3; ++r) wt[r] = dd[r] ? t[r] : 1.0 - t[r];
          int64_t x = (int64_t)f[0] + dd[0], y = (int64_t)f[1] + dd[1],
                  z = (int64_t)f[2] + dd[2];
          double val = image_at(&v, x, y, z);
          for (int r = 0; r < 3; ++r) {
            double w_other = 1.0;
            for (int p = 0; p < 3; ++p)
              if (p != r) w_other *= wt[p];
            dv[r] += (dd[r] ? 1.0 : -1.0) * w_other * val;
          }
          if (grad_in && in_volume(&v, x, y, z))
            grad_in[((size_t)z * (size_t)ny + (size_t)y) * (size_t)nx + (size_t)x] +=
                ga * wt[0] * wt[1] * wt[2];
        }
        double obar[4] = {(double)i, (double)j, (double)k, 1.0};
        for (int r = 0; r < 3; ++r)
          for (int c = 0; c < 4; ++c) gt[r][c] += ga * dv[r] * obar[c];
        if (dvds)
          for (int r = 0; r < 3; ++r) dvds[3 * q + r] = dv[r];
      }
  if (grad_T)
    for (int r = 0; r < 3; ++r)
      for (int c = 0; c < 4; ++c) grad_T[4 * r + c] = gt[r][c];
}

/* ------------------------------------------------------------------------ */
/* Soft IOU loss of one volume (Sec. 5.C).                                   */
/* p: [C][nvox] probabilities, y: [nvox] labels in 0..C-1 (other values      */
/* belong to no class).  For each class c, with y_k = [label_k == c]:        */
/*   I = sum p y, P = sum p, Y = sum y, U = P + Y - I,                       */
/*   L_c = 1 - I / U   (U = 0: L_c = 0, the score of an empty prediction of  */
/*                      an empty class being 1),                             */
/*   dL_c/dp_k = y_k ? -1/U : I/U^2   (0 where U = 0),                        */
/* grad[c][k] = grad_scale * dL_c/dp_k (double).  sums: [C][3] = (I, P, Y);  */
/* loss_c: [C].  grad and sums may be NULL.                                  */
/* ------------------------------------------------------------------------ */
ORACLE_EXPORT void oracle_iou(const float* p, const uint8_t* y, int n_classes, int64_t nvox,
                              double grad_scale, double* loss_c, double* sums, double* grad) {
  for (int c = 0; c < n_classes; ++c) {
    const float* pc = p + (size_t)c * (size_t)nvox;
    double I = 0.0, P = 0.0, Y = 0.0;
    for (int64_t k = 0; k < nvox; ++k) {
      double pk = (double)pc[k];
      double yk = (y[k] == c) ? 1.0 : 0.0;
      I += pk * yk;
      P += pk;
      Y += yk;
    }
    double U = P + Y - I;
    loss_c[c] = (U > 0.0) ? 1.0 - I / U : 0.0;
    if (sums) {
      sums[3 * c + 0] = I;
      sums[3 * c + 1] = P;
      sums[3 * c + 2] = Y;
    }
    if (grad) {
      double* gc = grad + (size_t)c * (size_t)nvox;
      for (int64_t k = 0; k < nvox; ++k) {
        double d = 0.0;
        if (U > 0.0) d = (y[k] == c) ? -1.0 / U : I / (U * U);
        gc[k] = grad_scale * d;
      }
    }
  }
}

/* ------------------------------------------------------------------------ */
/* Loss variants of Sec. 5.C on one volume, same layouts as oracle_iou, with  */
/* q_k = p_k^m (m > 0; q = p for m = 1, the L^m family of Sec. 5.C):          */
/*   kind 0  IOU     L = 1 - I/U,            U = P + Y - I                    */
/*   kind 1  Dice    L = 1 - 2I/(P + Y)                                       */
/* with I = sum q y, P = sum q, Y = sum y, and a zero denominator giving     */
/* loss 0 and gradient 0.  Gradients:                                         */
/*   IOU    dL/dq_k = y_k ? -1/U : I/U^2                                      */
/*   Dice   dL/dq_k = (2I - 2 y_k (P + Y)) / (P + Y)^2                        */
/*   dL/dp_k = m p_k^(m-1) dL/dq_k                                            */
/* With logits != 0 the input x holds per-voxel class scores and             */
/* p_{c,k} = exp(x_{c,k}) / sum_j exp(x_{j,k}) (softmax over the classes);    */
/* the gradient is then taken with respect to x:                              */
/*   dL/dx_{c,k} = p_{c,k} (g_{c,k} - sum_j p_{j,k} g_{j,k}),  g = dL/dp.      */
/* L here is the batch-level mean over classes, so the class terms of the    */
/* softmax chain rule add up across classes.                                  */
/* ------------------------------------------------------------------------ */
ORACLE_EXPORT void oracle_loss(const float* x, const uint8_t* y, int n_classes, int64_t nvox,
                               int kind, double m, int logits, double grad_scale,
                               double* loss_c, double* sums, double* grad) {
  const size_t n = (size_t)n_classes * (size_t)nvox;
  double* p = (double*)malloc(n * sizeof(double));
  double* g = (double*)malloc(n * sizeof(double));
  for (int64_t k = 0; k < nvox; ++k) {
    if (logits) {
      double mx = -INFINITY, z = 0.0;
      for (int c = 0; c < n_classes; ++c) mx = fmax(mx, (double)x[(size_t)c * nvox + k]);
      for (int c = 0; c < n_classes; ++c) z += exp((double)x[(size_t)c * nvox + k] - mx);
      for (int c = 0; c < n_classes; ++c)
        p[(size_t)c * nvox + k] = exp((double)x[(size_t)c * nvox + k] - mx) / z;
    } else {
      for (int c = 0; c < n_classes; ++c) p[(size_t)c * nvox + k] = (double)x[(size_t)c * nvox + k];
    }
  }
  for (int c = 0; c < n_classes; ++c) {
    const double* pc = p + (size_t)c * (size_t)nvox;
    double I = 0.0, P = 0.0, Y = 0.0;
    for (int64_t k = 0; k < nvox; ++k) {
      double q = (m == 1.0) ? pc[k] : pow(pc[k], m);
      double yk = (y[k] == c) ? 1.0 : 0.0;
      I += q * yk;
      P += q;
      Y += yk;
    }
    double den = (kind == 1) ? P + Y : P + Y - I;
    double l = 0.0;
    if (den > 0.0) l = (kind == 1) ? 1.0 - 2.0 * I / den : 1.0 - I / den;
    loss_c[c] = l;
    if (sums) {
      sums[3 * c + 0] = I;
      sums[3 * c + 1] = P;
      sums[3 * c + 2] = Y;
    }
    double* gc = g + (size_t)c * (size_t)nvox;
    for (int64_t k = 0; k < nvox; ++k) {
      double d = 0.0;
      int yk = y[k] == c;
      if (den > 0.0) {
        if (kind == 1)
          d = (2.0 * I - (yk ? 2.0 * den : 0.0)) / (den * den);
        else
          d = yk ? -1.0 / den : I / (den * den);
        if (m != 1.0) d *= m * pow(pc[k], m - 1.0);
      }
      gc[k] = grad_scale * d;
    }
  }
  if (grad) {
    for (int64_t k = 0; k < nvox; ++k) {
      double dot = 0.0;
      if (logits)
        for (int c = 0; c < n_classes; ++c)
          dot += p[(size_t)c * nvox + k] * g[(size_t)c * nvox + k];
      for (int c = 0; c < n_classes; ++c) {
        const size_t i = (size_t)c * nvox + k;
        grad[i] = logits ? p[i] * (g[i] - dot) : g[i];
      }
    }
  }
  free(p);
  free(g);
}

/* ------------------------------------------------------------------------ */
/* Random augmentation parameters of one volume (Sec. 4), drawn from        */
/* Philox4x32-10 with key (lo32 seed, hi32 seed) and counter                 */
/* (j, noise_id, lo32 draw, 0x80000000 | hi32 draw), j = 0..7: words        */
/* w[4j..4j+3], uniforms u_n = (w_n >> 8) 2^-24 in [0, 1).  (The set top    */
/* bit of the last counter word keeps these counters apart from the noise's, */
/* whose last word is 0.)                                                    */
/*                                                                           */
/* spec (float32, this order):                                               */
/*   [0..2] rot_max  [3..5] scale_min  [6..8] scale_max  [9..11] reflect_prob */
/*   [12] shear_max  [13] generic_max  [14..16] extra_scale  [17..19] shift_max */
/*   [20,21] photo_a range  [22,23] photo_b range  [24,25] sigma range       */
/*   [26,27] window lo range  [28,29] window hi range  [30] occ_max_frac     */
/* draw_mask: 1 affine, 2 intensity affine + sigma, 4 window (+ sigma),     */
/*            8 occlusion.                                                   */
/*                                                                           */
/* Affine: angles g_r = rot_max_r (2u_r - 1) (u0..u2), scales               */
/* s_r = min_r + (max_r - min_r) u_{3+r}, reflection sign -1 where          */
/* u_{6+r} < reflect_prob_r, shear entries (0,1), (0,2), (1,2) =            */
/* shear_max (2u - 1) (u9..u11), generic perturbation G (row-major) =        */
/* generic_max (2u - 1) (u12..u20), displacement d_r = shift_max_r (2u - 1) */
/* (u21..u23);                                                               */
/*   A = (I + G) Rz(g_z) Ry(g_y) Rx(g_x) Sh diag(refl s) diag(extra),        */
/*   b = c_in + d - A c_out,  c = (N - 1) / 2,                               */
/* so that A c_out + b = c_in + d: the output centre lands on the input      */
/* centre displaced by d.  T = (A | b) rounded to float32.                   */
/* Intensity: a, b, sigma from their ranges (u24, u25, u26).  Window:        */
/* lo, hi from their ranges (u27, u28), a = 1/(hi - lo), b = -lo/(hi - lo),  */
/* sigma = (sigma range draw u26) / (hi - lo), flag 1.  Occlusion:           */
/* dmax = occ_max_frac out_nz, dz = dmax u29, z0 = -dmax + (out_nz - 1 +     */
/* dmax) u30, flag 2.  Groups that are not drawn leave their outputs as      */
/* passed in.                                                                */
/* ------------------------------------------------------------------------ */
static void mat3_mul(const double a[9], const double b[9], double out[9]) {
  double t[9];
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) {
      double s = 0.0;
      for (int k = 0; k < 3; ++k) s += a[3 * i + k] * b[3 * k + j];
      t[3 * i + j] = s;
    }
  memcpy(out, t, sizeof(t));
}

static void rotation(int axis, double g, double m[9]) {
  /* Rotation by angle g about coordinate axis `axis` (0 = x, 1 = y, 2 = z). */
  const int pa[3] = {1, 0, 0}, pb[3] = {2, 2, 1};
  const int a = pa[axis], b = pb[axis];
  for (int i = 0; i < 9; ++i) m[i] = (i % 4 == 0) ? 1.0 : 0.0;
  m[3 * a + a] = cos(g);
  m[3 * a + b] = -sin(g);
  m[3 * b + a] = sin(g);
  m[3 * b + b] = cos(g);
}

ORACLE_EXPORT void oracle_sample_params(const float* spec, uint32_t draw_mask, uint64_t seed,
                                        uint64_t draw, uint32_t noise_id,
                                        const int64_t in_dims[3], const int64_t out_dims[3],
                                        float T[12], float photo[3], int32_t* flags,
                                        float occ[2], double d_out[3], double A_out[9]) {
  const double two_m24 = 1.0 / 16777216.0;
  uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
  double u[32];
  for (uint32_t j = 0; j < 8; ++j) {
    uint32_t ctr[4] = {j, noise_id, (uint32_t)draw, 0x80000000u | (uint32_t)(draw >> 32)};
    uint32_t w[4];
    oracle_philox4x32_10(ctr, key, w);
    for (int n = 0; n < 4; ++n) u[4 * j + n] = (double)(w[n] >> 8) * two_m24;
  }
  double S[32];
  for (int i = 0; i < 31; ++i) S[i] = (double)spec[i];

  if (draw_mask & 1u) {
    double g[3], s[3], refl[3], d[3];
    for (int r = 0; r < 3; ++r) {
      g[r] = S[r] * (2.0 * u[r] - 1.0);
      s[r] = S[3 + r] + (S[6 + r] - S[3 + r]) * u[3 + r];
      refl[r] = (u[6 + r] < S[9 + r]) ? -1.0 : 1.0;
      d[r] = S[17 + r] * (2.0 * u[21 + r] - 1.0);
    }
    double IG[9], Rx[9], Ry[9], Rz[9], Sh[9], D[9], A[9];
    for (int i = 0; i < 9; ++i) IG[i] = ((i % 4 == 0) ? 1.0 : 0.0) + S[13] * (2.0 * u[12 + i] - 1.0);
    rotation(0, g[0], Rx);
    rotation(1, g[1], Ry);
    rotation(2, g[2], Rz);
    for (int i = 0; i < 9; ++i) Sh[i] = (i % 4 == 0) ? 1.0 : 0.0;
    Sh[1] = S[12] * (2.0 * u[9] - 1.0);
    Sh[2] = S[12] * (2.0 * u[10] - 1.0);
    Sh[5] = S[12] * (2.0 * u[11] - 1.0);
    for (int i = 0; i < 9; ++i) D[i] = 0.0;
    for (int r = 0; r < 3; ++r) D[4 * r] = refl[r] * s[r] * S[14 + r];
    mat3_mul(IG, Rz, A);
    mat3_mul(A, Ry, A);
    mat3_mul(A, Rx, A);
    mat3_mul(A, Sh, A);
    mat3_mul(A, D, A);
    for (int r = 0; r < 3; ++r) {
      const double c_in = ((double)in_dims[r] - 1.0) / 2.0;
      double Ac = 0.0;
      for (int k = 0; k < 3; ++k) Ac += A[3 * r + k] * (((double)out_dims[k] - 1.0) / 2.0);
      const double b = c_in + d[r] - Ac;
      for (int k = 0; k < 3; ++k) T[4 * r + k] = (float)A[3 * r + k];
      T[4 * r + 3] = (float)b;
    }
    if (d_out) memcpy(d_out, d, sizeof(d));
    if (A_out) memcpy(A_out, A, sizeof(A));
  }
  const double sigma = S[24] + (S[25] - S[24]) * u[26];
  if (draw_mask & 4u) {
    const double lo = S[26] + (S[27] - S[26]) * u[27];
    const double hi = S[28] + (S[29] - S[28]) * u[28];
    photo[0] = (float)(1.0 / (hi - lo));
    photo[1] = (float)(-lo / (hi - lo));
    photo[2] = (float)(sigma / (hi - lo));
    *flags |= 1;
  } else if (draw_mask & 2u) {
    photo[0] = (float)(S[20] + (S[21] - S[20]) * u[24]);
    photo[1] = (float)(S[22] + (S[23] - S[22]) * u[25]);
    photo[2] = (float)sigma;
  }
  if (draw_mask & 8u) {
    const double dmax = S[30] * (double)out_dims[2];
    occ[1] = (float)(dmax * u[29]);
    occ[0] = (float)(-dmax + ((double)out_dims[2] - 1.0 + dmax) * u[30]);
    *flags |= 2;
  }
}

/* ------------------------------------------------------------------------ */
/* Anti-aliasing Gaussian of the resampling step (Sec. 5.A):                */
/*   S(p) = sum_{a,b,c} g(a, b, c) E(p + (a, b, c)),                         */
/*   g(x) = prod_k exp(-x_k^2 / sigma_k^2) / (normalisation over the support) */
/* with E the input extended by `fill` outside the volume, the support       */
/* |x_k| <= ceil(3 sigma_k) (a single tap where sigma_k = 0), and            */
/* sigma_k = max(r / u_k - 1, 0) / 3 for spacing u_k and target resolution r */
/* (both in mm; sigma in input voxels).  The triple sum is taken directly.   */
/* ------------------------------------------------------------------------ */
ORACLE_EXPORT double oracle_antialias_sigma(double r, double u) {
  const double t = r / u - 1.0;
  return (t > 0.0 ? t : 0.0) / 3.0;
}

ORACLE_EXPORT int oracle_gauss_radius(double sigma) {
  return sigma > 0.0 ? (int)ceil(3.0 * sigma) : 0;
}

/* Normalised 1-D weights w[0..2R], w[R + a] for offset a. */
ORACLE_EXPORT void oracle_gauss_weights(double sigma, double* w) {
  const int R = oracle_gauss_radius(sigma);
  double s = 0.0;
  for (int a = -R; a <= R; ++a) {
    w[R + a] = (R == 0) ? 1.0 : exp(-(double)a * (double)a / (sigma * sigma));
    s += w[R + a];
  }
  for (int a = 0; a <= 2 * R; ++a) w[a] /= s;
}

static double smooth_at(const void* image, int is_i16, int64_t nx, int64_t ny, int64_t nz,
                        const double* w[3], const int R[3], double fill, int64_t i, int64_t j,
                        int64_t k) {
  double s = 0.0;
  for (int c = -R[2]; c <= R[2]; ++c)
    for (int b = -R[1]; b <= R[1]; ++b)
      for (int a = -R[0]; a <= R[0]; ++a) {
        const int64_t x = i + a, y = j + b, z = k + c;
        double v = fill;
        if (x >= 0 && x < nx && y >= 0 && y < ny && z >= 0 && z < nz) {
          const int64_t n = (z * ny + y) * nx + x;
          v = is_i16 ? (double)((const int16_t*)image)[n] : (double)((const float*)image)[n];
        }
        s += w[0][R[0] + a] * w[1][R[1] + b] * w[2][R[2] + c] * v;
      }
  return s;
}

/* Smoothed value at output indices q (flattened (k*ny + j)*nx + i of the
 * input grid), FP64. */
ORACLE_EXPORT void oracle_smooth_points(const void* image, int is_i16, int64_t nx, int64_t ny,
                                        int64_t nz, const double sigma[3], double fill,
                                        const int64_t* q, int64_t n, double* out) {
  double wx[64], wy[64], wz[64];
  const double* w[3] = {wx, wy, wz};
  int R[3];
  for (int r = 0; r < 3; ++r) {
    R[r] = oracle_gauss_radius(sigma[r]);
    oracle_gauss_weights(sigma[r], (double*)w[r]);
  }
  for (int64_t m = 0; m < n; ++m) {
    const int64_t i = q[m] % nx, j = (q[m] / nx) % ny, k = q[m] / (nx * ny);
    out[m] = smooth_at(image, is_i16, nx, ny, nz, w, R, fill, i, j, k);
  }
}

/* Whole smoothed volume, FP64. */
ORACLE_EXPORT void oracle_smooth(const void* image, int is_i16, int64_t nx, int64_t ny,
                                 int64_t nz, const double sigma[3], double fill, double* out) {
  double wx[64], wy[64], wz[64];
  const double* w[3] = {wx, wy, wz};
  int R[3];
  for (int r = 0; r < 3; ++r) {
    R[r] = oracle_gauss_radius(sigma[r]);
    oracle_gauss_weights(sigma[r], (double*)w[r]);
  }
  for (int64_t k = 0; k < nz; ++k)
    for (int64_t j = 0; j < ny; ++j)
      for (int64_t i = 0; i < nx; ++i)
        out[(k * ny + j) * nx + i] = smooth_at(image, is_i16, nx, ny, nz, w, R, fill, i, j, k);
}
