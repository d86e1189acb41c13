// Device-side random augmentation parameters (Sec. 4): per volume, the affine
// (rotation, scale, reflection, shear and generic factors composed, then the
// offset b = c_in + d - A c_out that moves the output centre onto the input
// centre displaced by d), the intensity affine or window, and the occlusion
// slab, drawn from Philox4x32-10 and written into the descriptors in device
// memory.  One CTA; a thread per volume.  The composition is done in double:
// it is a few hundred operations per volume, and double makes the float32
// results the correctly rounded values of the exact composition in nearly
// every case.  Products and sums are rounded one at a time (no fused
// multiply-add), left to right, so that only sin/cos can differ in the last
// bit from a plain double evaluation of the same formulas.
#include "kernels.h"

namespace augk {
namespace {

__device__ __forceinline__ double mul(double a, double b) { return __dmul_rn(a, b); }
__device__ __forceinline__ double add(double a, double b) { return __dadd_rn(a, b); }
__device__ __forceinline__ double sub(double a, double b) { return __dsub_rn(a, b); }
// 2u - 1 (exact for the 24-bit uniforms).
__device__ __forceinline__ double sym(double u) { return sub(mul(2.0, u), 1.0); }

__device__ __forceinline__ void mat3_mul(const double* a, const double* b, double* out) {
  double t[9];
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int j = 0; j < 3; ++j)
      t[3 * i + j] = add(add(mul(a[3 * i], b[j]), mul(a[3 * i + 1], b[3 + j])),
                         mul(a[3 * i + 2], b[6 + j]));
#pragma unroll
  for (int i = 0; i < 9; ++i) out[i] = t[i];
}

// Rotation by angle g about axis 0 (x), 1 (y) or 2 (z), acting on the other two.
__device__ __forceinline__ void rotation(int axis, double g, double* m) {
  const int a = axis == 0 ? 1 : 0, b = axis == 2 ? 1 : 2;
#pragma unroll
  for (int i = 0; i < 9; ++i) m[i] = (i % 4 == 0) ? 1.0 : 0.0;
  double sn, cs;
  sincos(g, &sn, &cs);
  m[3 * a + a] = cs;
  m[3 * a + b] = -sn;
  m[3 * b + a] = sn;
  m[3 * b + b] = cs;
}

__device__ __forceinline__ double lerp_u(const float* range, double u) {
  return add((double)range[0], mul(sub((double)range[1], (double)range[0]), u));
}

}  // namespace

__global__ void __launch_bounds__(256)
    k_sample_params(aug_volume_desc* descs, int n_vols, aug_param_spec sp, unsigned key0,
                    unsigned key1, unsigned long long draw0, unsigned long long* counter) {
  __shared__ unsigned long long s_draw;
  if (threadIdx.x == 0) s_draw = draw0 + (counter ? *counter : 0ull);
  __syncthreads();
  const unsigned long long n = s_draw;
  // Every thread has its copy of n; the counter can advance.
  if (threadIdx.x == 0 && counter) *counter = n - draw0 + 1ull;
  for (int v = threadIdx.x; v < n_vols; v += blockDim.x) {
    aug_volume_desc& d = descs[v];
    double u[32];
#pragma unroll
    for (unsigned j = 0; j < 8; ++j) {
      const uint4 w = philox4x32_10(
          make_uint4(j, d.noise_id, (unsigned)n, 0x80000000u | (unsigned)(n >> 32)), key0, key1);
      u[4 * j + 0] = (double)(w.x >> 8) * 5.9604644775390625e-8;
      u[4 * j + 1] = (double)(w.y >> 8) * 5.9604644775390625e-8;
      u[4 * j + 2] = (double)(w.z >> 8) * 5.9604644775390625e-8;
      u[4 * j + 3] = (double)(w.w >> 8) * 5.9604644775390625e-8;
    }
    unsigned flags = d.flags;
    if (sp.draw & AUG_DRAW_AFFINE) {
      double A[9], R[9], M[9];
#pragma unroll
      for (int i = 0; i < 9; ++i)
        A[i] = add((i % 4 == 0) ? 1.0 : 0.0, mul((double)sp.generic_max, sym(u[12 + i])));
      rotation(2, mul((double)sp.rot_max[2], sym(u[2])), R);
      mat3_mul(A, R, A);
      rotation(1, mul((double)sp.rot_max[1], sym(u[1])), R);
      mat3_mul(A, R, A);
      rotation(0, mul((double)sp.rot_max[0], sym(u[0])), R);
      mat3_mul(A, R, A);
#pragma unroll
      for (int i = 0; i < 9; ++i) M[i] = (i % 4 == 0) ? 1.0 : 0.0;
      M[1] = mul((double)sp.shear_max, sym(u[9]));
      M[2] = mul((double)sp.shear_max, sym(u[10]));
      M[5] = mul((double)sp.shear_max, sym(u[11]));
      mat3_mul(A, M, A);
      // Right factor diag(refl s extra): scales column r.
#pragma unroll
      for (int r = 0; r < 3; ++r) {
        const double s = add((double)sp.scale_min[r],
                             mul(sub((double)sp.scale_max[r], (double)sp.scale_min[r]), u[3 + r]));
        const double refl = (u[6 + r] < (double)sp.reflect_prob[r]) ? -1.0 : 1.0;
        const double f = mul(mul(refl, s), (double)sp.extra_scale[r]);
#pragma unroll
        for (int i = 0; i < 3; ++i) A[3 * i + r] = mul(A[3 * i + r], f);
      }
      const int in_n[3] = {d.in_nx, d.in_ny, d.in_nz};
      // (N - 1) / 2 is exact.
      const double c_out[3] = {((double)d.out_nx - 1.0) / 2.0, ((double)d.out_ny - 1.0) / 2.0,
                               ((double)d.out_nz - 1.0) / 2.0};
#pragma unroll
      for (int r = 0; r < 3; ++r) {
        const double disp = mul((double)sp.shift_max[r], sym(u[21 + r]));
        const double Ac = add(add(mul(A[3 * r], c_out[0]), mul(A[3 * r + 1], c_out[1])),
                              mul(A[3 * r + 2], c_out[2]));
        const double b = sub(add(((double)in_n[r] - 1.0) / 2.0, disp), Ac);
        d.affine[4 * r + 0] = (float)A[3 * r + 0];
        d.affine[4 * r + 1] = (float)A[3 * r + 1];
        d.affine[4 * r + 2] = (float)A[3 * r + 2];
        d.affine[4 * r + 3] = (float)b;
      }
    }
    const double sigma = lerp_u(sp.sigma, u[26]);
    if (sp.draw & AUG_DRAW_WINDOW) {
      const double lo = lerp_u(sp.window_lo, u[27]), hi = lerp_u(sp.window_hi, u[28]);
      const double w = sub(hi, lo);
      d.photo_a = (float)__ddiv_rn(1.0, w);
      d.photo_b = (float)__ddiv_rn(-lo, w);
      d.noise_sigma = (float)__ddiv_rn(sigma, w);
      flags |= AUG_FLAG_WINDOW;
    } else if (sp.draw & AUG_DRAW_PHOTO) {
      d.photo_a = (float)lerp_u(sp.photo_a, u[24]);
      d.photo_b = (float)lerp_u(sp.photo_b, u[25]);
      d.noise_sigma = (float)sigma;
    }
    if (sp.draw & AUG_DRAW_OCCLUDE) {
      const double dmax = mul((double)sp.occ_max_frac, (double)d.out_nz);
      d.occ_dz = (float)mul(dmax, u[29]);
      d.occ_z0 = (float)add(-dmax, mul(add((double)d.out_nz - 1.0, dmax), u[30]));
      flags |= AUG_FLAG_OCCLUDE;
    }
    d.flags = flags;
  }
}

cudaError_t launch_sample_params(aug_volume_desc* d, int n, const aug_param_spec& sp,
                                 unsigned k0, unsigned k1, unsigned long long draw,
                                 unsigned long long* counter, cudaStream_t st) {
  k_sample_params<<<1, 256, 0, st>>>(d, n, sp, k0, k1, draw, counter);
  return cudaGetLastError();
}

}  // namespace augk
