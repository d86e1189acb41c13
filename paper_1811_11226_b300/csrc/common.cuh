// Device helpers shared by the augmentation kernels (sm_103a).
//
// Coordinates: s = A o + b (Sec. 4) is evaluated in signed 64-bit fixed point
// with 40 fractional bits ("Q.40").  Every float32 affine entry with
// |T| >= 2^-17 is exact in Q.40 and integer output indices are exact, so the
// coordinate equals the real-number value A o + b exactly; floor/round
// decisions (cell choice, nearest label) are therefore exact, and only the
// interpolation weight is rounded (to 23 bits).  Float32 coordinates would be
// off by up to ~1.5e-5 voxel at |s| ~ 200, i.e. ~0.02 HU at a 1000 HU edge.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <cmath>

#include "augwarp.h"

namespace augk {

constexpr unsigned FULL_MASK = 0xffffffffu;
constexpr int MAX_DIM = 8192;

// Workspace layout: a 256-byte header (status words), then op scratch.
struct WsHeader {
  int status;      // first device-side error (aug_status), 0 if none
  int bad_volume;  // volume index of that error
  unsigned long long tile_next;  // dynamic tile counter (zeroed by the prologue)
  int pad[60];
};
static_assert(sizeof(WsHeader) == 256, "header size");

__device__ __forceinline__ void record_error(WsHeader* ws, int code, int vol) {
  if (ws == nullptr) return;
  if (atomicCAS(&ws->status, 0, code) == 0) ws->bad_volume = vol;
}

// Per-volume constants staged in shared memory by each CTA.
struct VolConst {
  long long tq[3][4];  // affine in Q.40
  const void* image;
  const uint8_t* label;
  float* out_image;
  uint8_t* out_label;
  int nx, ny, nz, dtype;
  int onx, ony, onz, fill_label;
  float a, b, sigma, fill;
  unsigned noise_id;
  int ok;
  int flags;             // AUG_FLAG_* bits
  int occ_klo, occ_khi;  // occluded output z indices k_lo <= k <= k_hi (empty if k_lo > k_hi)
  // Inverse of the affine, o = ainv s + binv (input coordinate -> output
  // index), and the half-widths of the output box holding every o whose
  // sample lies within 1 of a given input voxel on each axis (the gather
  // adjoint); inv_ok = 0 when |det A| < 1e-6.
  double ainv[3][3], binv[3];
  float inv_h[3];
  int inv_ok;
};

// Full check of one descriptor (pure).  need_image: an image of a known
// dtype is required when out_image is set (forward) or always (adjoint);
// f32_only: the image must be float32 (adjoint with grad_in).
__device__ inline bool desc_valid(const aug_volume_desc& d, bool need_image, bool f32_only) {
  bool ok = true;
  ok &= d.in_nx >= 1 && d.in_ny >= 1 && d.in_nz >= 1 && d.in_nx <= MAX_DIM &&
        d.in_ny <= MAX_DIM && d.in_nz <= MAX_DIM;
  ok &= d.out_nx >= 1 && d.out_ny >= 1 && d.out_nz >= 1 && d.out_nx <= MAX_DIM &&
        d.out_ny <= MAX_DIM && d.out_nz <= MAX_DIM;
  ok &= (long long)d.in_nx * d.in_ny * d.in_nz < (1LL << 31);
  ok &= (long long)d.out_nx * d.out_ny * d.out_nz < (1LL << 31);
  ok &= d.fill_label >= 0 && d.fill_label <= 255;
  for (int m = 0; m < 12; ++m) {
    const float t = d.affine[m];
    ok &= isfinite(t) && fabsf(t) <= (((m & 3) < 3) ? 64.0f : 1048576.0f);
  }
  ok &= isfinite(d.photo_a) && isfinite(d.photo_b) && isfinite(d.noise_sigma) &&
        d.noise_sigma >= 0.0f && isfinite(d.fill_image);
  ok &= (d.flags & ~(unsigned)(AUG_FLAG_WINDOW | AUG_FLAG_OCCLUDE)) == 0u;
  ok &= isfinite(d.occ_z0) && isfinite(d.occ_dz) && d.occ_dz >= 0.0f;
  if (need_image) {
    ok &= d.image != nullptr && (d.image_dtype == AUG_F32 || d.image_dtype == AUG_I16);
    // element-aligned image (a misaligned pointer would fault on the first load)
    ok &= ((uintptr_t)d.image & (d.image_dtype == AUG_I16 ? 1u : 3u)) == 0u;
    if (f32_only) ok &= d.image_dtype == AUG_F32;
  }
  ok &= !(d.out_label != nullptr && d.label == nullptr);
  return ok;
}

// Parses one descriptor into per-volume constants (one thread).  with_inverse:
// also the inverse affine (double arithmetic, slow on this GPU's FP64 units:
// only the adjoint's prologue computes it, once per volume, for the gather).
// Also a host function (the plain one-volume launch builds the constants on the
// host and passes them by value): t * 2^40 is an integer-valued double for
// every float32 t with |t| <= 2^20, so both conversions below are exact.
__host__ __device__ inline void make_volconst(const aug_volume_desc& d, bool ok, VolConst& vc,
                                              bool with_inverse = true) {
#pragma unroll
  for (int m = 0; m < 12; ++m) {
    const float t = d.affine[m];
    const float lim = ((m & 3) < 3) ? 64.0f : 1048576.0f;
#ifdef __CUDA_ARCH__
    vc.tq[m >> 2][m & 3] =
        (isfinite(t) && fabsf(t) <= lim) ? __double2ll_rn((double)t * 1099511627776.0) : 0LL;
#else
    vc.tq[m >> 2][m & 3] =
        (std::isfinite(t) && std::fabs(t) <= lim) ? std::llrint((double)t * 1099511627776.0)
                                                  : 0LL;
#endif
  }
  vc.image = d.image;
  vc.label = d.label;
  vc.out_image = d.out_image;
  vc.out_label = d.out_label;
  vc.nx = d.in_nx;
  vc.ny = d.in_ny;
  vc.nz = d.in_nz;
  vc.dtype = d.image_dtype;
  vc.onx = d.out_nx;
  vc.ony = d.out_ny;
  vc.onz = d.out_nz;
  vc.fill_label = d.fill_label;
  vc.a = d.photo_a;
  vc.b = d.photo_b;
  vc.sigma = d.noise_sigma;
  vc.fill = d.fill_image;
  vc.noise_id = d.noise_id;
  vc.flags = (int)d.flags;
  // z0 <= k <= z0 + dz over integers k, decided in double exactly as written.
  vc.occ_klo = 1;
  vc.occ_khi = 0;
  if ((d.flags & AUG_FLAG_OCCLUDE) && isfinite(d.occ_z0) && isfinite(d.occ_dz)) {
    const double lo = ceil((double)d.occ_z0), hi = floor((double)d.occ_z0 + (double)d.occ_dz);
    vc.occ_klo = (int)fmin(fmax(lo, -1.0), 1073741824.0);
    vc.occ_khi = (int)fmin(fmax(hi, -2.0), 1073741824.0);
  }
  vc.inv_ok = 0;
  vc.ok = ok ? 1 : 0;
  if (!with_inverse) return;
  double A[3][3], b[3];
  for (int r = 0; r < 3; ++r) {
    for (int c = 0; c < 3; ++c) A[r][c] = (double)vc.tq[r][c] * 0x1p-40;
    b[r] = (double)vc.tq[r][3] * 0x1p-40;
  }
  const double c00 = A[1][1] * A[2][2] - A[1][2] * A[2][1];
  const double c01 = A[1][2] * A[2][0] - A[1][0] * A[2][2];
  const double c02 = A[1][0] * A[2][1] - A[1][1] * A[2][0];
  const double det = A[0][0] * c00 + A[0][1] * c01 + A[0][2] * c02;
  vc.inv_ok = fabs(det) > 1e-6 ? 1 : 0;
  const double id = vc.inv_ok ? 1.0 / det : 0.0;
  vc.ainv[0][0] = c00 * id;
  vc.ainv[1][0] = c01 * id;
  vc.ainv[2][0] = c02 * id;
  vc.ainv[0][1] = (A[0][2] * A[2][1] - A[0][1] * A[2][2]) * id;
  vc.ainv[1][1] = (A[0][0] * A[2][2] - A[0][2] * A[2][0]) * id;
  vc.ainv[2][1] = (A[0][1] * A[2][0] - A[0][0] * A[2][1]) * id;
  vc.ainv[0][2] = (A[0][1] * A[1][2] - A[0][2] * A[1][1]) * id;
  vc.ainv[1][2] = (A[0][2] * A[1][0] - A[0][0] * A[1][2]) * id;
  vc.ainv[2][2] = (A[0][0] * A[1][1] - A[0][1] * A[1][0]) * id;
  for (int c = 0; c < 3; ++c) {
    vc.binv[c] = -(vc.ainv[c][0] * b[0] + vc.ainv[c][1] * b[1] + vc.ainv[c][2] * b[2]);
    // a margin far above the rounding of the box centre (below 1e-3 voxel)
    vc.inv_h[c] =
        (float)(fabs(vc.ainv[c][0]) + fabs(vc.ainv[c][1]) + fabs(vc.ainv[c][2])) + 0.02f;
  }
}

// ---- Q.40 coordinate helpers ------------------------------------------------
__device__ __forceinline__ int q40_hi(long long s) { return (int)(s >> 32); }
// floor(s)
__device__ __forceinline__ int q40_floor(long long s) { return q40_hi(s) >> 8; }
// floor(s + 1/2): adding 2^39 only touches the high word.
__device__ __forceinline__ int q40_round(long long s) { return (q40_hi(s) + 128) >> 8; }
// s - floor(s), truncated to 23 bits (error < 2^-23): the top 23 fractional
// bits become the mantissa of a float in [1, 2), minus 1 (exact).
__device__ __forceinline__ float q40_one_plus_frac(long long s) {
  const unsigned m = (unsigned)((unsigned long long)s >> 17) & 0x7FFFFFu;
  return __uint_as_float(0x3F800000u | m);
}
__device__ __forceinline__ float q40_frac(long long s) { return q40_one_plus_frac(s) - 1.0f; }
// Bit 39 of s: 1 when frac(s) >= 1/2, i.e. floor(s + 1/2) = floor(s) + bit.
__device__ __forceinline__ int q40_halfbit(long long s) { return (q40_hi(s) >> 7) & 1; }

template <typename T>
__device__ __forceinline__ float ld_val(const T* p);
template <>
__device__ __forceinline__ float ld_val<float>(const float* p) {
  return __ldg(p);
}
template <>
__device__ __forceinline__ float ld_val<int16_t>(const int16_t* p) {
  return (float)__ldg(p);
}

// ---- fire-and-forget reductions -------------------------------------------------
// atomicAdd with an unused result may still be emitted as a returning atomic,
// whose destination register the warp then waits for; the reduction forms
// below never return a value.
__device__ __forceinline__ void red_add_global(float* p, float v) {
  asm volatile("red.global.add.f32 [%0], %1;" ::"l"(p), "f"(v) : "memory");
}
__device__ __forceinline__ void red_add_shared(float* p, float v) {
  asm volatile("red.shared.add.f32 [%0], %1;" ::"r"((unsigned)__cvta_generic_to_shared(p)),
               "f"(v)
               : "memory");
}
// Predicated forms: the reduction is issued only where pred holds, under a
// predicate inside the instruction rather than a branch around it (the
// address is formed either way and must only be valid where pred holds).
__device__ __forceinline__ void red_add_global_if(float* p, float v, bool pred) {
  asm volatile(
      "{\n\t.reg .pred q;\n\tsetp.ne.b32 q, %2, 0;\n\t@q red.global.add.f32 [%0], %1;\n\t}"
      ::"l"(p), "f"(v), "r"((int)pred)
      : "memory");
}
__device__ __forceinline__ void red_add_shared_if(float* p, float v, bool pred) {
  asm volatile(
      "{\n\t.reg .pred q;\n\tsetp.ne.b32 q, %2, 0;\n\t@q red.shared.add.f32 [%0], %1;\n\t}"
      ::"r"((unsigned)__cvta_generic_to_shared(p)), "f"(v), "r"((int)pred)
      : "memory");
}

// ---- packed FP32 pairs (sm_100+ f32x2 instructions) ----------------------------
// Two independent float lanes in one 64-bit register; each lane is rounded
// exactly like the scalar instruction, so packed and scalar code give
// bitwise-identical results.
typedef unsigned long long f32x2;
__device__ __forceinline__ f32x2 pk2(float lo, float hi) {
  f32x2 r;
  asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(lo), "f"(hi));
  return r;
}
__device__ __forceinline__ void upk2(f32x2 r, float& lo, float& hi) {
  asm("mov.b64 {%0, %1}, %2;" : "=f"(lo), "=f"(hi) : "l"(r));
}
__device__ __forceinline__ f32x2 fma2(f32x2 a, f32x2 b, f32x2 c) {
  f32x2 d;
  asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(d) : "l"(a), "l"(b), "l"(c));
  return d;
}
__device__ __forceinline__ f32x2 sub2(f32x2 a, f32x2 b) {
  f32x2 d;
  asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
  return d;
}
// Fractions of two Q.40 coordinates, packed (see q40_frac).
__device__ __forceinline__ f32x2 q40_frac2(long long s0, long long s1) {
  const unsigned m0 = (unsigned)((unsigned long long)s0 >> 17) & 0x7FFFFFu;
  const unsigned m1 = (unsigned)((unsigned long long)s1 >> 17) & 0x7FFFFFu;
  return sub2(pk2(__uint_as_float(0x3F800000u | m0), __uint_as_float(0x3F800000u | m1)),
              pk2(1.0f, 1.0f));
}

// ---- Philox4x32-10 (Salmon et al., SC'11) -----------------------------------
// Round: (hi0, lo0) = M0 * c0, (hi1, lo1) = M1 * c2;
//        c <- (hi1 ^ c1 ^ k0, lo1, hi0 ^ c3 ^ k1, lo0); key += Weyl constants.
__device__ __forceinline__ uint4 philox4x32_10(uint4 c, unsigned k0, unsigned k1) {
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    if (r > 0) {
      k0 += 0x9E3779B9u;
      k1 += 0xBB67AE85u;
    }
    const unsigned long long p0 = (unsigned long long)0xD2511F53u * c.x;
    const unsigned long long p1 = (unsigned long long)0xCD9E8D57u * c.z;
    c = make_uint4((unsigned)(p1 >> 32) ^ c.y ^ k0, (unsigned)p1, (unsigned)(p0 >> 32) ^ c.w ^ k1,
                   (unsigned)p0);
  }
  return c;
}

// The ten round keys of a Philox4x32-10 key.  They depend only on the seed:
// the host computes them and passes them to the noise kernels as a by-value
// parameter, so each round's XOR reads its key from the constant bank instead
// of recomputing k + r * Weyl in registers on every call.
struct PhiloxKey {
  unsigned k0[10], k1[10];
};
__host__ __device__ __forceinline__ PhiloxKey philox_schedule(unsigned k0, unsigned k1) {
  PhiloxKey k;
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    k.k0[r] = k0 + (unsigned)r * 0x9E3779B9u;
    k.k1[r] = k1 + (unsigned)r * 0xBB67AE85u;
  }
  return k;
}
// The same rounds as philox4x32_10 with the scheduled keys.
__device__ __forceinline__ uint4 philox4x32_10(uint4 c, const PhiloxKey& key) {
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    const unsigned long long p0 = (unsigned long long)0xD2511F53u * c.x;
    const unsigned long long p1 = (unsigned long long)0xCD9E8D57u * c.z;
    c = make_uint4((unsigned)(p1 >> 32) ^ c.y ^ key.k0[r], (unsigned)p1,
                   (unsigned)(p0 >> 32) ^ c.w ^ key.k1[r], (unsigned)p0);
  }
  return c;
}

// Streaming byte store to global memory.
__device__ __forceinline__ void st_cs_u8(uint8_t* p, int v) {
  asm volatile("st.global.cs.u8 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

// Documented approximate PTX instructions (special-function unit).
__device__ __forceinline__ float lg2_approx(float x) {
  float r;
  asm("lg2.approx.f32 %0, %1;" : "=f"(r) : "f"(x));
  return r;
}
__device__ __forceinline__ float ex2_approx(float x) {
  float r;
  asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
  return r;
}
// Flush-to-zero forms, for arguments that are never subnormal: they give the
// same results as the plain forms there and skip the subnormal fix-up code
// that the plain forms carry around the hardware instruction.
__device__ __forceinline__ float lg2_approx_ftz(float x) {
  float r;
  asm("lg2.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
  return r;
}
__device__ __forceinline__ float sqrt_approx_ftz(float x) {
  float r;
  asm("sqrt.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
  return r;
}
__device__ __forceinline__ float sin_approx_ftz(float x) {
  float r;
  asm("sin.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
  return r;
}
__device__ __forceinline__ float cos_approx_ftz(float x) {
  float r;
  asm("cos.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
  return r;
}

// Box-Muller on one pair of words: (R cos 2 pi u2, R sin 2 pi u2) with
// u1 = ((ra >> 8) + 1) 2^-24 in (0, 1], u2 = (rb >> 8) 2^-24 in [0, 1),
// R = sqrt(-2 ln u1).
//
// -2 ln u1: for v = 1 - u1 < 2^-6 (exact in float) the series
// v (2 + v (1 + 2v/3)) (Taylor series of -2 ln(1 - v), relative truncation
// error < v^3/2 < 2e-6, i.e. < 2e-7 absolute on R <= 0.18) keeps full
// accuracy where R is small; otherwise -2 ln 2 * log2(u1) with the hardware log2 (absolute error
// ~2^-22), which changes R by < 1e-6 there since R > 0.17.  R uses the
// hardware square root (relative error ~2^-23).  The angle is
// a = 2 pi u2 - pi in [-pi, pi), where the hardware sine/cosine have absolute
// error ~2^-21, and cos(2 pi u2) = -cos a, sin(2 pi u2) = -sin a.  Overall
// |n - n_exact| < ~5e-6 for |n| <= 5.8, i.e. < 2.5e-4 HU at sigma = 50.
// No argument of the hardware functions is subnormal (u1 >= 2^-24; x is 0 or
// >= 2^-23; a is 0 or |a| >= 2^-22), so their flush-to-zero forms are exact
// stand-ins for the plain ones.
__device__ __forceinline__ float2 box_muller(unsigned ra, unsigned rb) {
  const unsigned m1 = ra >> 8, m2 = rb >> 8;
  const float u1 = (float)(m1 + 1u) * 5.9604644775390625e-8f;
  const float v = 1.0f - u1;  // exact: u1 lies on the 2^-24 grid of (0, 1]
  const float series = v * fmaf(v, fmaf(v, 0.666666667f, 1.0f), 2.0f);
  const float x = (v < 0.015625f) ? series : -1.38629436112f * lg2_approx_ftz(u1);
  const float r = sqrt_approx_ftz(x);
  // (m2 2^-24) 2 pi rounds like m2 (2 pi 2^-24): scaling by 2^-24 is exact.
  const float a = fmaf((float)m2, 6.28318530718f * 5.9604644775390625e-8f, -3.14159265359f);
  return make_float2(-r * cos_approx_ftz(a), -r * sin_approx_ftz(a));
}

// Four normals of one quad (lanes 0..3).
__device__ __forceinline__ void quad_normals(unsigned long long quad, unsigned noise_id,
                                             const PhiloxKey& key, float z[4]) {
  const uint4 r = philox4x32_10(
      make_uint4((unsigned)quad, (unsigned)(quad >> 32), noise_id, 0u), key);
  const float2 p = box_muller(r.x, r.y), q = box_muller(r.z, r.w);
  z[0] = p.x;
  z[1] = p.y;
  z[2] = q.x;
  z[3] = q.y;
}

__device__ __forceinline__ float warp_sum(float v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(FULL_MASK, v, o);
  return v;
}

// Static round-robin tile schedule over the concatenated tile lists of all
// volumes: CTA b of G takes global tiles b, b + G, ...  For a volume whose
// tiles start at global index `base`, returns the first local tile of this CTA.
__device__ __forceinline__ long long first_tile(long long base) {
  const long long G = gridDim.x;
  return ((long long)blockIdx.x - base % G + G) % G;
}

}  // namespace augk
