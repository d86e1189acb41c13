// Fused nearest-label warp + overlap loss (soft IOU or Dice, Sec. 5.C), forward
// and backward.
//
//   pass 1 (k_iou_pass<SUMS=true>): per output voxel, the warped label y is
//       computed in registers (exact Q.40 coordinate, floor(s + 1/2)) and the
//       class inputs x[c] are streamed once; they become q[c] (see XF below)
//       and per class the sums I = sum q [y == c], P = sum q, Y = sum [y == c]
//       are reduced per tile (warp shuffles, then a fixed-order block sum in
//       double) and per CTA, and written to workspace partials
//       [CTA][volume][3C].
//   finalize (k_iou_finalize): one CTA per volume sums the partials over CTAs
//       in a fixed order, writes loss[b] = mean_c L_c and the two values of
//       dL/dq of each class: one for the voxels of the class, one for the
//       others (IOU: -s/U and s I/U^2; Dice: s (2I - 2D)/D^2 and s 2I/D^2,
//       U = P + Y - I, D = P + Y, s = 1/(B C)).
//   pass 2 (k_iou_pass<SUMS=false>): recomputes the label and writes the
//       gradient.  For plain probabilities that is a write-only stream (x is
//       not re-read); the transforms re-read x.
// The warped labels never reach memory.
//
// Input transform XF (bit mask):
//   0             q = x                                (probabilities)
//   XF_POW        q = x^m, m > 0                       (the L^m family)
//   XF_LOGITS     q = softmax over the classes of x    (class scores)
//   both          q = softmax(x)^m
// The gradient pass applies the chain rule of the transform:
//   dL/dp_c = dL/dq_c * m p_c^(m-1), and for scores
//   dL/dx_c = p_c (dL/dp_c - sum_j p_j dL/dp_j).
#pragma once

#include "kernels.h"
#include "sample.cuh"
#include "sched.cuh"

namespace augk {

enum { XF_POW = 1, XF_LOGITS = 2 };

// p^m for p >= 0, m > 0: products for m = 2, 3, 4 (the kernel argument m is
// uniform, so the choice is a uniform branch), else hardware log2/exp2 (0 at
// p = 0).
__device__ __forceinline__ float pow_pos(float p, float m) {
  if (m == 2.0f) return p * p;
  if (m == 3.0f) return p * p * p;
  if (m == 4.0f) {
    const float q = p * p;
    return q * q;
  }
  return p > 0.0f ? ex2_approx(m * lg2_approx(p)) : 0.0f;
}
// d(p^m)/dp = m p^(m-1); at p = 0: 0 (m > 1), 1 (m = 1), +inf (m < 1).
__device__ __forceinline__ float dpow_pos(float p, float m) {
  if (m == 2.0f) return 2.0f * p;
  if (m == 3.0f) return 3.0f * (p * p);
  if (m == 4.0f) return 4.0f * (p * p * p);
  if (p > 0.0f) return m * ex2_approx((m - 1.0f) * lg2_approx(p));
  return m > 1.0f ? 0.0f : (m == 1.0f ? 1.0f : __int_as_float(0x7f800000));
}

// Loads the C class inputs of one voxel and returns p (the probabilities after
// the optional softmax) and q (after the optional power).
template <int C, int XF>
__device__ __forceinline__ void loss_inputs(const float* __restrict__ x, int nvox, int o,
                                            float m, float pr[C], float q[C]) {
  float v[C];
#pragma unroll
  for (int c = 0; c < C; ++c) v[c] = __ldcs(x + (size_t)c * nvox + o);
  if (XF & XF_LOGITS) {
    float mx = v[0];
#pragma unroll
    for (int c = 1; c < C; ++c) mx = fmaxf(mx, v[c]);
    float z = 0.0f;
#pragma unroll
    for (int c = 0; c < C; ++c) {
      v[c] = ex2_approx((v[c] - mx) * 1.4426950408889634f);  // exp(x - max), in (0, 1]
      z += v[c];
    }
    const float r = __frcp_rn(z);  // z >= 1
#pragma unroll
    for (int c = 0; c < C; ++c) pr[c] = v[c] * r;
  } else {
#pragma unroll
    for (int c = 0; c < C; ++c) pr[c] = v[c];
  }
#pragma unroll
  for (int c = 0; c < C; ++c) q[c] = (XF & XF_POW) ? pow_pos(pr[c], m) : pr[c];
}

template <int MODE, int C, bool SUMS, int XF>
__device__ __forceinline__ void iou_run(const VolConst& vc, const TileCoord& tc, long long sx,
                                        long long sy, long long sz,
                                        const float* __restrict__ p, float* __restrict__ gp,
                                        const float2* __restrict__ cf, float m,
                                        float acc[3 * C]) {
  const long long dx = vc.tq[0][2], dy = vc.tq[1][2], dz = vc.tq[2][2];
  const int plane = vc.onx * vc.ony;
  const int nvox = plane * vc.onz;
  int o = (tc.k0 * vc.ony + tc.jc) * vc.onx + tc.ic;
  float2 coef[C];
  if (!SUMS) {
#pragma unroll
    for (int c = 0; c < C; ++c) coef[c] = cf[c];
  }
#pragma unroll 4
  for (int k = tc.k0; k < tc.k1; ++k) {
    const int y = load_label<MODE>(vc.label, sx, sy, sz, vc.nx, vc.ny, vc.nz, vc.fill_label);
    if (tc.valid) {
      if (XF == 0 && SUMS) {
#pragma unroll
        for (int c = 0; c < C; ++c) {
          const float pc = __ldcs(p + (size_t)c * nvox + o);
          const bool hit = y == c;
          acc[3 * c + 0] += hit ? pc : 0.0f;
          acc[3 * c + 1] += pc;
          acc[3 * c + 2] += hit ? 1.0f : 0.0f;
        }
      } else if (XF == 0) {
#pragma unroll
        for (int c = 0; c < C; ++c)
          __stcs(gp + (size_t)c * nvox + o, y == c ? coef[c].y : coef[c].x);
      } else {
        float pr[C], q[C];
        loss_inputs<C, XF>(p, nvox, o, m, pr, q);
        if (SUMS) {
#pragma unroll
          for (int c = 0; c < C; ++c) {
            const bool hit = y == c;
            acc[3 * c + 0] += hit ? q[c] : 0.0f;
            acc[3 * c + 1] += q[c];
            acc[3 * c + 2] += hit ? 1.0f : 0.0f;
          }
        } else {
          float g[C];
#pragma unroll
          for (int c = 0; c < C; ++c) {
            const float gq = y == c ? coef[c].y : coef[c].x;
            // A zero coefficient (empty denominator) stays 0 even where the
            // power's derivative is infinite.
            g[c] = (XF & XF_POW) ? (gq == 0.0f ? 0.0f : gq * dpow_pos(pr[c], m)) : gq;
          }
          if (XF & XF_LOGITS) {
            float dot = 0.0f;
#pragma unroll
            for (int c = 0; c < C; ++c) dot = fmaf(pr[c], g[c], dot);
#pragma unroll
            for (int c = 0; c < C; ++c) g[c] = pr[c] * (g[c] - dot);
          }
#pragma unroll
          for (int c = 0; c < C; ++c) __stcs(gp + (size_t)c * nvox + o, g[c]);
        }
      }
    }
    sx += dx;
    sy += dy;
    sz += dz;
    o += plane;
  }
}

template <int NW, int C>
struct IouShared {
  float red[NW][3 * C];
  double acc[3 * C];
};

template <int NW, int QZ, int C, bool SUMS, int XF>
__global__ void __launch_bounds__(NW * 32)
    k_iou_pass(const aug_volume_desc* __restrict__ descs, int n_vols,
               const VolConst* __restrict__ tab, const float* __restrict__ p,
               float* __restrict__ gp, const float2* __restrict__ coefs, double* partials,
               float m) {
  __shared__ IouShared<NW, C> sh;
  __shared__ SchedSmem<NW * 32> sm;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  int staged = -1;
  // Threads 0..3C-1 own sh.acc: they zero, accumulate and flush it.
  auto flush = [&]() {
    if (SUMS && staged >= 0 && threadIdx.x < 3 * C)
      partials[((size_t)blockIdx.x * n_vols + staged) * (3 * C) + threadIdx.x] =
          sh.acc[threadIdx.x];
  };
  // Balanced tile order for the plain-probability passes (memory-bound); the
  // p^m and class-score passes, with their special-function work per class,
  // keep every CTA working (measured: 0.338 / 0.429 ms against 0.344 / 0.448 ms
  // balanced for the p^2 and softmax^2 IOU steps).
  for_each_tile<NW, QZ, false, XF == 0>(
      descs, n_vols, sm,
      [&](int c0, int cnt) {
        if (SUMS) {
          for (int i = threadIdx.x; i < cnt * 3 * C; i += blockDim.x)
            partials[((size_t)blockIdx.x * n_vols + c0) * (3 * C) + i] = 0.0;
          __syncthreads();
        }
      },
      [&](int v, int t, long long voxoff) {
        if (v != staged) {
          flush();
          if (SUMS && threadIdx.x < 3 * C) sh.acc[threadIdx.x] = 0.0;
          staged = v;
        }
        const VolConst& vc = tab[v];
        if (!vc.ok) return;
        const TileCoord tc = tile_coord<NW, QZ>(t, vc.onx, vc.ony, vc.onz);
        long long s[3], ds[3];
#pragma unroll
        for (int r = 0; r < 3; ++r) {
          s[r] = coord_q40(vc.tq[r], tc.ic, tc.jc, tc.k0);
          ds[r] = vc.tq[r][2];
        }
        float acc[3 * C];
#pragma unroll
        for (int i = 0; i < 3 * C; ++i) acc[i] = 0.0f;
        const int mode =
            warp_mode(classify_run<false>(s, ds, tc.k1 - 1 - tc.k0, vc.nx, vc.ny, vc.nz));
        const size_t poff = (size_t)C * (size_t)voxoff;
        const float* pv = p + poff;
        float* gv = SUMS ? nullptr : gp + poff;
        const float2* cf = SUMS ? nullptr : coefs + (size_t)v * C;
        if (mode == MODE_INTERIOR)
          iou_run<MODE_INTERIOR, C, SUMS, XF>(vc, tc, s[0], s[1], s[2], pv, gv, cf, m, acc);
        else if (mode == MODE_EXTERIOR)
          iou_run<MODE_EXTERIOR, C, SUMS, XF>(vc, tc, s[0], s[1], s[2], pv, gv, cf, m, acc);
        else
          iou_run<MODE_GENERAL, C, SUMS, XF>(vc, tc, s[0], s[1], s[2], pv, gv, cf, m, acc);
        if (SUMS) {
#pragma unroll
          for (int i = 0; i < 3 * C; ++i) {
            const float w = warp_sum(acc[i]);
            if (lane == 0) sh.red[warp][i] = w;
          }
          __syncthreads();
          if (threadIdx.x < 3 * C) {
            double tot = 0.0;
#pragma unroll
            for (int w = 0; w < NW; ++w) tot += (double)sh.red[w][threadIdx.x];
            sh.acc[threadIdx.x] += tot;
          }
          __syncthreads();
        }
      });
  flush();
}

// One CTA per volume: loss and the per-class values of dL/dq (x: other
// voxels, y: voxels of the class).  kind: AUG_LOSS_IOU or AUG_LOSS_DICE.
template <int C>
__global__ void k_iou_finalize(const double* __restrict__ partials, int n_ctas, int n_vols,
                               int kind, float* loss, float2* coefs) {
  __shared__ double tot[3 * C];
  const int v = blockIdx.x;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  for (int i = warp; i < 3 * C; i += blockDim.x >> 5) {
    double s = 0.0;
    for (int c = lane; c < n_ctas; c += 32)
      s += partials[((size_t)c * n_vols + v) * (3 * C) + i];
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) s += __shfl_xor_sync(FULL_MASK, s, off);
    if (lane == 0) tot[i] = s;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    const double scale = 1.0 / ((double)n_vols * (double)C);
    double lsum = 0.0;
    for (int c = 0; c < C; ++c) {
      const double I = tot[3 * c], P = tot[3 * c + 1], Y = tot[3 * c + 2];
      double l = 0.0, g_other = 0.0, g_class = 0.0;
      if (kind == AUG_LOSS_DICE) {
        const double D = P + Y;
        if (D > 0.0) {
          l = 1.0 - 2.0 * I / D;
          g_other = scale * 2.0 * I / (D * D);
          g_class = scale * (2.0 * I - 2.0 * D) / (D * D);
        }
      } else {
        const double U = P + Y - I;
        if (U > 0.0) {
          l = 1.0 - I / U;
          g_other = scale * I / (U * U);
          g_class = -scale / U;
        }
      }
      lsum += l;
      if (coefs) coefs[(size_t)v * C + c] = make_float2((float)g_other, (float)g_class);
    }
    loss[v] = (float)(lsum / C);
  }
}

// ---- kernel tables ---------------------------------------------------------------
using IouPassK = void (*)(const aug_volume_desc*, int, const VolConst*, const float*, float*,
                          const float2*, double*, float);
struct IouPasses {
  int nw, qz;
  IouPassK sums[8];  // by C - 1
  IouPassK grad[8];
};

// Tile shapes of the variants (warps along y, z-run per thread), in variant order.
#define AUGK_IOU_TILES(X) X(8, 4) X(4, 4) X(8, 8) X(4, 8)
constexpr int kIouVariants = 4;

// Pass kernels of transform XF for one variant.  Each transform is
// instantiated in its own translation unit (explicit instantiation below).
template <int XF>
const IouPasses& iou_passes(int variant) {
#define AUGK_IOU_K(NW, QZ, S)                                                             \
  {                                                                                       \
    k_iou_pass<NW, QZ, 1, S, XF>, k_iou_pass<NW, QZ, 2, S, XF>,                           \
        k_iou_pass<NW, QZ, 3, S, XF>, k_iou_pass<NW, QZ, 4, S, XF>,                       \
        k_iou_pass<NW, QZ, 5, S, XF>, k_iou_pass<NW, QZ, 6, S, XF>,                       \
        k_iou_pass<NW, QZ, 7, S, XF>, k_iou_pass<NW, QZ, 8, S, XF>                        \
  }
#define AUGK_IOU_V(NW, QZ) {NW, QZ, AUGK_IOU_K(NW, QZ, true), AUGK_IOU_K(NW, QZ, false)},
  static const IouPasses table[kIouVariants] = {AUGK_IOU_TILES(AUGK_IOU_V)};
#undef AUGK_IOU_V
#undef AUGK_IOU_K
  return table[variant];
}
extern template const IouPasses& iou_passes<0>(int);
extern template const IouPasses& iou_passes<XF_POW>(int);
extern template const IouPasses& iou_passes<XF_LOGITS>(int);
extern template const IouPasses& iou_passes<XF_LOGITS | XF_POW>(int);

}  // namespace augk
