// Adjoint of the image warp (the backward pass of the augmentation, which the
// paper does not have; it lets gradients reach the input volume and the 12
// affine parameters).
//
// For out(o) = a * sum_d w_d(o) V(f(o) + d) + b + sigma n(o):
//   grad_in[n]   += a g(o) w_d(o)                  (scatter, in-volume taps)
//   dv/ds_x       = lerp_z(lerp_y(V1yz - V0yz))     (x-differences of the cell)
//   dv/ds_y       = lerp_z(c1z - c0z),  dv/ds_z = c1 - c0   (from the lerps)
//   grad_T[r][c] += a g(o) dv/ds_r obar_c,  obar = (i, j, k, 1).
//
// This header holds the per-tile code shared by the kernels of bwd.cu and the
// brick adjoint of bwd_brick.cu.
//
// grad_in is accumulated with float atomics straight into the caller's
// buffer (zeroed first by k_zero_grad_in).  grad_T: per thread, S_r = sum
// a g dv_r and K_r = sum a g dv_r k over its z-run (i, j fixed); the tile's
// 12 sums (i S_r, j S_r, K_r, S_r) are warp-reduced, block-reduced in a
// fixed order, accumulated per CTA and volume in double, written to
// workspace partials [CTA][volume][12], and summed over CTAs in a fixed order
// by k_bwd_finalize: bitwise reproducible.
#pragma once

#include "kernels.h"
#include "sample.cuh"
#include "sched.cuh"

namespace augk {

// Scatter target of the input gradient: the caller's grad_in volume
// (global atomics), or a shared-memory brick covering the tile's input
// bounding box (shared atomics; index = x + y*bsy + z*bsz + boff).
struct BrickMap {
  float* brick;
  int bsy, bsz, boff;
};

// PR: every conditional reduction is issued under a predicate inside the
// instruction and the merges are selects, so the loop body has no divergent
// branches (no convergence barriers per voxel); the sums are the same.
// TXW: lanes per output row of the warp (32: one row; 8 or 16: box patches);
// the x-merge hands over only within a row segment.
template <typename TIn, int MODE, bool GIN, bool GT, bool SMEM, bool XM = false, bool PR = false,
          int TXW = 32>
__device__ __forceinline__ void bwd_run(const VolConst& vc, const TileCoord& tc, long long sx,
                                        long long sy, long long sz,
                                        const float* __restrict__ g, float* __restrict__ gin,
                                        const BrickMap& bm, float acc[6]) {
  const TIn* __restrict__ img = (const TIn*)vc.image;
  const long long dx = vc.tq[0][2], dy = vc.tq[1][2], dz = vc.tq[2][2];
  const int nx = vc.nx, ny = vc.ny, nz = vc.nz, nxy = nx * ny;
  const int plane = vc.onx * vc.ony;
  const float a = vc.a, fill = vc.fill;
  const int klo = vc.occ_klo, khi = vc.occ_khi;
  int o = (tc.k0 * vc.ony + tc.jc) * vc.onx + tc.ic;
  // Interior runs merge along z: when the next voxel's cell is the current
  // one moved by +1 in z, the four z+1 contributions of this voxel land on the
  // next voxel's four z taps; they are held in registers and added there
  // instead of being issued as separate reductions.
  float pend[4] = {0.f, 0.f, 0.f, 0.f};
  int pend_base = -1;
  const int sy_ = SMEM ? bm.bsy : nx, sz_ = SMEM ? bm.bsz : nxy;
  float* const tgt = SMEM ? bm.brick : gin;
#define RADD(p, v) (SMEM ? red_add_shared((p), (v)) : red_add_global((p), (v)))
#define RADD_IF(p, v, c) \
  (SMEM ? red_add_shared_if((p), (v), (c)) : red_add_global_if((p), (v), (c)))
#pragma unroll 4
  for (int k = tc.k0; k < tc.k1; ++k) {
    // An occluded output voxel is the constant 0: no gradient flows through it.
    const bool occ = k >= klo && k <= khi;
    const float ga = (tc.valid && !occ) ? a * __ldcs(g + o) : 0.0f;
    Taps t;
    load_taps<TIn, MODE>(img, sx, sy, sz, nx, ny, nz, fill, t);
    // With XM the interior branch runs in every lane of the warp (its shuffles
    // need them all); lanes outside the output only carry zeros and never
    // issue a reduction.
    if (GIN && (PR || tc.valid || (XM && MODE == MODE_INTERIOR))) {
      const float wx1 = t.tx, wx0 = 1.0f - t.tx, wy1 = t.ty, wy0 = 1.0f - t.ty;
      const float wz1 = t.tz, wz0 = 1.0f - t.tz;
      const float g00 = ga * wy0 * wz0, g10 = ga * wy1 * wz0;
      const float g01 = ga * wy0 * wz1, g11 = ga * wy1 * wz1;
      if (MODE == MODE_INTERIOR) {
        const int base = SMEM ? t.fx + t.fy * bm.bsy + t.fz * bm.bsz + bm.boff
                              : (t.fz * ny + t.fy) * nx + t.fx;
        float c0 = g00 * wx0, c1 = g00 * wx1, c2 = g10 * wx0, c3 = g10 * wx1;
        if (PR) {
          const bool merge = base == pend_base;
          const bool flush = !merge && pend_base >= 0 && tc.valid;
          float* q = tgt + pend_base;
          RADD_IF(q, pend[0], flush);
          RADD_IF(q + 1, pend[1], flush);
          RADD_IF(q + sy_, pend[2], flush);
          RADD_IF(q + sy_ + 1, pend[3], flush);
          c0 = merge ? c0 + pend[0] : c0;
          c1 = merge ? c1 + pend[1] : c1;
          c2 = merge ? c2 + pend[2] : c2;
          c3 = merge ? c3 + pend[3] : c3;
        } else if (base == pend_base) {
          c0 += pend[0];
          c1 += pend[1];
          c2 += pend[2];
          c3 += pend[3];
        } else if (pend_base >= 0 && tc.valid) {
          float* q = tgt + pend_base;
          RADD(q, pend[0]);
          RADD(q + 1, pend[1]);
          RADD(q + sy_, pend[2]);
          RADD(q + sy_ + 1, pend[3]);
        }
        float* p = tgt + base;
        if (XM) {
          // Merge along x: when the next lane's cell is this one moved by +1
          // in x, this lane's x+1 taps are its x taps; hand the two values
          // over instead of issuing them.
          const int lane = threadIdx.x & 31, lx = lane % TXW;
          const int nb = __shfl_down_sync(FULL_MASK, base, 1);
          const int nv = __shfl_down_sync(FULL_MASK, (int)tc.valid, 1);
          const bool give = tc.valid && lx < TXW - 1 && nv && nb == base + 1;
          const float l1 = __shfl_up_sync(FULL_MASK, c1, 1);
          const float l3 = __shfl_up_sync(FULL_MASK, c3, 1);
          const int lg = __shfl_up_sync(FULL_MASK, (int)give, 1);
          if (PR) {
            const bool take = lx > 0 && lg;
            c0 = take ? c0 + l1 : c0;
            c2 = take ? c2 + l3 : c2;
            RADD_IF(p, c0, tc.valid);
            RADD_IF(p + sy_, c2, tc.valid);
            RADD_IF(p + 1, c1, tc.valid && !give);
            RADD_IF(p + sy_ + 1, c3, tc.valid && !give);
          } else {
          if (lx > 0 && lg) {
            c0 += l1;
            c2 += l3;
          }
          if (tc.valid) {
            RADD(p, c0);
            RADD(p + sy_, c2);
            if (!give) {
              RADD(p + 1, c1);
              RADD(p + sy_ + 1, c3);
            }
          }
          }
        } else if (PR) {
          RADD_IF(p, c0, tc.valid);
          RADD_IF(p + 1, c1, tc.valid);
          RADD_IF(p + sy_, c2, tc.valid);
          RADD_IF(p + sy_ + 1, c3, tc.valid);
        } else {
          RADD(p, c0);
          RADD(p + 1, c1);
          RADD(p + sy_, c2);
          RADD(p + sy_ + 1, c3);
        }
        pend[0] = g01 * wx0;
        pend[1] = g01 * wx1;
        pend[2] = g11 * wx0;
        pend[3] = g11 * wx1;
        pend_base = base + sz_;
      } else {
        const bool x0 = (unsigned)t.fx < (unsigned)nx, x1 = (unsigned)(t.fx + 1) < (unsigned)nx;
        const bool y0 = (unsigned)t.fy < (unsigned)ny, y1 = (unsigned)(t.fy + 1) < (unsigned)ny;
        const bool z0 = (unsigned)t.fz < (unsigned)nz, z1 = (unsigned)(t.fz + 1) < (unsigned)nz;
        // Indices are formed in unsigned arithmetic (wrapping harmlessly far
        // outside) and only used for taps inside the volume.
        const unsigned base = SMEM ? (unsigned)(t.fx + t.fy * bm.bsy + t.fz * bm.bsz + bm.boff)
                                   : ((unsigned)t.fz * (unsigned)ny + (unsigned)t.fy) *
                                             (unsigned)nx + (unsigned)t.fx;
        const unsigned ux = (unsigned)sy_, uxy = (unsigned)sz_;
        if (PR) {
          const bool v = tc.valid;
          RADD_IF(tgt + base, g00 * wx0, v && x0 && y0 && z0);
          RADD_IF(tgt + (base + 1u), g00 * wx1, v && x1 && y0 && z0);
          RADD_IF(tgt + (base + ux), g10 * wx0, v && x0 && y1 && z0);
          RADD_IF(tgt + (base + ux + 1u), g10 * wx1, v && x1 && y1 && z0);
          RADD_IF(tgt + (base + uxy), g01 * wx0, v && x0 && y0 && z1);
          RADD_IF(tgt + (base + uxy + 1u), g01 * wx1, v && x1 && y0 && z1);
          RADD_IF(tgt + (base + uxy + ux), g11 * wx0, v && x0 && y1 && z1);
          RADD_IF(tgt + (base + uxy + ux + 1u), g11 * wx1, v && x1 && y1 && z1);
        } else {
        if (x0 && y0 && z0) RADD(tgt + base, g00 * wx0);
        if (x1 && y0 && z0) RADD(tgt + (base + 1u), g00 * wx1);
        if (x0 && y1 && z0) RADD(tgt + (base + ux), g10 * wx0);
        if (x1 && y1 && z0) RADD(tgt + (base + ux + 1u), g10 * wx1);
        if (x0 && y0 && z1) RADD(tgt + (base + uxy), g01 * wx0);
        if (x1 && y0 && z1) RADD(tgt + (base + uxy + 1u), g01 * wx1);
        if (x0 && y1 && z1) RADD(tgt + (base + uxy + ux), g11 * wx0);
        if (x1 && y1 && z1) RADD(tgt + (base + uxy + ux + 1u), g11 * wx1);
        }
      }
    }
    if (GT) {
      float c00, c10, c01, c11, c0, c1;
      trilerp(t, c00, c10, c01, c11, c0, c1);
      const float e0 = fmaf(t.ty, (t.v110 - t.v010) - (t.v100 - t.v000), t.v100 - t.v000);
      const float e1 = fmaf(t.ty, (t.v111 - t.v011) - (t.v101 - t.v001), t.v101 - t.v001);
      const float dvx = fmaf(t.tz, e1 - e0, e0);
      const float dvy = fmaf(t.tz, (c11 - c01) - (c10 - c00), c10 - c00);
      const float dvz = c1 - c0;
      const float kf = (float)k;
      acc[0] = fmaf(ga, dvx, acc[0]);
      acc[1] = fmaf(ga, dvy, acc[1]);
      acc[2] = fmaf(ga, dvz, acc[2]);
      acc[3] = fmaf(ga * dvx, kf, acc[3]);
      acc[4] = fmaf(ga * dvy, kf, acc[4]);
      acc[5] = fmaf(ga * dvz, kf, acc[5]);
    }
    sx += dx;
    sy += dy;
    sz += dz;
    o += plane;
  }
  if (GIN && MODE == MODE_INTERIOR && pend_base >= 0 && tc.valid) {
    float* q = tgt + pend_base;
    RADD(q, pend[0]);
    RADD(q + 1, pend[1]);
    RADD(q + sy_, pend[2]);
    RADD(q + sy_ + 1, pend[3]);
  }
#undef RADD
#undef RADD_IF
}

template <int NW>
struct BwdShared {
  float red[NW][12];
  double acc[12];
};

// Adds one tile's 12 affine-gradient sums to sh.acc: per thread S_r = sum a g
// dv_r and K_r = sum a g dv_r k over its z-run (acc), times (i, j, 1) and k;
// warp sums, then a fixed-order block sum in double.  All threads.
template <int NW>
__device__ __forceinline__ void bwd_reduce_tile(BwdShared<NW>& sh, const TileCoord& tc,
                                                const float acc[6]) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const float fi = (float)tc.ic, fj = (float)tc.jc;
  float v[12];
#pragma unroll
  for (int r = 0; r < 3; ++r) {
    v[4 * r + 0] = fi * acc[r];
    v[4 * r + 1] = fj * acc[r];
    v[4 * r + 2] = acc[3 + r];
    v[4 * r + 3] = acc[r];
  }
#pragma unroll
  for (int m = 0; m < 12; ++m) {
    const float w = warp_sum(v[m]);
    if (lane == 0) sh.red[warp][m] = w;
  }
  __syncthreads();
  if (threadIdx.x < 12) {
    double tot = 0.0;
#pragma unroll
    for (int w = 0; w < NW; ++w) tot += (double)sh.red[w][threadIdx.x];
    sh.acc[threadIdx.x] += tot;
  }
  __syncthreads();
}

// Adjoint of one tile whose thread coordinates are tc (any lane mapping), with
// this tile's 12 affine-gradient sums added to sh.acc in a fixed order.
// QS: runs that straddle the input boundary are re-classified per quad.
template <typename TIn, int NW, bool GIN, bool GT, bool SMEM = false, bool XM = false,
          bool QS = false, bool PR = false, int TXW = 32>
__device__ __forceinline__ void bwd_tile_tc(const VolConst& vc, BwdShared<NW>& sh,
                                            const TileCoord& tc, const float* g, float* gin,
                                            const BrickMap& bm = BrickMap{nullptr, 0, 0, 0}) {
  long long s[3], ds[3];
#pragma unroll
  for (int r = 0; r < 3; ++r) {
    s[r] = coord_q40(vc.tq[r], tc.ic, tc.jc, tc.k0);
    ds[r] = vc.tq[r][2];
  }
  float acc[6] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
  const int mode =
      warp_mode(classify_run<true>(s, ds, tc.k1 - 1 - tc.k0, vc.nx, vc.ny, vc.nz));
  // Exterior cells have all taps equal to the fill value: no gradient at all.
  if (mode == MODE_INTERIOR) {
    bwd_run<TIn, MODE_INTERIOR, GIN, GT, SMEM, XM, PR, TXW>(vc, tc, s[0], s[1], s[2], g, gin,
                                                            bm, acc);
  } else if (mode == MODE_GENERAL && QS && tc.k1 - tc.k0 > 4) {
    // A run that straddles the input boundary, re-classified quad by quad:
    // only the quads that do straddle it take the per-tap checks.
#pragma unroll 1
    for (int kq = tc.k0; kq < tc.k1; kq += 4) {
      TileCoord tq = tc;
      tq.k0 = kq;
      tq.k1 = min(kq + 4, tc.k1);
      const int mq =
          warp_mode(classify_run<true>(s, ds, tq.k1 - 1 - tq.k0, vc.nx, vc.ny, vc.nz));
      if (mq == MODE_INTERIOR)
        bwd_run<TIn, MODE_INTERIOR, GIN, GT, SMEM, XM, PR, TXW>(vc, tq, s[0], s[1], s[2], g, gin,
                                                                bm, acc);
      else if (mq == MODE_GENERAL)
        bwd_run<TIn, MODE_GENERAL, GIN, GT, SMEM, false, PR>(vc, tq, s[0], s[1], s[2], g, gin,
                                                             bm, acc);
#pragma unroll
      for (int r = 0; r < 3; ++r) s[r] += (long long)(tq.k1 - tq.k0) * ds[r];
    }
  } else if (mode == MODE_GENERAL) {
    bwd_run<TIn, MODE_GENERAL, GIN, GT, SMEM, false, PR>(vc, tc, s[0], s[1], s[2], g, gin, bm,
                                                         acc);
  }
  if (GT) bwd_reduce_tile<NW>(sh, tc, acc);
}

template <typename TIn, int NW, int QZ, bool GIN, bool GT, bool SMEM = false, bool XM = false,
          bool QS = false, bool PR = false, int TXW = 32>
__device__ __forceinline__ void bwd_tile(const VolConst& vc, BwdShared<NW>& sh, int t,
                                         const float* g, float* gin,
                                         const BrickMap& bm = BrickMap{nullptr, 0, 0, 0}) {
  bwd_tile_tc<TIn, NW, GIN, GT, SMEM, XM, QS, PR, TXW>(
      vc, sh, box_tile_coord<TXW, NW, QZ>(t, vc.onx, vc.ony, vc.onz), g, gin, bm);
}

}  // namespace augk
