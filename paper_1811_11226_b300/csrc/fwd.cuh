// Direct-gather forward of one output tile (Sec. 4): affine coordinate map,
// trilinear image sample, nearest label sample, intensity affine, Philox
// noise.  Shared by the flat-tile kernels (fwd.cu) and, for tiles whose input
// footprint does not fit a shared-memory brick, the brick kernel
// (fwd_brick.cu).
//
// Each thread walks its z-run one quad (4 z-consecutive voxels, one Philox
// call) at a time.  The warp re-classifies every quad (interior / exterior /
// general, from the quad's first and last coordinates), so only quads that
// actually straddle the input boundary pay for per-tap checks.
#pragma once

#include "kernels.h"
#include "sample.cuh"
#include "sched.cuh"

namespace augk {

// Per-tile copy of the volume constants, held in registers.
template <typename TIn>
struct FwdP {
  const TIn* img;
  const uint8_t* lab;
  float* oimg;
  uint8_t* olab;
  long long dx, dy, dz;
  int nx, ny, nz, nxy, plane, fill_label;
  float a, b, sigma, fill, yfill;  // yfill = a * fill + b
  int klo, khi;                    // occluded output z indices (empty if klo > khi)
  bool window;                     // clamp the output to [0, 1] after the noise
};

// Final value of one output voxel: occluded voxels are exactly 0 (nothing
// after the warp applies to them); otherwise the optional window clamp.
// POST = false (a run that meets neither) compiles to nothing.
template <bool POST, typename TIn>
__device__ __forceinline__ float finish(const FwdP<TIn>& P, int k, float y) {
  if (!POST) return y;
  if (k >= P.klo && k <= P.khi) return 0.0f;
  return P.window ? __saturatef(y) : y;
}
template <bool POST, typename TIn>
__device__ __forceinline__ bool occluded(const FwdP<TIn>& P, int k) {
  return POST && k >= P.klo && k <= P.khi;
}

// Exterior quad: every tap reads the fill value, so the sample is constant;
// only the noise differs per voxel.  The coordinate advances by n steps at once.
template <bool POST, typename TIn, bool IMG, bool LAB>
__device__ __forceinline__ void fwd_quad_exterior(const FwdP<TIn>& P, int& o, int n, bool valid,
                                                  const float z[4], int kq) {
#pragma unroll
  for (int m = 0; m < 4; ++m) {
    if (m < n) {
      if (valid) {
        if (IMG) __stcs(P.oimg + o, finish<POST>(P, kq + m, fmaf(P.sigma, z[m], P.yfill)));
        if (LAB) st_cs_u8(P.olab + o, P.fill_label);
      }
      o += P.plane;
    }
  }
}

// Interior / general quad (n = 1..4 z-consecutive voxels, warp-uniform MODE),
// software-pipelined in groups of PD voxels: the coordinates are stepped
// once, every tap and label load of a group is issued before any of its
// samples is interpolated, and the quad's normals are computed while the
// first group's loads are in flight.  PD trades registers (occupancy) for
// memory-level parallelism; it is part of the kernel variant.
// The upper (z + 1) plane of the previous voxel's cell along an interior
// z-run: when the next voxel's cell is that cell moved by +1 in z (fx and fy
// unchanged), its lower four taps are these values and only the upper four
// are loaded (per lane; lanes that moved in x or y load all eight).
struct ZPlane {
  int base;  // cell index of the previous voxel (far out of range when none)
  float t[4];
};

template <bool POST, typename TIn, int MODE, bool IMG, bool LAB, bool FULL, int PD,
          bool ZR = false>
__device__ __forceinline__ void fwd_quad(const FwdP<TIn>& P, long long& sx, long long& sy,
                                         long long& sz, int& o, int n, bool valid,
                                         bool noisy, unsigned long long quad, unsigned noise_id,
                                         const PhiloxKey& key, int kq, ZPlane& zp) {
  float z[4] = {0.0f, 0.0f, 0.0f, 0.0f};
#pragma unroll
  for (int g0 = 0; g0 < 4; g0 += PD) {
    float tap[PD][8];
    float w[PD][3];
    int lab[PD];
#pragma unroll
    for (int i = 0; i < PD; ++i) {
      const int m = g0 + i;
      lab[i] = P.fill_label;
#pragma unroll
      for (int d = 0; d < 8; ++d) tap[i][d] = P.fill;
      w[i][0] = w[i][1] = w[i][2] = 0.0f;
      if (FULL || m < n) {
        const int fx = q40_floor(sx), fy = q40_floor(sy), fz = q40_floor(sz);
        const int hbx = q40_halfbit(sx), hby = q40_halfbit(sy), hbz = q40_halfbit(sz);
        // An occluded voxel skips the image fetch (warp-uniform: one k per warp).
        const bool fetch = !occluded<POST>(P, kq + m);
        if (IMG) {
          w[i][0] = q40_frac(sx);
          w[i][1] = q40_frac(sy);
          w[i][2] = q40_frac(sz);
        }
        if (MODE == MODE_INTERIOR) {
          // Interior cells lie inside the input: the index is non-negative, so
          // the addresses take it zero-extended.
          const int base = (fz * P.ny + fy) * P.nx + fx;
          if (IMG && fetch) {
            const TIn* p = P.img + (unsigned)base;
            if (ZR && base == zp.base + P.nxy) {
              tap[i][0] = zp.t[0];
              tap[i][1] = zp.t[1];
              tap[i][2] = zp.t[2];
              tap[i][3] = zp.t[3];
            } else {
              tap[i][0] = ld_val(p);
              tap[i][1] = ld_val(p + 1);
              tap[i][2] = ld_val(p + P.nx);
              tap[i][3] = ld_val(p + P.nx + 1);
            }
            tap[i][4] = ld_val(p + P.nxy);
            tap[i][5] = ld_val(p + P.nxy + 1);
            tap[i][6] = ld_val(p + P.nxy + P.nx);
            tap[i][7] = ld_val(p + P.nxy + P.nx + 1);
            if (ZR) {
              zp.base = base;
              zp.t[0] = tap[i][4];
              zp.t[1] = tap[i][5];
              zp.t[2] = tap[i][6];
              zp.t[3] = tap[i][7];
            }
          }
          if (LAB) lab[i] = __ldg(P.lab + (unsigned)(base + hbx + hby * P.nx + hbz * P.nxy));
        } else {
          if (IMG && fetch) {
            const bool x0 = (unsigned)fx < (unsigned)P.nx,
                       x1 = (unsigned)(fx + 1) < (unsigned)P.nx;
            const bool y0 = (unsigned)fy < (unsigned)P.ny,
                       y1 = (unsigned)(fy + 1) < (unsigned)P.ny;
            const bool z0 = (unsigned)fz < (unsigned)P.nz,
                       z1 = (unsigned)(fz + 1) < (unsigned)P.nz;
            // The cell index is formed in unsigned arithmetic (it wraps harmlessly
            // far outside) and sign-extended: for every tap inside the volume the
            // row pointers below plus 0 or 1 address it exactly, and a tap is only
            // dereferenced when it lies inside.
            const int b = (int)(((unsigned)fz * (unsigned)P.ny + (unsigned)fy) * (unsigned)P.nx +
                                (unsigned)fx);
            const TIn* r00 = P.img + b;
            const TIn* r10 = r00 + P.nx;
            const TIn* r01 = r00 + P.nxy;
            const TIn* r11 = r01 + P.nx;
            if (x0 && y0 && z0) tap[i][0] = ld_val(r00);
            if (x1 && y0 && z0) tap[i][1] = ld_val(r00 + 1);
            if (x0 && y1 && z0) tap[i][2] = ld_val(r10);
            if (x1 && y1 && z0) tap[i][3] = ld_val(r10 + 1);
            if (x0 && y0 && z1) tap[i][4] = ld_val(r01);
            if (x1 && y0 && z1) tap[i][5] = ld_val(r01 + 1);
            if (x0 && y1 && z1) tap[i][6] = ld_val(r11);
            if (x1 && y1 && z1) tap[i][7] = ld_val(r11 + 1);
          }
          if (LAB) {
            const int rx = fx + hbx, ry = fy + hby, rz = fz + hbz;
            if ((unsigned)rx < (unsigned)P.nx && (unsigned)ry < (unsigned)P.ny &&
                (unsigned)rz < (unsigned)P.nz)
              lab[i] = __ldg(P.lab + ((rz * P.ny + ry) * P.nx + rx));
          }
        }
        sx += P.dx;
        sy += P.dy;
        sz += P.dz;
      }
    }
    if (g0 == 0 && noisy) quad_normals(quad, noise_id, key, z);
    if (FULL && IMG && PD >= 2) {
      // Voxel pairs share packed f32x2 instructions (same rounding as scalar).
#pragma unroll
      for (int i = 0; i < PD; i += 2) {
        const int m = g0 + i;
        const f32x2 tx = pk2(w[i][0], w[i + 1][0]), ty = pk2(w[i][1], w[i + 1][1]);
        const f32x2 tz = pk2(w[i][2], w[i + 1][2]);
        f32x2 v0[8];
#pragma unroll
        for (int d = 0; d < 8; ++d) v0[d] = pk2(tap[i][d], tap[i + 1][d]);
        const f32x2 c00 = fma2(tx, sub2(v0[1], v0[0]), v0[0]);
        const f32x2 c10 = fma2(tx, sub2(v0[3], v0[2]), v0[2]);
        const f32x2 c01 = fma2(tx, sub2(v0[5], v0[4]), v0[4]);
        const f32x2 c11 = fma2(tx, sub2(v0[7], v0[6]), v0[6]);
        const f32x2 c0 = fma2(ty, sub2(c10, c00), c00);
        const f32x2 c1 = fma2(ty, sub2(c11, c01), c01);
        const f32x2 v = fma2(tz, sub2(c1, c0), c0);
        const f32x2 y = fma2(pk2(P.sigma, P.sigma), pk2(z[m], z[m + 1]),
                             fma2(pk2(P.a, P.a), v, pk2(P.b, P.b)));
        float y0, y1;
        upk2(y, y0, y1);
        y0 = finish<POST>(P, kq + m, y0);
        y1 = finish<POST>(P, kq + m + 1, y1);
        if (valid) {
          __stcs(P.oimg + o, y0);
          if (LAB) st_cs_u8(P.olab + o, lab[i]);
          __stcs(P.oimg + o + P.plane, y1);
          if (LAB) st_cs_u8(P.olab + o + P.plane, lab[i + 1]);
        }
        o += 2 * P.plane;
      }
      continue;
    }
#pragma unroll
    for (int i = 0; i < PD; ++i) {
      const int m = g0 + i;
      if (FULL || m < n) {
        if (IMG) {
          const float tx = w[i][0], ty = w[i][1], tz = w[i][2];
          const float c00 = fmaf(tx, tap[i][1] - tap[i][0], tap[i][0]);
          const float c10 = fmaf(tx, tap[i][3] - tap[i][2], tap[i][2]);
          const float c01 = fmaf(tx, tap[i][5] - tap[i][4], tap[i][4]);
          const float c11 = fmaf(tx, tap[i][7] - tap[i][6], tap[i][6]);
          const float c0 = fmaf(ty, c10 - c00, c00);
          const float c1 = fmaf(ty, c11 - c01, c01);
          const float v = fmaf(tz, c1 - c0, c0);
          if (valid)
            __stcs(P.oimg + o, finish<POST>(P, kq + m, fmaf(P.sigma, z[m], fmaf(P.a, v, P.b))));
        }
        if (LAB && valid) st_cs_u8(P.olab + o, lab[i]);
        o += P.plane;
      }
    }
  }
}

// Quad-by-quad walk of a z-run: every quad is classified on its own (warp
// vote), so a run that straddles the input boundary pays per-tap checks only
// where needed.
template <bool POST, typename TIn, int QZ, int PD, bool IMG, bool LAB>
__device__ __forceinline__ void fwd_quads(const FwdP<TIn>& P, const TileCoord& tc, long long sx,
                                          long long sy, long long sz, int o, bool noisy,
                                          unsigned onx, unsigned ony, unsigned noise_id,
                                          const PhiloxKey& key) {
  const long long ds[3] = {P.dx, P.dy, P.dz};
#pragma unroll 1
  for (int q = 0; q < QZ; ++q) {
    const int kq = tc.k0 + 4 * q;
    if (kq >= tc.k1) break;
    const int n = min(4, tc.k1 - kq);
    const unsigned long long quad =
        ((unsigned long long)(kq >> 2) * ony + (unsigned)tc.jc) * onx + (unsigned)tc.ic;
    const long long s[3] = {sx, sy, sz};
    const int mode = warp_mode(classify_run<true>(s, ds, n - 1, P.nx, P.ny, P.nz));
    if (mode == MODE_EXTERIOR) {
      float z[4] = {0.0f, 0.0f, 0.0f, 0.0f};
      if (noisy) quad_normals(quad, noise_id, key, z);
      fwd_quad_exterior<POST, TIn, IMG, LAB>(P, o, n, tc.valid, z, kq);
      sx += (long long)n * P.dx;
      sy += (long long)n * P.dy;
      sz += (long long)n * P.dz;
    } else if (n == 4) {
      ZPlane none;
      if (mode == MODE_INTERIOR)
        fwd_quad<POST, TIn, MODE_INTERIOR, IMG, LAB, true, PD>(
            P, sx, sy, sz, o, 4, tc.valid, noisy, quad, noise_id, key, kq, none);
      else
        fwd_quad<POST, TIn, MODE_GENERAL, IMG, LAB, true, PD>(
            P, sx, sy, sz, o, 4, tc.valid, noisy, quad, noise_id, key, kq, none);
    } else {
      ZPlane none;
      fwd_quad<POST, TIn, MODE_GENERAL, IMG, LAB, false, PD>(
          P, sx, sy, sz, o, n, tc.valid, noisy, quad, noise_id, key, kq, none);
    }
  }
}

// Direct-gather forward of one tile whose thread coordinates are tc (any
// lane mapping; the z-run of every thread is tc.k0 .. tc.k1 - 1, at most
// 4*QZ voxels, starting on a quad boundary).  ZR: the z + 1 plane reuse along
// fully interior runs.
template <typename TIn, int QZ, int PD, bool IMG, bool LAB, bool ZR = false>
__device__ __forceinline__ void fwd_tile_tc(const VolConst& vc, const TileCoord& tc,
                                            const PhiloxKey& key) {
  FwdP<TIn> P;
  P.img = (const TIn*)vc.image;
  P.lab = vc.label;
  P.oimg = vc.out_image;
  P.olab = vc.out_label;
  P.dx = vc.tq[0][2];
  P.dy = vc.tq[1][2];
  P.dz = vc.tq[2][2];
  P.nx = vc.nx;
  P.ny = vc.ny;
  P.nz = vc.nz;
  P.nxy = vc.nx * vc.ny;
  P.plane = vc.onx * vc.ony;
  P.fill_label = vc.fill_label;
  P.a = vc.a;
  P.b = vc.b;
  P.sigma = vc.sigma;
  P.fill = vc.fill;
  P.yfill = fmaf(vc.a, vc.fill, vc.b);
  P.klo = vc.occ_klo;
  P.khi = vc.occ_khi;
  P.window = (vc.flags & AUG_FLAG_WINDOW) != 0;
  const unsigned noise_id = vc.noise_id;
  const bool noisy = IMG && vc.sigma > 0.0f;
  const unsigned onx = (unsigned)vc.onx, ony = (unsigned)vc.ony;
  long long sx = coord_q40(vc.tq[0], tc.ic, tc.jc, tc.k0);
  long long sy = coord_q40(vc.tq[1], tc.ic, tc.jc, tc.k0);
  long long sz = coord_q40(vc.tq[2], tc.ic, tc.jc, tc.k0);
  const long long ds[3] = {P.dx, P.dy, P.dz};
  const int o = (tc.k0 * vc.ony + tc.jc) * vc.onx + tc.ic;
  // Occlusion and window are decided per run (the z-range is the same for the
  // whole CTA): runs that meet neither take the code without them.
  const bool post = P.window || (P.klo <= P.khi && P.klo < tc.k1 && P.khi >= tc.k0);
  if (!post) {
    // One warp vote for the whole z-run; quads are re-classified only when
    // the run straddles the input boundary.
    const long long s0[3] = {sx, sy, sz};
    const int run_mode =
        warp_mode(classify_run<true>(s0, ds, tc.k1 - 1 - tc.k0, P.nx, P.ny, P.nz));
    const bool full_run = tc.k1 - tc.k0 == 4 * QZ;
    int oo = o;
    if (run_mode == MODE_EXTERIOR) {
#pragma unroll 1
      for (int kq = tc.k0; kq < tc.k1; kq += 4) {
        const int n = min(4, tc.k1 - kq);
        float z[4] = {0.0f, 0.0f, 0.0f, 0.0f};
        if (noisy)
          quad_normals(((unsigned long long)(kq >> 2) * ony + (unsigned)tc.jc) * onx +
                           (unsigned)tc.ic,
                       noise_id, key, z);
        fwd_quad_exterior<false, TIn, IMG, LAB>(P, oo, n, tc.valid, z, kq);
      }
      return;
    }
    if (run_mode == MODE_INTERIOR && full_run) {
      unsigned long long quad =
          ((unsigned long long)(tc.k0 >> 2) * ony + (unsigned)tc.jc) * onx + (unsigned)tc.ic;
      const unsigned long long quad_step = (unsigned long long)onx * ony;
      ZPlane zp;
      zp.base = -0x40000000;  // no previous cell
#pragma unroll 1
      for (int kq = tc.k0; kq < tc.k1; kq += 4, quad += quad_step)
        fwd_quad<false, TIn, MODE_INTERIOR, IMG, LAB, true, PD, ZR>(
            P, sx, sy, sz, oo, 4, tc.valid, noisy, quad, noise_id, key, kq, zp);
      return;
    }
    fwd_quads<false, TIn, QZ, PD, IMG, LAB>(P, tc, sx, sy, sz, o, noisy, onx, ony, noise_id,
                                            key);
  } else {
    fwd_quads<true, TIn, QZ, PD, IMG, LAB>(P, tc, sx, sy, sz, o, noisy, onx, ony, noise_id,
                                           key);
  }
}

// Direct-gather forward of one tile, any input type and output set.
template <int QZ, int PD, bool ZR = false>
__device__ __forceinline__ void fwd_tile_direct(const VolConst& vc, const TileCoord& tc,
                                                const PhiloxKey& key) {
  const bool img = vc.out_image != nullptr, lab = vc.out_label != nullptr;
  if (vc.dtype == AUG_I16) {
    if (img && lab)
      fwd_tile_tc<int16_t, QZ, PD, true, true, ZR>(vc, tc, key);
    else if (img)
      fwd_tile_tc<int16_t, QZ, PD, true, false, ZR>(vc, tc, key);
    else
      fwd_tile_tc<int16_t, QZ, PD, false, true, ZR>(vc, tc, key);
  } else {
    if (img && lab)
      fwd_tile_tc<float, QZ, PD, true, true, ZR>(vc, tc, key);
    else if (img)
      fwd_tile_tc<float, QZ, PD, true, false, ZR>(vc, tc, key);
    else
      fwd_tile_tc<float, QZ, PD, false, true, ZR>(vc, tc, key);
  }
}

// Tile t of the flat plane mapping (tile_coord_flat).
template <int NW, int QZ, int PD, bool ZR = false>
__device__ __forceinline__ void fwd_tile(const VolConst& vc, int t, const PhiloxKey& key) {
  fwd_tile_direct<QZ, PD, ZR>(vc, tile_coord_flat<NW, QZ>(t, vc.onx, vc.ony, vc.onz), key);
}

}  // namespace augk
