// Per-tile geometry and per-voxel sampling shared by the forward, adjoint and
// IOU kernels.
//
// Thread mapping: a tile is 32 (x) * NW (y) * 4*QZ (z) output voxels.  Lane
// = x, warp = y, and each thread walks its z-run one voxel at a time, so a
// warp instruction touches 32 x-consecutive outputs (coalesced 128-byte
// stores, and gathers from a compact strip of the input).  Lanes beyond the
// output edge are clamped onto the last valid voxel and never store.
//
// Cell classification: along a z-run the coordinate is affine in k, so the
// floors of its first and last voxel bound every floor in between.  A warp
// whose runs keep all 8 taps inside the input takes the unpredicated
// INTERIOR path; one whose runs have every tap outside (on some axis) takes
// EXTERIOR (fill values, no loads); any other takes GENERAL (per-tap checks).
#pragma once

#include "common.cuh"

namespace augk {

enum { MODE_INTERIOR = 0, MODE_EXTERIOR = 1, MODE_GENERAL = 2 };

struct TileCoord {
  int i, j, ic, jc, k0, k1;
  bool valid;
};

template <int NW, int QZ>
__device__ __forceinline__ int tiles_in(int onx, int ony, int onz) {
  return ((onx + 31) / 32) * ((ony + NW - 1) / NW) * ((onz + 4 * QZ - 1) / (4 * QZ));
}

template <int NW, int QZ>
__device__ __forceinline__ TileCoord tile_coord(int t, int onx, int ony, int onz) {
  const int tx_n = (onx + 31) / 32, ty_n = (ony + NW - 1) / NW;
  const int tx = t % tx_n, ty = (t / tx_n) % ty_n, tz = t / (tx_n * ty_n);
  TileCoord c;
  c.i = tx * 32 + (int)(threadIdx.x & 31);
  c.j = ty * NW + (int)(threadIdx.x >> 5);
  c.valid = c.i < onx && c.j < ony;
  c.ic = min(c.i, onx - 1);
  c.jc = min(c.j, ony - 1);
  c.k0 = tz * 4 * QZ;
  c.k1 = min(c.k0 + 4 * QZ, onz);
  return c;
}

// Flat mapping (forward kernels): the tile's NW*32 threads take NW*32
// consecutive positions p = j*onx + i of the output plane (thread-fastest),
// times 4*QZ z values, so every warp is full whatever onx is (the 2-D tiles
// above leave onx mod 32 lanes of a row's last tile idle).  A warp still
// covers 32 memory-consecutive outputs, in at most two rows when onx >= 32.
template <int NW, int QZ>
__device__ __forceinline__ int tiles_in_flat(int onx, int ony, int onz) {
  return ((onx * ony + NW * 32 - 1) / (NW * 32)) * ((onz + 4 * QZ - 1) / (4 * QZ));
}

template <int NW, int QZ>
__device__ __forceinline__ TileCoord tile_coord_flat(int t, int onx, int ony, int onz) {
  const int plane = onx * ony;
  const int tp_n = (plane + NW * 32 - 1) / (NW * 32);
  const int tp = t % tp_n, tz = t / tp_n;
  const int p = tp * (NW * 32) + (int)threadIdx.x;
  TileCoord c;
  c.valid = p < plane;
  const int pc = min(p, plane - 1);
  c.jc = pc / onx;
  c.ic = pc - c.jc * onx;
  c.i = c.ic;
  c.j = c.jc;
  c.k0 = tz * 4 * QZ;
  c.k1 = min(c.k0 + 4 * QZ, onz);
  return c;
}

// Box tiles of TXW x (32 / TXW) * NW x 4 * QZ output voxels (x fastest, then y,
// then z): TXW lanes along x, 32 / TXW rows of the warp along y, warps stacked
// along y; each thread walks 4 * QZ z values.  TXW = 32 gives tile_coord's
// tiles in tile_coord's order.  Exact integer division (once per tile).
template <int TXW, int NW, int QZ>
__device__ __forceinline__ TileCoord box_tile_coord(int t, int onx, int ony, int onz) {
  constexpr int TX = TXW, TY = (32 / TXW) * NW, TZ = 4 * QZ;
  const int ntx = (onx + TX - 1) / TX, nty = (ony + TY - 1) / TY;
  const int q = t / ntx, tx = t - q * ntx, tz = q / nty, ty = q - tz * nty;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  TileCoord c;
  c.i = tx * TX + lane % TXW;
  c.j = ty * TY + warp * (32 / TXW) + lane / TXW;
  c.valid = c.i < onx && c.j < ony;
  c.ic = min(c.i, onx - 1);
  c.jc = min(c.j, ony - 1);
  c.k0 = tz * TZ;
  c.k1 = min(c.k0 + TZ, onz);
  return c;
}

// Q.40 coordinate of output voxel (i, j, k) along one axis.
__device__ __forceinline__ long long coord_q40(const long long (&tq)[4], int i, int j, int k) {
  return tq[0] * (long long)i + tq[1] * (long long)j + tq[2] * (long long)k + tq[3];
}

// Classify the z-run of n+1 voxels starting at coordinates s (step ds per k).
// TRILINEAR: taps floor(s) and floor(s)+1; else the nearest voxel
// floor(s + 1/2) only (label-only passes).
template <bool TRILINEAR>
__device__ __forceinline__ int classify_run(const long long s[3], const long long ds[3], int n,
                                            int nx, int ny, int nz) {
  const int dims[3] = {nx, ny, nz};
  bool inside = true, outside = false;
#pragma unroll
  for (int r = 0; r < 3; ++r) {
    const long long e = s[r] + (long long)n * ds[r];
    const int a = TRILINEAR ? q40_floor(s[r]) : q40_round(s[r]);
    const int b = TRILINEAR ? q40_floor(e) : q40_round(e);
    const int lo = min(a, b), hi = max(a, b);
    const int last = TRILINEAR ? dims[r] - 2 : dims[r] - 1;
    inside &= lo >= 0 && hi <= last;
    outside |= TRILINEAR ? (hi < -1 || lo > dims[r] - 1) : (hi < 0 || lo > dims[r] - 1);
  }
  return inside ? MODE_INTERIOR : (outside ? MODE_EXTERIOR : MODE_GENERAL);
}

// Warp-uniform mode: every lane must agree, else GENERAL.
__device__ __forceinline__ int warp_mode(int m) {
  if (__all_sync(FULL_MASK, m == MODE_INTERIOR)) return MODE_INTERIOR;
  if (__all_sync(FULL_MASK, m == MODE_EXTERIOR)) return MODE_EXTERIOR;
  return MODE_GENERAL;
}

// The 8 taps of the cell floor(s), with the fill value outside the input.
struct Taps {
  float v000, v100, v010, v110, v001, v101, v011, v111;
  float tx, ty, tz;
  int fx, fy, fz;
};

template <typename TIn, int MODE>
__device__ __forceinline__ void load_taps(const TIn* __restrict__ img, long long sx, long long sy,
                                          long long sz, int nx, int ny, int nz, float fill,
                                          Taps& t) {
  t.fx = q40_floor(sx);
  t.fy = q40_floor(sy);
  t.fz = q40_floor(sz);
  t.tx = q40_frac(sx);
  t.ty = q40_frac(sy);
  t.tz = q40_frac(sz);
  if (MODE == MODE_EXTERIOR) {
    t.v000 = t.v100 = t.v010 = t.v110 = t.v001 = t.v101 = t.v011 = t.v111 = fill;
    return;
  }
  const int nxy = nx * ny;
  if (MODE == MODE_INTERIOR) {
    const TIn* p = img + ((t.fz * ny + t.fy) * nx + t.fx);
    t.v000 = ld_val(p);
    t.v100 = ld_val(p + 1);
    t.v010 = ld_val(p + nx);
    t.v110 = ld_val(p + nx + 1);
    t.v001 = ld_val(p + nxy);
    t.v101 = ld_val(p + nxy + 1);
    t.v011 = ld_val(p + nxy + nx);
    t.v111 = ld_val(p + nxy + nx + 1);
  } else {
    const bool x0 = (unsigned)t.fx < (unsigned)nx, x1 = (unsigned)(t.fx + 1) < (unsigned)nx;
    const bool y0 = (unsigned)t.fy < (unsigned)ny, y1 = (unsigned)(t.fy + 1) < (unsigned)ny;
    const bool z0 = (unsigned)t.fz < (unsigned)nz, z1 = (unsigned)(t.fz + 1) < (unsigned)nz;
    // Unsigned arithmetic: wraps harmlessly when the cell is far outside; an
    // index is only dereferenced when its tap is inside the volume.
    const unsigned base = ((unsigned)t.fz * (unsigned)ny + (unsigned)t.fy) * (unsigned)nx +
                          (unsigned)t.fx;
    const unsigned ux = (unsigned)nx, uxy = (unsigned)nxy;
    t.v000 = (x0 && y0 && z0) ? ld_val(img + base) : fill;
    t.v100 = (x1 && y0 && z0) ? ld_val(img + (base + 1u)) : fill;
    t.v010 = (x0 && y1 && z0) ? ld_val(img + (base + ux)) : fill;
    t.v110 = (x1 && y1 && z0) ? ld_val(img + (base + ux + 1u)) : fill;
    t.v001 = (x0 && y0 && z1) ? ld_val(img + (base + uxy)) : fill;
    t.v101 = (x1 && y0 && z1) ? ld_val(img + (base + uxy + 1u)) : fill;
    t.v011 = (x0 && y1 && z1) ? ld_val(img + (base + uxy + ux)) : fill;
    t.v111 = (x1 && y1 && z1) ? ld_val(img + (base + uxy + ux + 1u)) : fill;
  }
}

// Trilinear combination, x then y then z (exact when t == 0).
__device__ __forceinline__ float trilerp(const Taps& t, float& c00, float& c10, float& c01,
                                         float& c11, float& c0, float& c1) {
  c00 = fmaf(t.tx, t.v100 - t.v000, t.v000);
  c10 = fmaf(t.tx, t.v110 - t.v010, t.v010);
  c01 = fmaf(t.tx, t.v101 - t.v001, t.v001);
  c11 = fmaf(t.tx, t.v111 - t.v011, t.v011);
  c0 = fmaf(t.ty, c10 - c00, c00);
  c1 = fmaf(t.ty, c11 - c01, c01);
  return fmaf(t.tz, c1 - c0, c0);
}

// Nearest label floor(s + 1/2); fill outside.
template <int MODE>
__device__ __forceinline__ int load_label(const uint8_t* __restrict__ lab, long long sx,
                                          long long sy, long long sz, int nx, int ny, int nz,
                                          int fill_label) {
  if (MODE == MODE_EXTERIOR) return fill_label;
  const int rx = q40_round(sx), ry = q40_round(sy), rz = q40_round(sz);
  if (MODE == MODE_INTERIOR) return __ldg(lab + ((rz * ny + ry) * nx + rx));
  const bool in = (unsigned)rx < (unsigned)nx && (unsigned)ry < (unsigned)ny &&
                  (unsigned)rz < (unsigned)nz;
  return in ? (int)__ldg(lab + ((rz * ny + ry) * nx + rx)) : fill_label;
}

}  // namespace augk
