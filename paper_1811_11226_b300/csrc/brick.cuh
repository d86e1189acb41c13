// Shared-memory bricks of a tile's input footprint, used by the brick forward
// (fwd_brick.cu) and the brick adjoint (bwd_brick.cu).
//
// A tile is a box of TX x TY x TZ output voxels.  Its image under the affine
// map is a parallelepiped whose coordinate extrema sit at the box's corners,
// so the floors at the 8 corners bound every trilinear tap (floor(s) and
// floor(s) + 1) and every nearest label (floor(s + 1/2)) of the tile: the
// brick [lo, hi] per axis, with lo the smallest corner floor and hi the
// largest plus 1.  Shared index of input element (x, y, z):
//   ((z - lo_z) BY + y - lo_y) P + x - lo_x + sh,
// with the row pitch P = nx (mod 4), P >= bx + 3, the slab pitch BY P = nx ny
// (mod 4) and the shift sh = (element address of the origin) mod 4, so every
// element's shared index is congruent to its global element address modulo
// 4: a 16-byte chunk of the input is 16-byte aligned in the brick too.
#pragma once

#include "kernels.h"
#include "sample.cuh"

namespace augk {

enum { BRICK_STAGED = 0, BRICK_EXTERIOR = 1, BRICK_DIRECT = 2 };

// Geometry of one tile's brick, computed by warp 0 and read by all threads.
struct BrickGeom {
  int lo[3];     // brick origin (input voxel indices, may lie outside the input)
  int bx, by, bz;
  int P, BY, PBY;  // row pitch, rows per slab and slab pitch of the shared bricks
  int shi, shl;  // shared index of the origin in the image / label brick
  int spr, lgs;  // chunks per row, log2 lanes per row
  int inner;     // the brick lies inside the input with an x margin of 3 elements
  int mode;
};

__device__ __forceinline__ unsigned smem_addr(const void* p) {
  return (unsigned)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ void cp_async16(void* s, const void* g) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(smem_addr(s)), "l"(g)
               : "memory");
}
__device__ __forceinline__ void cp_async4(void* s, const void* g) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(smem_addr(s)), "l"(g)
               : "memory");
}
__device__ __forceinline__ void cp_async_wait_all() {
  asm volatile("cp.async.wait_all;" ::: "memory");
}

// floor(a / b) for 0 <= a < 2^21 and 1 <= b < 2^24 (brick row indices), from the hardware
// reciprocal (relative error below 2^-23; b is never subnormal): the quotient
// (a + 1/2) / b lies at least 1/(2b) from an integer, and the reciprocal and
// the product move it by less than (a + 1/2) 1.5 2^-23 / b < 1/(2b).
__device__ __forceinline__ int small_div(int a, int b) {
  float r;
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"((float)b));
  return (int)(((float)a + 0.5f) * r);
}

// Box tile t -> (tx, ty, tz), x fastest (exact integer division: tile indices
// can exceed the range of small_div on large volumes).
template <int TX, int TY>
__device__ __forceinline__ void box_tile_index(int t, int onx, int ony, int& tx, int& ty,
                                               int& tz) {
  const int ntx = (onx + TX - 1) / TX, nty = (ony + TY - 1) / TY;
  const int q = t / ntx;
  tx = t - q * ntx;
  tz = q / nty;
  ty = q - tz * nty;
}

// Thread coordinates of box tile t: TXW lanes along x, 32 / TXW rows of the
// warp along y, warps stacked along y; each thread walks TZ = 4 * QZ z values
// (box_tile_coord).
template <int TXW, int NW, int QZ>
__device__ __forceinline__ TileCoord tile_coord_box(int t, int onx, int ony, int onz) {
  return box_tile_coord<TXW, NW, QZ>(t, onx, ony, onz);
}

// Brick of tile t (warp 0; lanes 8 r + c compute axis r at corner c).  CAP:
// capacity of the shared bricks in elements.
template <int TX, int TY, int TZ, int CAP>
__device__ __forceinline__ void brick_geometry(const VolConst& vc, int t, BrickGeom& bg) {
  if (threadIdx.x >= 32) return;
  const int lane = threadIdx.x;
  int tx, ty, tz;
  box_tile_index<TX, TY>(t, vc.onx, vc.ony, tx, ty, tz);
  // Lane 8 r + c (r < 3, c < 8): floor of axis r at corner c; min and max over
  // each group of 8 lanes.
  const int r = min(lane >> 3, 2), c = lane & 7;
  const int ci = (c & 1) ? min(tx * TX + TX - 1, vc.onx - 1) : tx * TX;
  const int cj = (c & 2) ? min(ty * TY + TY - 1, vc.ony - 1) : ty * TY;
  const int ck = (c & 4) ? min(tz * TZ + TZ - 1, vc.onz - 1) : tz * TZ;
  int mn = q40_floor(coord_q40(vc.tq[r], ci, cj, ck)), mx = mn;
#pragma unroll
  for (int o = 4; o > 0; o >>= 1) {
    mn = min(mn, __shfl_xor_sync(FULL_MASK, mn, o));
    mx = max(mx, __shfl_xor_sync(FULL_MASK, mx, o));
  }
  const int lo0 = __shfl_sync(FULL_MASK, mn, 0), lo1 = __shfl_sync(FULL_MASK, mn, 8),
            lo2 = __shfl_sync(FULL_MASK, mn, 16);
  const int hi0 = __shfl_sync(FULL_MASK, mx, 0) + 1, hi1 = __shfl_sync(FULL_MASK, mx, 8) + 1,
            hi2 = __shfl_sync(FULL_MASK, mx, 16) + 1;
  if (lane != 0) return;
  const int nx = vc.nx, ny = vc.ny, nz = vc.nz;
  bg.lo[0] = lo0;
  bg.lo[1] = lo1;
  bg.lo[2] = lo2;
  const bool exterior =
      hi0 < 0 || lo0 > nx - 1 || hi1 < 0 || lo1 > ny - 1 || hi2 < 0 || lo2 > nz - 1;
  if (exterior) {
    bg.mode = BRICK_EXTERIOR;
    return;
  }
  // Extents in 64 bits: a steep affine can span the whole input per axis.
  const long long bx = (long long)hi0 - lo0 + 1, by = (long long)hi1 - lo1 + 1,
                  bz = (long long)hi2 - lo2 + 1;
  const bool f32 = vc.dtype == AUG_F32;
  if (!f32 || bx > 120 || by > CAP || bz > CAP) {
    bg.mode = BRICK_DIRECT;
    return;
  }
  // P >= bx + 3 (room for a chunk's spill on either side of a row), P = nx mod 4;
  // BY >= by with BY * P = nx * ny mod 4.
  int P = (int)bx + 3;
  P += (nx - P) & 3;
  int BY = (int)by;
  while ((((long long)BY * P - (long long)nx * ny) & 3) != 0) ++BY;
  const long long size = (long long)P * BY * bz + 8;
  if (size > CAP) {
    bg.mode = BRICK_DIRECT;
    return;
  }
  bg.bx = (int)bx;
  bg.by = (int)by;
  bg.bz = (int)bz;
  bg.P = P;
  bg.BY = BY;
  bg.PBY = P * BY;
  // Shared index of element (x, y, z) = ((z - lo2) BY + y - lo1) P + x - lo0 + sh, with
  // sh = (global element address of the origin) mod 4.
  const long long flat_lo = ((long long)lo2 * ny + lo1) * nx + lo0;
  bg.shi = (int)(((long long)((uintptr_t)vc.image >> 2) + flat_lo) & 3);
  bg.shl = (int)(((long long)(uintptr_t)vc.label + flat_lo) & 3);
  const int spr = ((int)bx + 6) >> 2;
  bg.spr = spr;
  bg.lgs = spr <= 1 ? 0 : 32 - __clz(spr - 1);
  bg.inner = lo0 >= 3 && hi0 + 3 <= nx - 1 && lo1 >= 0 && hi1 <= ny - 1 && lo2 >= 0 &&
             hi2 <= nz - 1;
  bg.mode = BRICK_STAGED;
}

// ---- image brick staged by bulk row copies -------------------------------------------
// Every row (y, z) of the brick is one contiguous run of input elements
// [max(lx, 0), min(hx, nx - 1)] when (y, z) lies inside the input.  Its
// 16-byte-aligned part is one cp.async.bulk (the tensor-memory-access unit
// writes shared memory, no thread registers involved), widened to whole
// 16-byte chunks where those stay inside the row; the at most 3 + 3 elements
// at unaligned row ends are copied by the thread, and taps outside the input
// are written as fill.  One thread per row; completion on an mbarrier.
__device__ __forceinline__ void mbar_init_cta(uint32_t bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_arrive_tx(uint32_t bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes)
               : "memory");
}
// Bounded wait for the phase of the given parity: about a second at most.
__device__ __forceinline__ bool mbar_wait_bounded(uint32_t bar, uint32_t parity) {
  for (uint32_t it = 0; it < (1u << 24); ++it) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.test_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(bar), "r"(parity)
        : "memory");
    if (ok) return true;
    if (it >= 8) __nanosleep(32);
  }
  return false;
}
__device__ __forceinline__ void bulk_copy_g2s(uint32_t dst, const void* src, uint32_t bytes,
                                              uint32_t bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];"
      ::"r"(dst), "l"(src), "r"(bytes), "r"(bar)
      : "memory");
}

// Issues the copies of the image brick; returns the bytes the bulk copies
// will deliver.  rows r = threadIdx.x, threadIdx.x + NTHR, ...
template <int NTHR>
__device__ __forceinline__ uint32_t stage_rows_bulk(const VolConst& vc, const BrickGeom& g,
                                                    float* simg, uint32_t bar) {
  const int nx = vc.nx, ny = vc.ny, nz = vc.nz;
  const int lx = g.lo[0], ly = g.lo[1], lz = g.lo[2];
  const int hx = lx + g.bx - 1;
  const int xs = max(lx, 0), xe = min(hx, nx - 1);
  const float* __restrict__ img = (const float*)vc.image;
  // element address (address / 4) of the image's first element, mod 4 is all
  // that matters for chunk alignment
  const unsigned abase = (unsigned)((uintptr_t)img >> 2);
  const float fill = vc.fill;
  const int rows = g.by * g.bz;
  uint32_t bytes = 0;
  for (int r = threadIdx.x; r < rows; r += NTHR) {
    const int ez = small_div(r, g.by), ey = r - ez * g.by;
    const int y = ly + ey, z = lz + ez;
    float* row = simg + ((ez * g.BY + ey) * g.P + g.shi - lx);  // row[x] = element x
    const bool rin = (unsigned)y < (unsigned)ny && (unsigned)z < (unsigned)nz && xs <= xe;
    if (!rin) {
      for (int x = lx; x <= hx; ++x) row[x] = fill;
      continue;
    }
    for (int x = lx; x < xs; ++x) row[x] = fill;
    for (int x = xe + 1; x <= hx; ++x) row[x] = fill;
    const int grow = (z * ny + y) * nx;
    const float* src = img + grow;  // src[x] = element x of this row
    // whole chunks: widen [xs, xe] to 4-element boundaries of the element
    // address where the widened elements stay in [0, nx), else shrink
    const unsigned ms = (abase + (unsigned)(grow + xs)) & 3u;
    int xa = xs - (int)ms;
    if (xa < 0) xa += 4;
    const unsigned me = (abase + (unsigned)(grow + xe + 1)) & 3u;
    int xb = xe + 1 + (int)((4u - me) & 3u);
    if (xb > nx) xb -= 4;
    if (xb > xa) {
      bulk_copy_g2s(smem_addr(row + xa), src + xa, (uint32_t)(xb - xa) * 4u, bar);
      bytes += (uint32_t)(xb - xa) * 4u;
      for (int x = xs; x < xa; ++x) row[x] = __ldg(src + x);
      for (int x = xb; x <= xe; ++x) row[x] = __ldg(src + x);
    } else {
      for (int x = xs; x <= xe; ++x) row[x] = __ldg(src + x);
    }
  }
  return bytes;
}

}  // namespace augk
