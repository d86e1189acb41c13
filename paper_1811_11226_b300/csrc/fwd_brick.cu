// Forward augmentation (Sec. 4) with each tile's input footprint staged in a
// shared-memory brick (brick.cuh).  The CTA copies the brick of the image and
// of the labels into shared memory -- taps outside the input get the fill
// values there -- and then samples every voxel from shared memory with no
// bounds checks.
// The per-voxel arithmetic (exact Q.40 coordinates, weights, lerps, noise)
// is that of the direct kernels in fwd.cuh, so both give bitwise-equal
// outputs.
//
// Copies are cp.async (no register staging) of 4-element chunks: 16 bytes of
// float32 image, 4 bytes of labels.  A chunk must be aligned in global and in
// shared memory alike, so the brick's row pitch P and slab pitch BY * P are
// chosen congruent to the input's nx and nx * ny modulo 4, and the brick is
// shifted by the (address / element size) mod 4 of its origin: every element's
// shared index is then congruent to its global element address modulo 4, for
// any row length and any base alignment.  Chunks that straddle the input's x
// boundary are copied element by element, and taps outside the input are
// written as fill.
//
// Tiles with no tap inside the input take the fill-only path (no copies);
// tiles whose brick exceeds the shared-memory capacity (strong minification)
// and int16 inputs take the direct-gather path of fwd.cuh.
#include "brick.cuh"
#include "fwd.cuh"

namespace augk {

// One row of the bricks: the chunks of row (y, z) whose first element x0 is
// at most hx, with per-element checks (GENERAL) or without (a row inside the
// input with a margin of 3 elements on both sides in x: every chunk is a
// 4-element run of input elements).
template <bool IMG, bool LAB, bool GENERAL>
__device__ __forceinline__ void stage_row(const float* __restrict__ img,
                                          const uint8_t* __restrict__ lab, float* simg,
                                          uint8_t* slab, int rowbase, int shi, int shl, int slot,
                                          int lx, int hx, int nx, bool rin, int grow, float fill,
                                          uint8_t fill_label) {
  if (IMG) {
    const int d0 = rowbase + shi;  // shared index of x = lx
    const int si = (d0 & ~3) + 4 * slot;
    const int x0 = lx + (si - d0);
    if (x0 <= hx) {
      if (!GENERAL || (rin && x0 >= 0 && x0 + 3 < nx)) {
        cp_async16(simg + si, img + (grow + x0));
      } else {
#pragma unroll
        for (int m = 0; m < 4; ++m) {
          const int x = x0 + m;
          if (x < lx || x > hx) continue;
          if (rin && (unsigned)x < (unsigned)nx)
            cp_async4(simg + si + m, img + (grow + x));
          else
            simg[si + m] = fill;
        }
      }
    }
  }
  if (LAB) {
    const int d0 = rowbase + shl;
    const int si = (d0 & ~3) + 4 * slot;
    const int x0 = lx + (si - d0);
    if (x0 <= hx) {
      if (!GENERAL || (rin && x0 >= 0 && x0 + 3 < nx)) {
        cp_async4(slab + si, lab + (grow + x0));
      } else {
#pragma unroll
        for (int m = 0; m < 4; ++m) {
          const int x = x0 + m;
          if (x < lx || x > hx) continue;
          slab[si + m] =
              (rin && (unsigned)x < (unsigned)nx) ? __ldg(lab + (grow + x)) : fill_label;
        }
      }
    }
  }
}


// Copies the image (IMG) and label (LAB) bricks into shared memory, fill
// outside the input; all threads, then every copy is complete and visible.
// Warps take whole z-slabs of the brick; within a slab a warp covers
// 32 >> lgs rows at a time, 1 << lgs lanes per row (one 4-element chunk each).
template <int NW, bool IMG, bool LAB, bool GENERAL>
__device__ __forceinline__ void stage_brick_t(const VolConst& vc, const BrickGeom& g,
                                              float* simg, uint8_t* slab) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int nx = vc.nx, ny = vc.ny, nz = vc.nz;
  const int lx = g.lo[0], ly = g.lo[1], lz = g.lo[2];
  const int hx = lx + g.bx - 1;
  const int by = g.by, bz = g.bz, BY = g.BY, P = g.P, shi = g.shi, shl = g.shl;
  const int lgs = g.lgs, rpw = 32 >> lgs;
  const int sub = lane >> lgs, slot = lane & ((1 << lgs) - 1);
  const bool act = slot < g.spr;
  const float* __restrict__ img = (const float*)vc.image;
  const uint8_t* __restrict__ lab = vc.label;
  const float fill = vc.fill;
  const uint8_t fill_label = (uint8_t)vc.fill_label;
  for (int ez = warp; ez < bz; ez += NW) {
    const int z = lz + ez;
    for (int ey = sub; ey < by; ey += rpw) {
      if (!act) continue;
      const int y = ly + ey;
      const bool rin = !GENERAL || ((unsigned)y < (unsigned)ny && (unsigned)z < (unsigned)nz);
      // Global element index of (x = 0, y, z); used only when the row is inside.
      const int grow = rin ? (z * ny + y) * nx : 0;
      stage_row<IMG, LAB, GENERAL>(img, lab, simg, slab, (ez * BY + ey) * P, shi, shl, slot, lx,
                                   hx, nx, rin, grow, fill, fill_label);
    }
  }
  cp_async_wait_all();
  __syncthreads();
}

template <int NW, bool IMG, bool LAB>
__device__ __forceinline__ void stage_brick(const VolConst& vc, const BrickGeom& bg,
                                            float* simg, uint8_t* slab) {
  const BrickGeom g = bg;  // in registers: the copies' memory clobbers do not reload it
  if (g.inner)
    stage_brick_t<NW, IMG, LAB, false>(vc, g, simg, slab);
  else
    stage_brick_t<NW, IMG, LAB, true>(vc, g, simg, slab);
}

// One quad (n = 1..4 z-consecutive voxels) sampled from the shared bricks.
// The coordinates s are relative to the brick origin (Q.40); PD voxels'
// loads are issued before their samples are interpolated.
// Direct label gathers (labels not staged): the brick origin and whether its
// labels need bounds checks.
struct LabDirect {
  int lx, ly, lz;
  bool check;
};

template <bool POST, bool IMG, bool LAB, bool LST, bool FULL, int PD>
__device__ __forceinline__ void brick_quad(const FwdP<float>& P, const float* __restrict__ simg,
                                           const uint8_t* __restrict__ slab, int bP, int bPBY,
                                           int shi, int dsl, const LabDirect& ld, long long& sx,
                                           long long& sy, long long& sz, int& o, int n,
                                           bool valid, bool noisy, unsigned long long quad,
                                           unsigned noise_id, const PhiloxKey& key, int kq) {
  float z[4] = {0.0f, 0.0f, 0.0f, 0.0f};
#pragma unroll
  for (int g0 = 0; g0 < 4; g0 += PD) {
    float tap[PD][8];
    float w[PD][3];
    int lab[PD];
#pragma unroll
    for (int i = 0; i < PD; ++i) {
      const int m = g0 + i;
      lab[i] = 0;
#pragma unroll
      for (int d = 0; d < 8; ++d) tap[i][d] = 0.0f;
      w[i][0] = w[i][1] = w[i][2] = 0.0f;
      if (FULL || m < n) {
        const int fx = q40_floor(sx), fy = q40_floor(sy), fz = q40_floor(sz);
        const int b = fz * bPBY + fy * bP + fx;
        if (IMG) {
          w[i][0] = q40_frac(sx);
          w[i][1] = q40_frac(sy);
          w[i][2] = q40_frac(sz);
          const float* p = simg + (b + shi);
          tap[i][0] = p[0];
          tap[i][1] = p[1];
          tap[i][2] = p[bP];
          tap[i][3] = p[bP + 1];
          tap[i][4] = p[bPBY];
          tap[i][5] = p[bPBY + 1];
          tap[i][6] = p[bPBY + bP];
          tap[i][7] = p[bPBY + bP + 1];
        }
        if (LAB && LST) {
          const int off = q40_halfbit(sx) + (q40_halfbit(sy) ? bP : 0) +
                          (q40_halfbit(sz) ? bPBY : 0);
          lab[i] = slab[b + dsl + off];
        } else if (LAB) {
          const int rx = ld.lx + fx + q40_halfbit(sx), ry = ld.ly + fy + q40_halfbit(sy),
                    rz = ld.lz + fz + q40_halfbit(sz);
          lab[i] = P.fill_label;
          if (!ld.check || ((unsigned)rx < (unsigned)P.nx && (unsigned)ry < (unsigned)P.ny &&
                            (unsigned)rz < (unsigned)P.nz))
            lab[i] = __ldg(P.lab + ((rz * P.ny + ry) * P.nx + rx));
        }
        sx += P.dx;
        sy += P.dy;
        sz += P.dz;
      }
    }
    if (g0 == 0 && noisy) quad_normals(quad, noise_id, key, z);
    if (FULL && IMG && PD >= 2) {
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

template <bool IMG, bool LAB>
__device__ __forceinline__ FwdP<float> brick_params(const VolConst& vc) {
  FwdP<float> P;
  P.img = (const float*)vc.image;
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
  return P;
}

// Samples the whole z-run of this thread from the staged bricks (POST: the
// occlusion slab or the window clamp meets the run).
template <bool POST, bool IMG, bool LAB, bool LST, int PD>
__device__ __forceinline__ void brick_tile_run(const VolConst& vc, const BrickGeom& bg,
                                               const TileCoord& tc,
                                               const float* __restrict__ simg,
                                               const uint8_t* __restrict__ slab,
                                               const PhiloxKey& key) {
  const FwdP<float> P = brick_params<IMG, LAB>(vc);
  const unsigned onx = (unsigned)vc.onx, ony = (unsigned)vc.ony;
  const bool noisy = IMG && vc.sigma > 0.0f;
  long long sx = coord_q40(vc.tq[0], tc.ic, tc.jc, tc.k0) - ((long long)bg.lo[0] << 40);
  long long sy = coord_q40(vc.tq[1], tc.ic, tc.jc, tc.k0) - ((long long)bg.lo[1] << 40);
  long long sz = coord_q40(vc.tq[2], tc.ic, tc.jc, tc.k0) - ((long long)bg.lo[2] << 40);
  int o = (tc.k0 * vc.ony + tc.jc) * vc.onx + tc.ic;
  const int bP = bg.P, bPBY = bg.PBY, shi = bg.shi, dsl = bg.shl;
  const LabDirect ld{bg.lo[0], bg.lo[1], bg.lo[2], !bg.inner};
#pragma unroll 1
  for (int kq = tc.k0; kq < tc.k1; kq += 4) {
    const int n = min(4, tc.k1 - kq);
    const unsigned long long quad =
        ((unsigned long long)(kq >> 2) * ony + (unsigned)tc.jc) * onx + (unsigned)tc.ic;
    if (n == 4)
      brick_quad<POST, IMG, LAB, LST, true, PD>(P, simg, slab, bP, bPBY, shi, dsl, ld, sx, sy,
                                                sz, o, 4, tc.valid, noisy, quad, vc.noise_id,
                                                key, kq);
    else
      brick_quad<POST, IMG, LAB, LST, false, PD>(P, simg, slab, bP, bPBY, shi, dsl, ld, sx, sy,
                                                 sz, o, n, tc.valid, noisy, quad, vc.noise_id,
                                                 key, kq);
  }
}

// Tile with no tap inside the input: the fill value, the intensity affine and
// the noise (no loads).
template <bool POST, bool IMG, bool LAB>
__device__ __forceinline__ void brick_tile_exterior(const VolConst& vc, const TileCoord& tc,
                                                    const PhiloxKey& key) {
  const FwdP<float> P = brick_params<IMG, LAB>(vc);
  const unsigned onx = (unsigned)vc.onx, ony = (unsigned)vc.ony;
  const bool noisy = IMG && vc.sigma > 0.0f;
  int o = (tc.k0 * vc.ony + tc.jc) * vc.onx + tc.ic;
#pragma unroll 1
  for (int kq = tc.k0; kq < tc.k1; kq += 4) {
    const int n = min(4, tc.k1 - kq);
    float z[4] = {0.0f, 0.0f, 0.0f, 0.0f};
    if (noisy)
      quad_normals(((unsigned long long)(kq >> 2) * ony + (unsigned)tc.jc) * onx +
                       (unsigned)tc.ic,
                   vc.noise_id, key, z);
    fwd_quad_exterior<POST, float, IMG, LAB>(P, o, n, tc.valid, z, kq);
  }
}

template <int NW, int PD, bool IMG, bool LAB, bool LST>
__device__ __forceinline__ void brick_tile(const VolConst& vc, const BrickGeom& bg,
                                           const TileCoord& tc, float* simg, uint8_t* slab,
                                           const PhiloxKey& key) {
  const bool post = (vc.flags & AUG_FLAG_WINDOW) ||
                    (vc.occ_klo <= vc.occ_khi && vc.occ_klo < tc.k1 && vc.occ_khi >= tc.k0);
  if (bg.mode == BRICK_EXTERIOR) {
    if (post)
      brick_tile_exterior<true, IMG, LAB>(vc, tc, key);
    else
      brick_tile_exterior<false, IMG, LAB>(vc, tc, key);
    return;
  }
  stage_brick<NW, IMG, LAB && LST>(vc, bg, simg, slab);
  if (post)
    brick_tile_run<true, IMG, LAB, LST, PD>(vc, bg, tc, simg, slab, key);
  else
    brick_tile_run<false, IMG, LAB, LST, PD>(vc, bg, tc, simg, slab, key);
}

// TXW: lanes along x; NW: warps per CTA; QZ: quads per thread; PD: voxels whose
// loads are issued together; CAP: shared brick capacity (elements); MB: min
// CTAs per SM for the register allocator; LST: labels staged in a brick too
// (else gathered from global memory).  Dynamic shared memory: CAP floats
// (image) + CAP bytes (labels, LST only).
template <int TXW, int NW, int QZ, int PD, int CAP, int MB, bool LST>
__global__ void __launch_bounds__(NW * 32, MB)
    k_fwd_brick(const aug_volume_desc* __restrict__ descs, int n_vols,
                const VolConst* __restrict__ tab, const PhiloxKey key,
                unsigned long long* counter) {
  constexpr int TX = TXW, TY = (32 / TXW) * NW, TZ = 4 * QZ;
  extern __shared__ __align__(16) unsigned char brick_smem[];
  float* simg = (float*)brick_smem;
  uint8_t* slab = LST ? brick_smem + (size_t)CAP * sizeof(float) : nullptr;
  __shared__ SchedSmem<NW * 32> sm;
  __shared__ BrickGeom bg;
  for_each_tile_dynamic_t<NW, BoxTiles<TX, TY, TZ>>(
      descs, n_vols, sm, counter, [&](int v, int t, long long) {
        const VolConst& vc = tab[v];
        const bool img = vc.out_image != nullptr, lab = vc.out_label != nullptr;
        if (!vc.ok || (!img && !lab)) return;
        const TileCoord tc = tile_coord_box<TXW, NW, QZ>(t, vc.onx, vc.ony, vc.onz);
        brick_geometry<TX, TY, TZ, CAP>(vc, t, bg);
        __syncthreads();
        if (bg.mode == BRICK_DIRECT) {
          fwd_tile_direct<QZ, 1>(vc, tc, key);
        } else if (img && lab) {
          brick_tile<NW, PD, true, true, LST>(vc, bg, tc, simg, slab, key);
        } else if (img) {
          brick_tile<NW, PD, true, false, LST>(vc, bg, tc, simg, slab, key);
        } else {
          brick_tile<NW, PD, false, true, LST>(vc, bg, tc, simg, slab, key);
        }
      });
}

// The brick forward with the image brick staged by bulk row copies and the
// labels gathered from global memory (see stage_rows_bulk).  Same parameters
// as k_fwd_brick; dynamic shared memory: CAP floats.
template <int TXW, int NW, int QZ, int PD, int CAP, int MB>
__global__ void __launch_bounds__(NW * 32, MB)
    k_fwd_brick_bulk(const aug_volume_desc* __restrict__ descs, int n_vols,
                     const VolConst* __restrict__ tab, const PhiloxKey key,
                     unsigned long long* counter, WsHeader* ws) {
  constexpr int TX = TXW, TY = (32 / TXW) * NW, TZ = 4 * QZ;
  extern __shared__ __align__(16) unsigned char brick_smem[];
  float* simg = (float*)brick_smem;
  __shared__ SchedSmem<NW * 32> sm;
  __shared__ BrickGeom bg;
  __shared__ __align__(8) unsigned long long bar_word;
  const uint32_t bar = smem_addr(&bar_word);
  if (threadIdx.x == 0) {
    mbar_init_cta(bar, NW * 32);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();
  uint32_t parity = 0;
  bool failed = false;
  for_each_tile_dynamic_t<NW, BoxTiles<TX, TY, TZ>>(
      descs, n_vols, sm, counter, [&](int v, int t, long long) {
        if (failed) return;
        const VolConst& vc = tab[v];
        const bool img = vc.out_image != nullptr, lab = vc.out_label != nullptr;
        if (!vc.ok || (!img && !lab)) return;
        const TileCoord tc = tile_coord_box<TXW, NW, QZ>(t, vc.onx, vc.ony, vc.onz);
        brick_geometry<TX, TY, TZ, CAP>(vc, t, bg);
        __syncthreads();
        const BrickGeom g = bg;
        if (g.mode == BRICK_DIRECT || (g.mode == BRICK_STAGED && !img)) {
          fwd_tile_direct<QZ, 1>(vc, tc, key);
          return;
        }
        const bool post = (vc.flags & AUG_FLAG_WINDOW) ||
                          (vc.occ_klo <= vc.occ_khi && vc.occ_klo < tc.k1 && vc.occ_khi >= tc.k0);
        if (g.mode == BRICK_EXTERIOR) {
          if (img && lab) {
            if (post) brick_tile_exterior<true, true, true>(vc, tc, key);
            else brick_tile_exterior<false, true, true>(vc, tc, key);
          } else if (img) {
            if (post) brick_tile_exterior<true, true, false>(vc, tc, key);
            else brick_tile_exterior<false, true, false>(vc, tc, key);
          } else {
            if (post) brick_tile_exterior<true, false, true>(vc, tc, key);
            else brick_tile_exterior<false, false, true>(vc, tc, key);
          }
          return;
        }
        // The previous tile's reads of the brick (generic proxy) come before
        // this tile's bulk writes (async proxy).
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        const uint32_t bytes = stage_rows_bulk<NW * 32>(vc, g, simg, bar);
        mbar_arrive_tx(bar, bytes);
        const bool ok = mbar_wait_bounded(bar, parity);
        parity ^= 1u;
        if (__syncthreads_or(!ok)) {
          // A copy did not land in about a second: record it, let the copies
          // in flight finish (bounded again) and leave.
          if (threadIdx.x == 0) record_error(ws, AUG_ERR_TIMEOUT, v);
          mbar_wait_bounded(bar, parity ^ 1u);
          failed = true;
          return;
        }
        if (lab) {
          if (post) brick_tile_run<true, true, true, false, PD>(vc, g, tc, simg, nullptr, key);
          else brick_tile_run<false, true, true, false, PD>(vc, g, tc, simg, nullptr, key);
        } else {
          if (post) brick_tile_run<true, true, false, false, PD>(vc, g, tc, simg, nullptr, key);
          else brick_tile_run<false, true, false, false, PD>(vc, g, tc, simg, nullptr, key);
        }
      });
}

// ---- host side --------------------------------------------------------------------
namespace {
using BrickK = void (*)(const aug_volume_desc*, int, const VolConst*, const PhiloxKey,
                        unsigned long long*);
using BulkK = void (*)(const aug_volume_desc*, int, const VolConst*, const PhiloxKey,
                       unsigned long long*, WsHeader*);
struct BrickVariant {
  int threads, cap;
  bool lst;     // labels staged (chunk kernel only)
  BrickK k;     // chunk-copy kernel, or
  BulkK kb;     // bulk-row-copy kernel
  const char* name;
};
#define BRICK_V(TXW, NW, QZ, PD, CAP, MB, LST, NAME) \
  { NW * 32, CAP, LST, k_fwd_brick<TXW, NW, QZ, PD, CAP, MB, LST>, nullptr, NAME }
#define BULK_V(TXW, NW, QZ, PD, CAP, MB, NAME) \
  { NW * 32, CAP, false, nullptr, k_fwd_brick_bulk<TXW, NW, QZ, PD, CAP, MB>, NAME }
// (lanes along x, warps, quads per thread, pipeline depth, capacity, min CTAs/SM,
// labels staged)
const BrickVariant kBrick[] = {
    BRICK_V(16, 4, 4, 2, 9728, 4, true, "brick16x8x16_pd2_c9728"),
    BRICK_V(16, 8, 4, 2, 16384, 2, true, "brick16x16x16_pd2_c16384"),
    BRICK_V(16, 4, 4, 2, 9728, 4, false, "brick16x8x16_pd2_c9728_lg"),
    BRICK_V(16, 8, 2, 2, 9728, 4, false, "brick16x16x8_pd2_c9728_lg"),
    BULK_V(16, 4, 4, 2, 9728, 5, "bulk16x8x16_pd2_c9728"),
    BULK_V(16, 8, 2, 2, 9728, 4, "bulk16x16x8_pd2_c9728"),
    BULK_V(16, 8, 4, 2, 16384, 3, "bulk16x16x16_pd2_c16384"),
    BULK_V(16, 4, 4, 1, 9728, 5, "bulk16x8x16_pd1_c9728"),
};
#undef BRICK_V
#undef BULK_V
}  // namespace

int fwd_brick_num_variants() { return (int)(sizeof(kBrick) / sizeof(kBrick[0])); }
const char* fwd_brick_variant_name(int v) { return kBrick[v].name; }

cudaError_t launch_fwd_brick(int variant, const aug_volume_desc* d, int n, unsigned k0,
                             unsigned k1, VolConst* tab, WsHeader* ws, cudaStream_t st) {
  const BrickVariant& bv = kBrick[variant];
  if (ws == nullptr) return cudaErrorInvalidValue;
  const void* fn = bv.k ? (const void*)bv.k : (const void*)bv.kb;
  const size_t smem = (size_t)bv.cap * (sizeof(float) + (bv.lst ? 1 : 0));
  // Dynamic plus static shared memory may exceed the 48 KB a launch gets
  // without opting in.
  cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)smem);
  if (e != cudaSuccess) return e;
  const int grid = persistent_grid(fn, bv.threads, smem);
  if (grid <= 0) return cudaErrorInvalidConfiguration;
  e = launch_prepare(d, n, NEED_IMAGE_IF_OUT, false, nullptr, nullptr, false, tab, ws, st,
                     (unsigned long long)grid);
  if (e != cudaSuccess) return e;
  if (bv.k)
    bv.k<<<grid, bv.threads, smem, st>>>(d, n, tab, philox_schedule(k0, k1), &ws->tile_next);
  else
    bv.kb<<<grid, bv.threads, smem, st>>>(d, n, tab, philox_schedule(k0, k1), &ws->tile_next,
                                          ws);
  return cudaGetLastError();
}

}  // namespace augk
