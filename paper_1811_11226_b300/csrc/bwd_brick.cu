// Adjoint of the image warp with each tile's input footprint in shared memory
// (brick.cuh): the brick of the image (only when the affine gradient is
// wanted: dv/ds needs the taps) is staged by bulk row copies with the fill
// value outside the input, and the input gradient of the tile is accumulated
// in a second brick with shared-memory reductions.  Taps outside the input
// then need no check at all: they read the staged fill, and their gradient
// lands in brick positions that are never written back.  After the tile, the
// brick positions inside the input are added to grad_in with global
// reductions, a warp per brick row (consecutive addresses), zeros skipped.
//
// The per-voxel arithmetic is that of bwd.cuh: weights, the z-merge of the
// z+1 contributions into the next voxel's z taps, dv/ds from the cell's
// taps, and the 12 affine sums reduced per tile in a fixed order.  The static
// tile schedule keeps the affine gradient bitwise reproducible.  Tiles with no
// tap inside the input contribute nothing; tiles whose brick exceeds the
// capacity and int16 inputs take the direct path of bwd.cuh.
#include "brick.cuh"
#include "bwd.cuh"

namespace augk {

// The z-run of this thread, sampled from / scattered into the bricks.
template <bool GIN, bool GT>
__device__ __forceinline__ void bwd_brick_run(const VolConst& vc, const BrickGeom& bg,
                                              const TileCoord& tc,
                                              const float* __restrict__ simg, float* sgrad,
                                              const float* __restrict__ g, float acc[6]) {
  const long long dx = vc.tq[0][2], dy = vc.tq[1][2], dz = vc.tq[2][2];
  long long sx = coord_q40(vc.tq[0], tc.ic, tc.jc, tc.k0) - ((long long)bg.lo[0] << 40);
  long long sy = coord_q40(vc.tq[1], tc.ic, tc.jc, tc.k0) - ((long long)bg.lo[1] << 40);
  long long sz = coord_q40(vc.tq[2], tc.ic, tc.jc, tc.k0) - ((long long)bg.lo[2] << 40);
  const int plane = vc.onx * vc.ony;
  const float a = vc.a;
  const int klo = vc.occ_klo, khi = vc.occ_khi;
  const int P = bg.P, PBY = bg.PBY, sh = bg.shi;
  int o = (tc.k0 * vc.ony + tc.jc) * vc.onx + tc.ic;
  float pend[4] = {0.f, 0.f, 0.f, 0.f};
  int pend_base = -1;
#pragma unroll 2
  for (int k = tc.k0; k < tc.k1; ++k) {
    // An occluded output voxel is the constant 0: no gradient flows through it.
    const bool occ = k >= klo && k <= khi;
    const float ga = (tc.valid && !occ) ? a * __ldcs(g + o) : 0.0f;
    const int fx = q40_floor(sx), fy = q40_floor(sy), fz = q40_floor(sz);
    const float tx = q40_frac(sx), ty = q40_frac(sy), tz = q40_frac(sz);
    const int b = fz * PBY + fy * P + fx + sh;
    if (GIN) {
      const float wx1 = tx, wx0 = 1.0f - tx, wy1 = ty, wy0 = 1.0f - ty;
      const float wz1 = tz, wz0 = 1.0f - tz;
      const float g00 = ga * wy0 * wz0, g10 = ga * wy1 * wz0;
      const float g01 = ga * wy0 * wz1, g11 = ga * wy1 * wz1;
      float c0 = g00 * wx0, c1 = g00 * wx1, c2 = g10 * wx0, c3 = g10 * wx1;
      if (b == pend_base) {
        c0 += pend[0];
        c1 += pend[1];
        c2 += pend[2];
        c3 += pend[3];
      } else if (pend_base >= 0) {
        float* q = sgrad + pend_base;
        red_add_shared(q, pend[0]);
        red_add_shared(q + 1, pend[1]);
        red_add_shared(q + P, pend[2]);
        red_add_shared(q + P + 1, pend[3]);
      }
      float* p = sgrad + b;
      red_add_shared(p, c0);
      red_add_shared(p + 1, c1);
      red_add_shared(p + P, c2);
      red_add_shared(p + P + 1, c3);
      pend[0] = g01 * wx0;
      pend[1] = g01 * wx1;
      pend[2] = g11 * wx0;
      pend[3] = g11 * wx1;
      pend_base = b + PBY;
    }
    if (GT) {
      const float* t = simg + b;
      const float v000 = t[0], v100 = t[1], v010 = t[P], v110 = t[P + 1];
      const float v001 = t[PBY], v101 = t[PBY + 1], v011 = t[PBY + P], v111 = t[PBY + P + 1];
      const float c00 = fmaf(tx, v100 - v000, v000);
      const float c10 = fmaf(tx, v110 - v010, v010);
      const float c01 = fmaf(tx, v101 - v001, v001);
      const float c11 = fmaf(tx, v111 - v011, v011);
      const float c0 = fmaf(ty, c10 - c00, c00);
      const float c1 = fmaf(ty, c11 - c01, c01);
      const float e0 = fmaf(ty, (v110 - v010) - (v100 - v000), v100 - v000);
      const float e1 = fmaf(ty, (v111 - v011) - (v101 - v001), v101 - v001);
      const float dvx = fmaf(tz, e1 - e0, e0);
      const float dvy = fmaf(tz, (c11 - c01) - (c10 - c00), c10 - c00);
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
  if (GIN && pend_base >= 0) {
    float* q = sgrad + pend_base;
    red_add_shared(q, pend[0]);
    red_add_shared(q + 1, pend[1]);
    red_add_shared(q + P, pend[2]);
    red_add_shared(q + P + 1, pend[3]);
  }
}

// Adds the brick positions inside the input to grad_in: warps take brick rows,
// lanes consecutive x; zeros (no contribution) are skipped.  All threads.
template <int NW>
__device__ __forceinline__ void flush_grad_brick(const VolConst& vc, const BrickGeom& bg,
                                                 const float* sgrad, float* gin) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int nx = vc.nx, ny = vc.ny, nz = vc.nz;
  const int lx = bg.lo[0], ly = bg.lo[1], lz = bg.lo[2];
  const int xs = max(lx, 0), xe = min(lx + bg.bx - 1, nx - 1);
  const int y0 = max(ly, 0), y1 = min(ly + bg.by - 1, ny - 1);
  const int z0 = max(lz, 0), z1 = min(lz + bg.bz - 1, nz - 1);
  if (xs > xe || y0 > y1 || z0 > z1) return;
  const int ry = y1 - y0 + 1, rows = ry * (z1 - z0 + 1);
  for (int r = warp; r < rows; r += NW) {
    const int ez = small_div(r, ry), ey = r - ez * ry;
    const int y = y0 + ey, z = z0 + ez;
    const float* src = sgrad + (((z - lz) * bg.BY + (y - ly)) * bg.P + bg.shi - lx);
    float* dst = gin + (z * ny + y) * nx;
    for (int x = xs + lane; x <= xe; x += 32) {
      const float v = src[x];
      if (v != 0.0f) red_add_global(dst + x, v);
    }
  }
}

// TXW lanes along x, NW warps, QZ quads per thread (tiles TXW x (32/TXW) NW x
// 4 QZ), CAP brick capacity (elements), MB min CTAs per SM.  Dynamic shared
// memory: CAP floats of image brick (GT) + CAP floats of gradient brick (GIN).
template <int TXW, int NW, int QZ, int CAP, int MB, bool GIN, bool GT>
__global__ void __launch_bounds__(NW * 32, MB)
    k_bwd_brick(const aug_volume_desc* __restrict__ descs, int n_vols,
                const VolConst* __restrict__ tab, const float* const* gout,
                float* const* gin, double* partials, WsHeader* ws) {
  constexpr int TX = TXW, TY = (32 / TXW) * NW, TZ = 4 * QZ;
  extern __shared__ __align__(16) unsigned char brick_smem[];
  float* simg = (float*)brick_smem;
  float* sgrad = simg + (GT ? CAP : 0);
  __shared__ BwdShared<NW> sh;
  __shared__ SchedSmem<NW * 32> sm;
  __shared__ BrickGeom bgs;
  __shared__ __align__(8) unsigned long long bar_word;
  const uint32_t bar = smem_addr(&bar_word);
  if (GT && threadIdx.x == 0) {
    mbar_init_cta(bar, NW * 32);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();
  uint32_t parity = 0;
  bool failed = false;
  int staged = -1;
  // Threads 0..11 own sh.acc[0..11]: they zero, accumulate and flush it.
  auto flush_partials = [&]() {
    if (GT && staged >= 0 && threadIdx.x < 12)
      partials[((size_t)blockIdx.x * n_vols + staged) * 12 + threadIdx.x] = sh.acc[threadIdx.x];
  };
  for_each_tile_t<NW, BoxTiles<TX, TY, TZ>>(
      descs, n_vols, sm,
      [&](int c0, int cnt) {
        if (GT)
          for (int i = threadIdx.x; i < cnt * 12; i += blockDim.x)
            partials[((size_t)blockIdx.x * n_vols + c0) * 12 + i] = 0.0;
        __syncthreads();
      },
      [&](int v, int t, long long) {
        if (v != staged) {
          flush_partials();
          if (GT && threadIdx.x < 12) sh.acc[threadIdx.x] = 0.0;
          staged = v;
        }
        const VolConst& vc = tab[v];
        if (!vc.ok || failed) return;
        __syncthreads();  // every thread is done with the previous tile's bricks
        const TileCoord tc = tile_coord_box<TXW, NW, QZ>(t, vc.onx, vc.ony, vc.onz);
        brick_geometry<TX, TY, TZ, CAP>(vc, t, bgs);
        __syncthreads();
        const BrickGeom bg = bgs;
        const float* g = gout[v];
        float* gi = GIN ? gin[v] : nullptr;
        if (bg.mode == BRICK_EXTERIOR) return;  // every tap is fill: no gradient
        if (bg.mode == BRICK_DIRECT) {
          if (vc.dtype == AUG_I16)
            bwd_tile_tc<int16_t, NW, GIN, GT>(vc, sh, tc, g, gi);
          else
            bwd_tile_tc<float, NW, GIN, GT>(vc, sh, tc, g, gi);
          return;
        }
        if (GIN) {
          float4* z4 = reinterpret_cast<float4*>(sgrad);
          const int n4 = (bg.PBY * bg.bz + 8 + 3) >> 2;
          for (int i = threadIdx.x; i < n4; i += NW * 32) z4[i] = make_float4(0.f, 0.f, 0.f, 0.f);
        }
        if (GT) {
          asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
          const uint32_t bytes = stage_rows_bulk<NW * 32>(vc, bg, simg, bar);
          mbar_arrive_tx(bar, bytes);
          const bool ok = mbar_wait_bounded(bar, parity);
          parity ^= 1u;
          if (__syncthreads_or(!ok)) {
            if (threadIdx.x == 0) record_error(ws, AUG_ERR_TIMEOUT, v);
            mbar_wait_bounded(bar, parity ^ 1u);
            failed = true;
            return;
          }
        } else {
          __syncthreads();
        }
        float acc[6] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
        bwd_brick_run<GIN, GT>(vc, bg, tc, simg, sgrad, g, acc);
        if (GT) bwd_reduce_tile<NW>(sh, tc, acc);  // ends with a barrier
        else if (GIN) __syncthreads();
        if (GIN) flush_grad_brick<NW>(vc, bg, sgrad, gi);
      });
  flush_partials();
}

// ---- host side --------------------------------------------------------------------
namespace {
using BwdBrickK = void (*)(const aug_volume_desc*, int, const VolConst*, const float* const*,
                           float* const*, double*, WsHeader*);
struct BwdBrickVariant {
  int threads, cap;
  BwdBrickK k[3];  // [GIN && GT, GIN only, GT only]
  const char* name;
};
#define BWDB_V(TXW, NW, QZ, CAP, MB, NAME)                                       \
  {                                                                              \
    NW * 32, CAP,                                                                \
        {k_bwd_brick<TXW, NW, QZ, CAP, MB, true, true>,                          \
         k_bwd_brick<TXW, NW, QZ, CAP, MB, true, false>,                         \
         k_bwd_brick<TXW, NW, QZ, CAP, MB, false, true>},                        \
        NAME                                                                     \
  }
// (lanes along x, warps, quads per thread, brick capacity, min CTAs/SM)
const BwdBrickVariant kBwdBrick[] = {
    BWDB_V(16, 8, 2, 9728, 2, "bbrick16x16x8_c9728"),
    BWDB_V(16, 4, 4, 9728, 2, "bbrick16x8x16_c9728"),
    BWDB_V(16, 8, 4, 16384, 1, "bbrick16x16x16_c16384"),
    BWDB_V(32, 4, 2, 8192, 2, "bbrick32x4x8_c8192"),
};
#undef BWDB_V
}  // namespace

int bwd_brick_num_variants() { return (int)(sizeof(kBwdBrick) / sizeof(kBwdBrick[0])); }
const char* bwd_brick_variant_name(int v) { return kBwdBrick[v].name; }

// The brick adjoint kernel (after the prologue and the zeroing of grad_in,
// which launch_bwd issues); returns the grid used (for the finalize).
cudaError_t launch_bwd_brick(int variant, const aug_volume_desc* d, int n,
                             const float* const* gout, float* const* gin, bool want_gt,
                             VolConst* tab, double* partials, WsHeader* ws, cudaStream_t st,
                             int* grid_out) {
  const BwdBrickVariant& bv = kBwdBrick[variant];
  const bool want_gin = gin != nullptr;
  const BwdBrickK kern = bv.k[want_gin ? (want_gt ? 0 : 1) : 2];
  const size_t smem = (size_t)bv.cap * sizeof(float) * ((want_gin ? 1 : 0) + (want_gt ? 1 : 0));
  cudaError_t e = cudaFuncSetAttribute((const void*)kern,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  const int grid = persistent_grid((const void*)kern, bv.threads, smem);
  if (grid <= 0) return cudaErrorInvalidConfiguration;
  kern<<<grid, bv.threads, smem, st>>>(d, n, tab, gout, gin, partials, ws);
  *grid_out = grid;
  return cudaGetLastError();
}

}  // namespace augk
