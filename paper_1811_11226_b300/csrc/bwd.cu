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
// grad_in is accumulated with float atomics straight into the caller's
// buffer (zeroed first by k_zero_grad_in).  grad_T: per thread, S_r = sum
// a g dv_r and K_r = sum a g dv_r k over its z-run (i, j fixed); the tile's
// 12 sums (i S_r, j S_r, K_r, S_r) are warp-reduced, block-reduced in a
// fixed order, accumulated per CTA and volume in double, written to
// workspace partials [CTA][volume][12], and summed over CTAs in a fixed order
// by k_bwd_finalize: bitwise reproducible.
#include "bwd.cuh"

namespace augk {

template <int NW, int QZ, bool GIN, bool GT, bool XM = false, bool QS = false, bool PR = false,
          int TXW = 32>
__global__ void __launch_bounds__(NW * 32, 1024 / (NW * 32))
    k_bwd_batched(const aug_volume_desc* __restrict__ descs, int n_vols,
                  const VolConst* __restrict__ tab, const float* const* gout,
                  float* const* gin, double* partials) {
  __shared__ BwdShared<NW> sh;
  __shared__ SchedSmem<NW * 32> sm;
  int staged = -1;
  // Threads 0..11 own sh.acc[0..11]: they zero, accumulate and flush it, so
  // the flush needs no barrier.
  auto flush = [&]() {
    if (GT && staged >= 0 && threadIdx.x < 12)
      partials[((size_t)blockIdx.x * n_vols + staged) * 12 + threadIdx.x] = sh.acc[threadIdx.x];
  };
  for_each_tile_t<NW, BoxTiles<TXW, (32 / TXW) * NW, 4 * QZ>>(
      descs, n_vols, sm,
      [&](int c0, int cnt) {
        // This CTA's partials of the chunk's volumes start at zero (volumes in
        // which it has no tile keep them).
        if (GT)
          for (int i = threadIdx.x; i < cnt * 12; i += blockDim.x)
            partials[((size_t)blockIdx.x * n_vols + c0) * 12 + i] = 0.0;
        __syncthreads();
      },
      [&](int v, int t, long long) {
        if (v != staged) {
          flush();
          if (GT && threadIdx.x < 12) sh.acc[threadIdx.x] = 0.0;
          staged = v;
        }
        const VolConst& vc = tab[v];
        if (!vc.ok) return;
        const float* g = gout[v];
        float* gi = GIN ? gin[v] : nullptr;
        if (vc.dtype == AUG_I16)
          bwd_tile<int16_t, NW, QZ, GIN, GT, false, XM, QS, PR, TXW>(vc, sh, t, g, gi);
        else
          bwd_tile<float, NW, QZ, GIN, GT, false, XM, QS, PR, TXW>(vc, sh, t, g, gi);
      });
  flush();
}

// Input bounding box of one output tile: the tile is a box of output indices,
// its image under the affine map is a parallelepiped whose coordinate extrema
// sit at the 8 corners, so floor(min)..floor(max)+1 per axis (clipped to the
// volume) holds every in-volume tap of the tile.  Threads 0..2 each reduce one
// axis; lo > hi means no in-volume tap on that axis.
template <int NW, int QZ>
__device__ __forceinline__ void tile_bbox(const VolConst& vc, int t, int* lo, int* hi) {
  if (threadIdx.x < 3) {
    const int r = threadIdx.x;
    const int tx_n = (vc.onx + 31) / 32, ty_n = (vc.ony + NW - 1) / NW;
    const int tx = t % tx_n, ty = (t / tx_n) % ty_n, tz = t / (tx_n * ty_n);
    const int i0 = tx * 32, j0 = ty * NW, k0 = tz * 4 * QZ;
    const int ii[2] = {i0, min(i0 + 31, vc.onx - 1)};
    const int jj[2] = {j0, min(j0 + NW - 1, vc.ony - 1)};
    const int kk[2] = {k0, min(k0 + 4 * QZ - 1, vc.onz - 1)};
    int mn = 0x7fffffff, mx = -0x7fffffff;
#pragma unroll
    for (int c = 0; c < 8; ++c) {
      const int f = q40_floor(coord_q40(vc.tq[r], ii[c & 1], jj[(c >> 1) & 1], kk[c >> 2]));
      mn = min(mn, f);
      mx = max(mx, f);
    }
    const int n = r == 0 ? vc.nx : (r == 1 ? vc.ny : vc.nz);
    lo[r] = max(mn, 0);
    hi[r] = min(mx + 1, n - 1);
  }
}

// Adjoint with the input gradient accumulated per tile in a shared-memory
// brick (CAP floats) and flushed with coalesced global atomics, one per
// non-zero brick element, row by row.  Tiles whose bounding box exceeds the
// brick fall back to direct global atomics.  The flush leaves the brick
// zeroed for the next tile.
template <int NW, int QZ, bool GT, int CAP>
__global__ void __launch_bounds__(NW * 32)
    k_bwd_smem(const aug_volume_desc* __restrict__ descs, int n_vols,
               const VolConst* __restrict__ tab, const float* const* gout, float* const* gin,
               double* partials) {
  extern __shared__ float brick[];
  __shared__ BwdShared<NW> sh;
  __shared__ SchedSmem<NW * 32> sm;
  __shared__ int box_lo[3], box_hi[3];
  for (int e = threadIdx.x; e < CAP; e += blockDim.x) brick[e] = 0.0f;
  int staged = -1;
  auto flush_partials = [&]() {
    if (GT && staged >= 0 && threadIdx.x < 12)
      partials[((size_t)blockIdx.x * n_vols + staged) * 12 + threadIdx.x] = sh.acc[threadIdx.x];
  };
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for_each_tile<NW, QZ>(
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
        if (!vc.ok) return;
        const float* g = gout[v];
        float* gi = gin[v];
        __syncthreads();  // every thread is done with the previous tile's box
        tile_bbox<NW, QZ>(vc, t, box_lo, box_hi);
        __syncthreads();
        const int lx = box_lo[0], ly = box_lo[1], lz = box_lo[2];
        const int bx = box_hi[0] - lx + 1, by = box_hi[1] - ly + 1, bz = box_hi[2] - lz + 1;
        const bool empty = bx <= 0 || by <= 0 || bz <= 0;
        const long long size = empty ? 0 : (long long)bx * by * bz;
        if (size > 0 && size <= CAP) {
          const BrickMap bm{brick, bx, bx * by, -(lx + ly * bx + lz * bx * by)};
          if (vc.dtype == AUG_I16)
            bwd_tile<int16_t, NW, QZ, true, GT, true>(vc, sh, t, g, gi, bm);
          else
            bwd_tile<float, NW, QZ, true, GT, true>(vc, sh, t, g, gi, bm);
          __syncthreads();
          const int nxy = vc.nx * vc.ny;
          for (int row = warp; row < by * bz; row += NW) {
            const int ey = row % by, ez = row / by;
            float* src = brick + row * bx;
            float* dst = gi + ((lz + ez) * nxy + (ly + ey) * vc.nx + lx);
            for (int ex = lane; ex < bx; ex += 32) {
              const float val = src[ex];
              if (val != 0.0f) {
                red_add_global(dst + ex, val);
                src[ex] = 0.0f;
              }
            }
          }
          __syncthreads();
        } else {
          if (vc.dtype == AUG_I16)
            bwd_tile<int16_t, NW, QZ, true, GT, false>(vc, sh, t, g, gi);
          else
            bwd_tile<float, NW, QZ, true, GT, false>(vc, sh, t, g, gi);
        }
      });
  flush_partials();
}

// Zero every grad_in volume (float32 input shape) before the scatter.
__global__ void k_zero_grad_in(const aug_volume_desc* __restrict__ descs, int n_vols,
                               float* const* gin) {
  for (int v = 0; v < n_vols; ++v) {
    float* p = gin[v];
    const aug_volume_desc& d = descs[v];
    if (p == nullptr || d.in_nx < 1 || d.in_ny < 1 || d.in_nz < 1 || d.in_nx > MAX_DIM ||
        d.in_ny > MAX_DIM || d.in_nz > MAX_DIM)
      continue;
    const long long n = (long long)d.in_nx * d.in_ny * d.in_nz;
    if (n >= (1LL << 31)) continue;
    const long long stride = (long long)gridDim.x * blockDim.x;
    const long long t0 = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if ((((uintptr_t)p) & 15) == 0) {
      float4* p4 = reinterpret_cast<float4*>(p);
      const long long n4 = n >> 2;
      for (long long m = t0; m < n4; m += stride) p4[m] = make_float4(0.f, 0.f, 0.f, 0.f);
      for (long long m = (n4 << 2) + t0; m < n; m += stride) p[m] = 0.0f;
    } else {
      for (long long m = t0; m < n; m += stride) p[m] = 0.0f;
    }
  }
}

// grad_affine[v][m] = sum over CTAs of partials[cta][v][m], fixed order.
__global__ void k_bwd_finalize(const double* __restrict__ partials, int n_ctas, int n_vols,
                               float* grad_affine) {
  const int v = blockIdx.x;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  for (int m = warp; m < 12; m += blockDim.x >> 5) {
    double s = 0.0;
    for (int c = lane; c < n_ctas; c += 32) s += partials[((size_t)c * n_vols + v) * 12 + m];
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) s += __shfl_xor_sync(FULL_MASK, s, off);
    if (lane == 0) grad_affine[(size_t)v * 12 + m] = (float)s;
  }
}

// ---- host launchers ------------------------------------------------------------
namespace {
using BwdK = void (*)(const aug_volume_desc*, int, const VolConst*, const float* const*,
                      float* const*, double*);
struct BwdVariant {
  int nw, qz, cap;  // cap > 0: input gradient through a shared brick of cap floats
  BwdK k[4];        // [GIN*2 + GT]
};
#define BWD_V(NW, QZ)                                                                  \
  {                                                                                    \
    NW, QZ, 0,                                                                         \
        {k_bwd_batched<NW, QZ, false, false>, k_bwd_batched<NW, QZ, false, true>,      \
         k_bwd_batched<NW, QZ, true, false>, k_bwd_batched<NW, QZ, true, true> }       \
  }
#define BWD_S(NW, QZ, CAP)                                                             \
  {                                                                                    \
    NW, QZ, CAP,                                                                       \
        {k_bwd_batched<NW, QZ, false, false>, k_bwd_batched<NW, QZ, false, true>,      \
         k_bwd_smem<NW, QZ, false, CAP>, k_bwd_smem<NW, QZ, true, CAP> }               \
  }
#define BWD_X(NW, QZ)                                                                  \
  {                                                                                    \
    NW, QZ, 0,                                                                         \
        {k_bwd_batched<NW, QZ, false, false>, k_bwd_batched<NW, QZ, false, true>,      \
         k_bwd_batched<NW, QZ, true, false, true>, k_bwd_batched<NW, QZ, true, true, true> } \
  }
// x-merge with predicated reductions (PR), optionally per-quad re-classified;
// the affine gradient alone takes the whole-run form (the quad-wise one is
// slower there: 2.53 against 2.46 ms for the int16 training step).
#define BWD_XP(NW, QZ, QS)                                                               \
  {                                                                                      \
    NW, QZ, 0,                                                                           \
        {k_bwd_batched<NW, QZ, false, false>,                                            \
         k_bwd_batched<NW, QZ, false, true>,                                             \
         k_bwd_batched<NW, QZ, true, false, true, QS, true>,                             \
         k_bwd_batched<NW, QZ, true, true, true, QS, true> }                             \
  }
// The same on box patches: each warp covers TXW x (32 / TXW) output positions.
#define BWD_XPB(TXW, NW, QZ, QS)                                                         \
  {                                                                                      \
    NW, QZ, 0,                                                                           \
        {k_bwd_batched<NW, QZ, false, false>,                                            \
         k_bwd_batched<NW, QZ, false, true, false, false, false, TXW>,                   \
         k_bwd_batched<NW, QZ, true, false, true, QS, true, TXW>,                        \
         k_bwd_batched<NW, QZ, true, true, true, QS, true, TXW> }                        \
  }
const BwdVariant kBwd[] = {BWD_V(8, 4),         BWD_V(4, 4),        BWD_V(8, 2),
                           BWD_V(8, 8),         BWD_S(16, 2, 24576), BWD_S(8, 2, 16384),
                           BWD_S(8, 4, 24576),  BWD_X(8, 4),        BWD_X(8, 8),
                           BWD_XP(8, 8, false), BWD_XP(8, 8, true), BWD_XP(8, 4, true),
                           BWD_XPB(8, 8, 8, true), BWD_XPB(16, 8, 8, true), BWD_XPB(8, 4, 8, true),
                           BWD_XPB(16, 4, 8, true), BWD_XPB(16, 8, 4, true), BWD_XPB(16, 16, 8, true)};
#undef BWD_V
#undef BWD_S
#undef BWD_X
#undef BWD_XP
#undef BWD_XPB
const char* kBwdNames[] = {"t32x8x16_atomic",   "t32x4x16_atomic",  "t32x8x8_atomic",
                           "t32x8x32_atomic",   "t32x16x8_brick96k", "t32x8x8_brick64k",
                           "t32x8x16_brick96k", "t32x8x16_atomic_xmerge",
                           "t32x8x32_atomic_xmerge", "t32x8x32_atomic_xmerge_pr",
                           "t32x8x32_atomic_xmerge_qs_pr", "t32x8x16_atomic_xmerge_qs_pr",
                           "b8x32x32_atomic_xmerge_qs_pr", "b16x16x32_atomic_xmerge_qs_pr",
                           "b8x16x32_atomic_xmerge_qs_pr", "b16x8x32_atomic_xmerge_qs_pr",
                           "b16x16x16_atomic_xmerge_qs_pr", "b16x32x32_atomic_xmerge_qs_pr"};
}  // namespace

constexpr int kBwdDirect = (int)(sizeof(kBwd) / sizeof(kBwd[0]));
static_assert(sizeof(kBwdNames) / sizeof(kBwdNames[0]) == sizeof(kBwd) / sizeof(kBwd[0]),
              "one name per adjoint variant");

// Variants 0 .. kBwdDirect - 1 are the kernels of this file, the following
// ones the brick adjoint (bwd_brick.cu), then the gather adjoint
// (bwd_gather.cu, whose affine gradient is the output-driven pass of variant
// kGatherGt).
constexpr int kGatherGt = 8;
int bwd_num_variants() {
  return kBwdDirect + bwd_brick_num_variants() + bwd_gather_num_variants();
}
const char* bwd_variant_name(int v) {
  if (v < kBwdDirect) return kBwdNames[v];
  v -= kBwdDirect;
  if (v < bwd_brick_num_variants()) return bwd_brick_variant_name(v);
  return bwd_gather_variant_name(v - bwd_brick_num_variants());
}

cudaError_t launch_bwd(int variant, const aug_volume_desc* d, int n, const float* const* gout,
                       float* const* gin, float* gaff, VolConst* tab, double* partials,
                       WsHeader* ws, cudaStream_t st) {
  const bool want_gt = gaff != nullptr;
  if (gin == nullptr && !want_gt) return cudaSuccess;
  const bool want_gin0 = gin != nullptr;
  cudaError_t e =
      launch_prepare(d, n, NEED_IMAGE_ALWAYS, want_gin0, gout, gin, false, tab, ws, st);
  if (e != cudaSuccess) return e;
  if (variant >= kBwdDirect + bwd_brick_num_variants()) {
    // Gather: grad_in input-driven (every element written, no zeroing), then
    // grad_T from the output-driven pass alone.
    if (want_gin0) {
      e = launch_bwd_gather(variant - kBwdDirect - bwd_brick_num_variants(), d, n, gout, gin,
                            tab, ws, st);
      if (e != cudaSuccess) return e;
    }
    if (!want_gt) return cudaSuccess;
    variant = kGatherGt;
    gin = nullptr;
  }
  const bool want_gin = gin != nullptr;
  if (want_gin) {
    const int zgrid = persistent_grid((const void*)k_zero_grad_in, 256, 0);
    if (zgrid <= 0) return cudaErrorInvalidConfiguration;
    k_zero_grad_in<<<zgrid, 256, 0, st>>>(d, n, gin);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
  }
  if (variant >= kBwdDirect) {
    int grid = 0;
    e = launch_bwd_brick(variant - kBwdDirect, d, n, gout, gin, want_gt, tab, partials, ws, st,
                         &grid);
    if (e != cudaSuccess) return e;
    if (want_gt) {
      k_bwd_finalize<<<n, 384, 0, st>>>(partials, grid, n, gaff);
      if ((e = cudaGetLastError()) != cudaSuccess) return e;
    }
    return cudaSuccess;
  }
  const BwdVariant& bv = kBwd[variant];
  const BwdK kern = bv.k[(want_gin ? 2 : 0) + (want_gt ? 1 : 0)];
  const int block = bv.nw * 32;
  const size_t smem = (want_gin && bv.cap > 0) ? (size_t)bv.cap * sizeof(float) : 0;
  if (smem > 48 * 1024) {
    e = cudaFuncSetAttribute((const void*)kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)smem);
    if (e != cudaSuccess) return e;
  }
  const int grid = persistent_grid((const void*)kern, block, smem);
  if (grid <= 0) return cudaErrorInvalidConfiguration;
  kern<<<grid, block, smem, st>>>(d, n, tab, gout, gin, partials);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  if (want_gt) {
    k_bwd_finalize<<<n, 384, 0, st>>>(partials, grid, n, gaff);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
  }
  return cudaSuccess;
}

}  // namespace augk
