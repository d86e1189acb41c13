// Forward augmentation kernels (Sec. 4): affine coordinate map, trilinear
// image sample, nearest label sample, intensity affine, Philox noise.
//
//  * k_fwd_batched: ONE persistent launch for a whole batch of unequal
//    volumes.  The CTAs take the tiles of the concatenated tile list of all
//    volumes in order, each claiming the next unclaimed tile when it finishes
//    one, so CTAs that run at the same time work on neighbouring tiles of the
//    same volume (the input they gather from stays in L2) and all of them
//    finish together.
//  * k_fwd_volume: the plain form -- one launch per volume, one CTA per tile,
//    the volume's constants passed by value.
//
// The per-tile code is in fwd.cuh.  The shared-memory brick kernel and its
// variants are in fwd_brick.cu; they follow this file's variants in the
// variant numbering of op 0.
#include "fwd.cuh"

namespace augk {

// MB: minimum resident CTAs per SM requested from the register allocator
// (1 = no constraint); part of the variant, chosen by measurement.  Tiles are
// handed out dynamically (counter = the workspace's tile counter, set to the
// grid size by the prologue), which keeps every SM busy until the last tiles.
// ZR: fully interior z-runs reuse the z + 1 plane of taps (ZPlane).
template <int NW, int QZ, int MB, int PD, bool ZR = false>
__global__ void __launch_bounds__(NW * 32, MB)
    k_fwd_batched(const aug_volume_desc* __restrict__ descs, int n_vols,
                  const VolConst* __restrict__ tab, const PhiloxKey key,
                  unsigned long long* counter) {
  __shared__ SchedSmem<NW * 32> sm;
  for_each_tile_dynamic<NW, QZ, true>(descs, n_vols, sm, counter, [&](int v, int t, long long) {
    const VolConst& vc = tab[v];
    if (vc.ok && (vc.out_image != nullptr || vc.out_label != nullptr))
      fwd_tile<NW, QZ, PD, ZR>(vc, t, key);
  });
}

// Box-tiled form: each warp covers TXW x (32 / TXW) output positions (x, y)
// instead of 32 consecutive positions of a row, so a rotated warp's gathers
// fall on fewer input lines; stores are TXW-wide row segments.
template <int TXW, int NW, int QZ, int MB, int PD, bool ZR>
__global__ void __launch_bounds__(NW * 32, MB)
    k_fwd_batched_box(const aug_volume_desc* __restrict__ descs, int n_vols,
                      const VolConst* __restrict__ tab, const PhiloxKey key,
                      unsigned long long* counter) {
  __shared__ SchedSmem<NW * 32> sm;
  for_each_tile_dynamic_t<NW, BoxTiles<TXW, (32 / TXW) * NW, 4 * QZ>>(
      descs, n_vols, sm, counter, [&](int v, int t, long long) {
        const VolConst& vc = tab[v];
        if (vc.ok && (vc.out_image != nullptr || vc.out_label != nullptr))
          fwd_tile_direct<QZ, PD, ZR>(vc, box_tile_coord<TXW, NW, QZ>(t, vc.onx, vc.ony, vc.onz),
                                      key);
      });
}

// The volume's constants come by value, built on the host from a descriptor
// that the host has already checked.
template <int NW, int QZ, int MB, int PD>
__global__ void __launch_bounds__(NW * 32, MB)
    k_fwd_volume(const VolConst vc, const PhiloxKey key) {
  fwd_tile<NW, QZ, PD>(vc, blockIdx.x, key);
}

// The same on box patches (one CTA per box tile).
template <int TXW, int NW, int QZ, int MB, int PD, bool ZR>
__global__ void __launch_bounds__(NW * 32, MB)
    k_fwd_volume_box(const VolConst vc, const PhiloxKey key) {
  fwd_tile_direct<QZ, PD, ZR>(vc, box_tile_coord<TXW, NW, QZ>(blockIdx.x, vc.onx, vc.ony, vc.onz),
                              key);
}

// ---- host launchers ----------------------------------------------------------
namespace {
using FwdBK = void (*)(const aug_volume_desc*, int, const VolConst*, const PhiloxKey,
                       unsigned long long*);
using FwdVK = void (*)(const VolConst, const PhiloxKey);
struct FwdVariant {
  int nw, qz;
  FwdBK batched;
  FwdVK volume;
  int txw;  // box patches of txw lanes per row (volume kernel too); 0: flat plane mapping
};
#define FWD_V(NW, QZ, MB, PD) \
  { NW, QZ, k_fwd_batched<NW, QZ, MB, PD>, k_fwd_volume<NW, QZ, MB, PD>, 0 }
#define FWD_Z(NW, QZ, MB) \
  { NW, QZ, k_fwd_batched<NW, QZ, MB, 1, true>, k_fwd_volume<NW, QZ, MB, 1>, 0 }
#define FWD_B(TXW, NW, QZ, MB)                                     \
  {                                                                \
    NW, QZ, k_fwd_batched_box<TXW, NW, QZ, MB, 1, true>,           \
        k_fwd_volume_box<TXW, NW, QZ, MB, 1, true>, TXW            \
  }
#define FWD_Z2(NW, QZ, MB) \
  { NW, QZ, k_fwd_batched<NW, QZ, MB, 2, true>, k_fwd_volume<NW, QZ, MB, 2>, 0 }
// (warps per CTA, quads per thread, min CTAs per SM, pipeline depth)
const FwdVariant kFwd[] = {FWD_V(4, 8, 8, 2),  FWD_V(4, 8, 1, 2),  FWD_V(4, 8, 6, 4),
                           FWD_V(4, 8, 8, 1),  FWD_V(4, 8, 12, 1), FWD_V(4, 8, 10, 2),
                           FWD_V(8, 4, 4, 1),  FWD_V(8, 4, 6, 1),  FWD_V(8, 4, 4, 2),
                           FWD_V(4, 4, 12, 1), FWD_V(2, 8, 16, 1), FWD_V(4, 8, 9, 2),
                           FWD_Z(2, 8, 16),    FWD_Z(4, 8, 8),     FWD_Z(2, 8, 12),
                           FWD_V(2, 8, 12, 1), FWD_V(2, 8, 10, 1), FWD_Z(2, 8, 10),
                           FWD_V(2, 8, 12, 2), FWD_V(2, 8, 10, 2), FWD_Z(2, 8, 14),
                           FWD_Z2(2, 8, 12),   FWD_Z2(2, 8, 10),   FWD_Z2(4, 8, 6),
                           FWD_Z(2, 10, 12),   FWD_Z(1, 8, 24),    FWD_Z(1, 10, 24),
                           FWD_B(8, 1, 10, 24), FWD_B(8, 2, 10, 12), FWD_B(8, 3, 10, 8),
                           FWD_B(8, 2, 8, 12),  FWD_B(8, 2, 10, 14), FWD_B(8, 1, 10, 28),
                           FWD_B(8, 2, 8, 14)};
#undef FWD_V
#undef FWD_Z
#undef FWD_Z2
#undef FWD_B
const char* kFwdNames[] = {"t32x4x32_pd2_32w", "t32x4x32_pd2",     "t32x4x32_pd4_24w",
                           "t32x4x32_pd1_32w", "t32x4x32_pd1_48w", "t32x4x32_pd2_40w",
                           "t32x8x16_pd1_32w", "t32x8x16_pd1_48w", "t32x8x16_pd2_32w",
                           "t32x4x16_pd1_48w", "t32x2x32_pd1_32w", "t32x4x32_pd2_36w",
                           "t32x2x32_pd1_32w_zr", "t32x4x32_pd1_32w_zr", "t32x2x32_pd1_24w_zr",
                           "t32x2x32_pd1_24w",    "t32x2x32_pd1_20w",    "t32x2x32_pd1_20w_zr",
                           "t32x2x32_pd2_24w",    "t32x2x32_pd2_20w",    "t32x2x32_pd1_28w_zr",
                           "t32x2x32_pd2_24w_zr", "t32x2x32_pd2_20w_zr", "t32x4x32_pd2_24w_zr",
                           "t32x2x40_pd1_24w_zr", "t32x1x32_pd1_24w_zr", "t32x1x40_pd1_24w_zr",
                           "b8x4x40_pd1_24w_zr",  "b8x8x40_pd1_24w_zr",  "b8x12x40_pd1_24w_zr",
                           "b8x8x32_pd1_24w_zr",  "b8x8x40_pd1_28w_zr",  "b8x4x40_pd1_28w_zr",
                           "b8x8x32_pd1_28w_zr"};
}  // namespace

constexpr int kDirectVariants = (int)(sizeof(kFwd) / sizeof(kFwd[0]));
static_assert(sizeof(kFwdNames) / sizeof(kFwdNames[0]) == sizeof(kFwd) / sizeof(kFwd[0]),
              "one name per forward variant");
// Variant of the plain one-volume-per-launch form when the selected batched
// variant is a flat-mapped tap-reuse or register-budget variant (12 and up,
// but not a box variant, whose own one-volume kernel runs) or a brick
// variant: the one-volume kernel of the variant measured fastest per volume.
constexpr int kPlainVariants = 12;
constexpr int kDirectDefault = 10;

int fwd_num_variants() { return kDirectVariants + fwd_brick_num_variants(); }
const char* fwd_variant_name(int v) {
  return v < kDirectVariants ? kFwdNames[v] : fwd_brick_variant_name(v - kDirectVariants);
}

cudaError_t launch_fwd_batched(int variant, const aug_volume_desc* d, int n, unsigned k0,
                               unsigned k1, VolConst* tab, WsHeader* ws, cudaStream_t st) {
  if (variant >= kDirectVariants)
    return launch_fwd_brick(variant - kDirectVariants, d, n, k0, k1, tab, ws, st);
  const FwdVariant& fv = kFwd[variant];
  if (ws == nullptr) return cudaErrorInvalidValue;
  const int block = fv.nw * 32;
  // The forward keeps no per-CTA partials: up to 32 one- or two-warp CTAs per SM.
  const int grid = persistent_grid((const void*)fv.batched, block, 0, 32);
  if (grid <= 0) return cudaErrorInvalidConfiguration;
  // The prologue sets the tile counter to the grid size: CTA b takes tile b
  // first and claims later tiles from the counter.
  cudaError_t e = launch_prepare(d, n, NEED_IMAGE_IF_OUT, false, nullptr, nullptr, false, tab, ws,
                                 st, (unsigned long long)grid);
  if (e != cudaSuccess) return e;
  fv.batched<<<grid, block, 0, st>>>(d, n, tab, philox_schedule(k0, k1), &ws->tile_next);
  return cudaGetLastError();
}

cudaError_t launch_fwd_volume(int variant, const aug_volume_desc& h, unsigned k0, unsigned k1,
                              cudaStream_t st) {
  const bool own = variant < kPlainVariants ||
                   (variant < kDirectVariants && kFwd[variant].txw > 0);
  const FwdVariant& fv = kFwd[own ? variant : kDirectDefault];
  long long tiles;
  if (fv.txw > 0) {
    // Box patches (box_tile_coord): txw x (32 / txw) * NW positions x 4*QZ slices.
    const long long tx = fv.txw, ty = (32 / fv.txw) * fv.nw, tz = 4 * fv.qz;
    tiles = ((h.out_nx + tx - 1) / tx) * ((h.out_ny + ty - 1) / ty) * ((h.out_nz + tz - 1) / tz);
  } else {
    // Flat plane mapping (tile_coord_flat): NW*32 plane positions x 4*QZ slices.
    const long long plane = (long long)h.out_nx * h.out_ny;
    tiles = ((plane + fv.nw * 32 - 1) / (fv.nw * 32)) *
            ((h.out_nz + 4 * fv.qz - 1) / (4 * fv.qz));
  }
  if (tiles <= 0 || tiles > 0x7fffffffLL) return cudaErrorInvalidConfiguration;
  VolConst vc;
  make_volconst(h, true, vc, false);
  fv.volume<<<(unsigned)tiles, fv.nw * 32, 0, st>>>(vc, philox_schedule(k0, k1));
  return cudaGetLastError();
}

}  // namespace augk
