// Forward augmentation kernels (Sec. 4): affine coordinate map, trilinear
// image sample, nearest label sample, intensity affine, Philox noise.
//
//  * k_fwd_batched: ONE persistent launch for a whole batch of unequal
//    volumes.  Every CTA walks the concatenated tile list of all volumes
//    (static round-robin: CTA b takes global tiles b, b+G, ...), so CTAs that
//    run at the same time work on neighbouring tiles of the same volume and
//    the input they gather from stays in L2.
//  * k_fwd_volume: the plain form -- one launch per volume, one CTA per tile,
//    descriptor passed by value.
#include "kernels.h"
#include "sample.cuh"

namespace augk {

// One z-run of one thread (4*QZ voxels at most), for a warp-uniform MODE.
template <typename TIn, int MODE, int QZ>
__device__ __forceinline__ void fwd_run(const VolConst& vc, const TileCoord& tc, long long sx,
                                        long long sy, long long sz, unsigned key0,
                                        unsigned key1) {
  const TIn* __restrict__ img = (const TIn*)vc.image;
  const long long dx = vc.tq[0][2], dy = vc.tq[1][2], dz = vc.tq[2][2];
  const int nx = vc.nx, ny = vc.ny, nz = vc.nz;
  const int onx = vc.onx, ony = vc.ony;
  const int plane = onx * ony;
  float* __restrict__ out_img = vc.out_image;
  uint8_t* __restrict__ out_lab = vc.out_label;
  const bool want_img = out_img != nullptr, want_lab = out_lab != nullptr;
  const bool noisy = vc.sigma > 0.0f;
  const float a = vc.a, b = vc.b, sigma = vc.sigma, fill = vc.fill;
  int o = (tc.k0 * ony + tc.jc) * onx + tc.ic;
#pragma unroll 1
  for (int q = 0; q < QZ; ++q) {
    const int kq = tc.k0 + 4 * q;
    if (kq >= tc.k1) break;
    float z[4] = {0.0f, 0.0f, 0.0f, 0.0f};
    if (noisy && want_img)
      quad_normals(((unsigned long long)(kq >> 2) * (unsigned)ony + (unsigned)tc.jc) *
                           (unsigned)onx + (unsigned)tc.ic,
                   vc.noise_id, key0, key1, z);
#pragma unroll
    for (int m = 0; m < 4; ++m) {
      if (kq + m < tc.k1) {
        if (want_img) {
          Taps t;
          load_taps<TIn, MODE>(img, sx, sy, sz, nx, ny, nz, fill, t);
          float c00, c10, c01, c11, c0, c1;
          const float v = trilerp(t, c00, c10, c01, c11, c0, c1);
          const float y = fmaf(sigma, z[m], fmaf(a, v, b));
          if (tc.valid) __stcs(out_img + o, y);
        }
        if (want_lab) {
          const int l = load_label<MODE>(vc.label, sx, sy, sz, nx, ny, nz, vc.fill_label);
          if (tc.valid) out_lab[o] = (uint8_t)l;
        }
        sx += dx;
        sy += dy;
        sz += dz;
        o += plane;
      }
    }
  }
}

template <typename TIn, int NW, int QZ>
__device__ __forceinline__ void fwd_tile(const VolConst& vc, int t, unsigned key0,
                                         unsigned key1) {
  const TileCoord tc = tile_coord<NW, QZ>(t, vc.onx, vc.ony, vc.onz);
  long long s[3], ds[3];
#pragma unroll
  for (int r = 0; r < 3; ++r) {
    s[r] = coord_q40(vc.tq[r], tc.ic, tc.jc, tc.k0);
    ds[r] = vc.tq[r][2];
  }
  const int mode =
      warp_mode(classify_run<true>(s, ds, tc.k1 - 1 - tc.k0, vc.nx, vc.ny, vc.nz));
  if (mode == MODE_INTERIOR)
    fwd_run<TIn, MODE_INTERIOR, QZ>(vc, tc, s[0], s[1], s[2], key0, key1);
  else if (mode == MODE_EXTERIOR)
    fwd_run<TIn, MODE_EXTERIOR, QZ>(vc, tc, s[0], s[1], s[2], key0, key1);
  else
    fwd_run<TIn, MODE_GENERAL, QZ>(vc, tc, s[0], s[1], s[2], key0, key1);
}

template <int NW, int QZ>
__global__ void __launch_bounds__(NW * 32)
    k_fwd_batched(const aug_volume_desc* __restrict__ descs, int n_vols, unsigned key0,
                  unsigned key1, WsHeader* ws) {
  __shared__ VolConst vc;
  long long base = 0;
  for (int v = 0; v < n_vols; ++v) {
    __syncthreads();
    stage_volume(descs + v, v, vc, ws, descs[v].out_image != nullptr, false);
    __syncthreads();
    if (!vc.ok) continue;
    const int nt = tiles_in<NW, QZ>(vc.onx, vc.ony, vc.onz);
    if (vc.out_image != nullptr || vc.out_label != nullptr) {
      for (long long t = first_tile(base); t < nt; t += gridDim.x) {
        if (vc.dtype == AUG_I16)
          fwd_tile<int16_t, NW, QZ>(vc, (int)t, key0, key1);
        else
          fwd_tile<float, NW, QZ>(vc, (int)t, key0, key1);
      }
    }
    base += nt;
  }
}

template <int NW, int QZ>
__global__ void __launch_bounds__(NW * 32)
    k_fwd_volume(const aug_volume_desc desc, unsigned key0, unsigned key1) {
  __shared__ VolConst vc;
  stage_volume(&desc, 0, vc, nullptr, desc.out_image != nullptr, false);
  __syncthreads();
  if (!vc.ok) return;
  if (vc.dtype == AUG_I16)
    fwd_tile<int16_t, NW, QZ>(vc, blockIdx.x, key0, key1);
  else
    fwd_tile<float, NW, QZ>(vc, blockIdx.x, key0, key1);
}

// ---- host launchers ----------------------------------------------------------
namespace {
struct FwdVariant {
  int nw, qz;
  const void* batched;
  const void* volume;
};
#define FWD_V(NW, QZ) \
  { NW, QZ, (const void*)k_fwd_batched<NW, QZ>, (const void*)k_fwd_volume<NW, QZ> }
const FwdVariant kFwd[] = {FWD_V(8, 4),  FWD_V(4, 4), FWD_V(8, 2), FWD_V(8, 8),
                           FWD_V(4, 8),  FWD_V(16, 2), FWD_V(2, 8)};
#undef FWD_V
const char* kFwdNames[] = {"tile32x8x16", "tile32x4x16", "tile32x8x8", "tile32x8x32",
                           "tile32x4x32", "tile32x16x8", "tile32x2x32"};
}  // namespace

int fwd_num_variants() { return (int)(sizeof(kFwd) / sizeof(kFwd[0])); }
const char* fwd_variant_name(int v) { return kFwdNames[v]; }

cudaError_t launch_fwd_batched(int variant, const aug_volume_desc* d, int n, unsigned k0,
                               unsigned k1, WsHeader* ws, cudaStream_t st) {
  const FwdVariant& fv = kFwd[variant];
  const int block = fv.nw * 32;
  const int grid = persistent_grid(fv.batched, block, 0);
  if (grid <= 0) return cudaErrorInvalidConfiguration;
  void* args[] = {(void*)&d, (void*)&n, (void*)&k0, (void*)&k1, (void*)&ws};
  return cudaLaunchKernel(fv.batched, dim3(grid), dim3(block), args, 0, st);
}

cudaError_t launch_fwd_volume(int variant, const aug_volume_desc& h, unsigned k0, unsigned k1,
                              cudaStream_t st) {
  const FwdVariant& fv = kFwd[variant];
  const long long tiles = (long long)((h.out_nx + 31) / 32) *
                          ((h.out_ny + fv.nw - 1) / fv.nw) *
                          ((h.out_nz + 4 * fv.qz - 1) / (4 * fv.qz));
  if (tiles <= 0 || tiles > 0x7fffffffLL) return cudaErrorInvalidConfiguration;
  aug_volume_desc copy = h;
  void* args[] = {(void*)&copy, (void*)&k0, (void*)&k1};
  return cudaLaunchKernel(fv.volume, dim3((unsigned)tiles), dim3(fv.nw * 32), args, 0, st);
}

}  // namespace augk
