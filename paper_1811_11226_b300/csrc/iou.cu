// Fused nearest-label warp + soft IOU loss, forward and backward (Sec. 5.C).
//
//   pass 1 (k_iou_pass<SUMS=true>): per output voxel, the warped label y is
//       computed in registers (exact Q.40 coordinate, floor(s + 1/2)) and the
//       class probabilities p[c] are streamed once; per class the sums
//       I = sum p [y == c], P = sum p, Y = sum [y == c] are reduced per tile
//       (warp shuffles, then a fixed-order block sum in double) and per CTA,
//       and written to workspace partials [CTA][volume][3C].
//   finalize (k_iou_finalize): one CTA per volume sums the partials over CTAs
//       in a fixed order, writes loss[b] = mean_c (1 - I/U) and the two
//       gradient values of each class: -s/U (voxels of the class) and
//       s I/U^2 (other voxels), s = 1/(B C).
//   pass 2 (k_iou_pass<SUMS=false>): recomputes the label and writes grad_p
//       (a write-only stream; p is not re-read).
// The warped labels never reach memory.
#include <map>
#include <mutex>

#include "kernels.h"
#include "sample.cuh"
#include "sched.cuh"

namespace augk {

template <int MODE, int C, bool SUMS>
__device__ __forceinline__ void iou_run(const VolConst& vc, const TileCoord& tc, long long sx,
                                        long long sy, long long sz,
                                        const float* __restrict__ p, float* __restrict__ gp,
                                        const float2* __restrict__ cf, float acc[3 * C]) {
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
      if (SUMS) {
#pragma unroll
        for (int c = 0; c < C; ++c) {
          const float pc = __ldcs(p + (size_t)c * nvox + o);
          const bool hit = y == c;
          acc[3 * c + 0] += hit ? pc : 0.0f;
          acc[3 * c + 1] += pc;
          acc[3 * c + 2] += hit ? 1.0f : 0.0f;
        }
      } else {
#pragma unroll
        for (int c = 0; c < C; ++c)
          __stcs(gp + (size_t)c * nvox + o, y == c ? coef[c].y : coef[c].x);
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

template <int NW, int QZ, int C, bool SUMS>
__global__ void __launch_bounds__(NW * 32)
    k_iou_pass(const aug_volume_desc* __restrict__ descs, int n_vols,
               const VolConst* __restrict__ tab, const float* __restrict__ p,
               float* __restrict__ gp, const float2* __restrict__ coefs, double* partials) {
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
  for_each_tile<NW, QZ>(
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
        for (int m = 0; m < 3 * C; ++m) acc[m] = 0.0f;
        const int mode =
            warp_mode(classify_run<false>(s, ds, tc.k1 - 1 - tc.k0, vc.nx, vc.ny, vc.nz));
        const size_t poff = (size_t)C * (size_t)voxoff;
        const float* pv = p + poff;
        float* gv = SUMS ? nullptr : gp + poff;
        const float2* cf = SUMS ? nullptr : coefs + (size_t)v * C;
        if (mode == MODE_INTERIOR)
          iou_run<MODE_INTERIOR, C, SUMS>(vc, tc, s[0], s[1], s[2], pv, gv, cf, acc);
        else if (mode == MODE_EXTERIOR)
          iou_run<MODE_EXTERIOR, C, SUMS>(vc, tc, s[0], s[1], s[2], pv, gv, cf, acc);
        else
          iou_run<MODE_GENERAL, C, SUMS>(vc, tc, s[0], s[1], s[2], pv, gv, cf, acc);
        if (SUMS) {
#pragma unroll
          for (int m = 0; m < 3 * C; ++m) {
            const float w = warp_sum(acc[m]);
            if (lane == 0) sh.red[warp][m] = w;
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

// One CTA per volume: loss and the per-class gradient values.
template <int C>
__global__ void k_iou_finalize(const double* __restrict__ partials, int n_ctas, int n_vols,
                               float* loss, float2* coefs) {
  __shared__ double tot[3 * C];
  const int v = blockIdx.x;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  for (int m = warp; m < 3 * C; m += blockDim.x >> 5) {
    double s = 0.0;
    for (int c = lane; c < n_ctas; c += 32)
      s += partials[((size_t)c * n_vols + v) * (3 * C) + m];
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) s += __shfl_xor_sync(FULL_MASK, s, off);
    if (lane == 0) tot[m] = s;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    const double scale = 1.0 / ((double)n_vols * (double)C);
    double lsum = 0.0;
    for (int c = 0; c < C; ++c) {
      const double I = tot[3 * c], P = tot[3 * c + 1], Y = tot[3 * c + 2];
      const double U = P + Y - I;
      double l = 0.0, g_other = 0.0, g_class = 0.0;
      if (U > 0.0) {
        l = 1.0 - I / U;
        g_other = scale * I / (U * U);
        g_class = -scale / U;
      }
      lsum += l;
      if (coefs) coefs[(size_t)v * C + c] = make_float2((float)g_other, (float)g_class);
    }
    loss[v] = (float)(lsum / C);
  }
}

// ---- host launchers ----------------------------------------------------------------
namespace {
using PassK = void (*)(const aug_volume_desc*, int, const VolConst*, const float*, float*,
                       const float2*, double*);
using FinK = void (*)(const double*, int, int, float*, float2*);
struct IouVariant {
  int nw, qz;
  PassK sums[8];
  PassK grad[8];
};
#define IOU_K(NW, QZ, S)                                                                 \
  {                                                                                      \
    k_iou_pass<NW, QZ, 1, S>, k_iou_pass<NW, QZ, 2, S>, k_iou_pass<NW, QZ, 3, S>,        \
        k_iou_pass<NW, QZ, 4, S>, k_iou_pass<NW, QZ, 5, S>, k_iou_pass<NW, QZ, 6, S>,    \
        k_iou_pass<NW, QZ, 7, S>, k_iou_pass<NW, QZ, 8, S>                               \
  }
#define IOU_V(NW, QZ) \
  { NW, QZ, IOU_K(NW, QZ, true), IOU_K(NW, QZ, false) }
const IouVariant kIou[] = {IOU_V(8, 4), IOU_V(4, 4), IOU_V(8, 8), IOU_V(4, 8)};
#undef IOU_V
#undef IOU_K
const FinK kIouFin[8] = {k_iou_finalize<1>, k_iou_finalize<2>, k_iou_finalize<3>,
                         k_iou_finalize<4>, k_iou_finalize<5>, k_iou_finalize<6>,
                         k_iou_finalize<7>, k_iou_finalize<8>};
const char* kIouNames[] = {"tile32x8x16", "tile32x4x16", "tile32x8x32", "tile32x4x32"};
}  // namespace

int iou_num_variants() { return (int)(sizeof(kIou) / sizeof(kIou[0])); }
const char* iou_variant_name(int v) { return kIouNames[v]; }

cudaError_t launch_iou(int variant, const aug_volume_desc* d, int n, const float* p, int C,
                       float* loss, float* gp, VolConst* tab, double* partials, float2* coefs,
                       WsHeader* ws, cudaStream_t st) {
  const IouVariant& iv = kIou[variant];
  const int block = iv.nw * 32;
  const PassK ks = iv.sums[C - 1];
  const int grid = persistent_grid((const void*)ks, block, 0);
  if (grid <= 0) return cudaErrorInvalidConfiguration;
  cudaError_t e = launch_prepare(d, n, NEED_IMAGE_NEVER, false, nullptr, nullptr, true, tab, ws,
                                 st);
  if (e != cudaSuccess) return e;
  ks<<<grid, block, 0, st>>>(d, n, tab, p, nullptr, nullptr, partials);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  kIouFin[C - 1]<<<n, 256, 0, st>>>(partials, grid, n, loss, gp ? coefs : nullptr);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  if (gp) {
    const PassK kg = iv.grad[C - 1];
    const int g2 = persistent_grid((const void*)kg, block, 0);
    if (g2 <= 0) return cudaErrorInvalidConfiguration;
    kg<<<g2, block, 0, st>>>(d, n, tab, p, gp, coefs, nullptr);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
  }
  return cudaSuccess;
}

}  // namespace augk

// ---- allocation-free IOU entry point ----------------------------------------------
// The same three kernels as iou_loss_fwd_bwd, with the workspace replaced by a
// fixed-size array that lives in the library's own device memory, for callers
// that may not allocate device memory themselves.
namespace augk {
namespace {

constexpr int kStaticMaxVols = 64;
constexpr int kStaticMaxClasses = 8;
constexpr int kStaticMaxCtas = 256;
constexpr size_t kStaticTableBytes =
    ((size_t)kStaticMaxVols * sizeof(VolConst) + 255) & ~(size_t)255;
constexpr size_t kStaticPartialBytes =
    (size_t)kStaticMaxCtas * kStaticMaxVols * 3 * kStaticMaxClasses * sizeof(double);
constexpr size_t kStaticCoefBytes = (size_t)kStaticMaxVols * kStaticMaxClasses * sizeof(float2);
constexpr size_t kStaticScratchBytes =
    sizeof(WsHeader) + kStaticTableBytes + kStaticPartialBytes + kStaticCoefBytes;

// Every device that loads the library holds this array until the process exits.
static __device__ __align__(256) unsigned char g_iou_scratch[kStaticScratchBytes];

std::mutex g_scratch_mu;
std::map<int, void*> g_scratch_ptr;  // device -> device address of g_iou_scratch

// Device address of the scratch array on the current device, looked up once per
// device (the host-side symbol is only a stand-in, never a device pointer).
cudaError_t scratch_address(void** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  std::lock_guard<std::mutex> lk(g_scratch_mu);
  auto it = g_scratch_ptr.find(dev);
  if (it != g_scratch_ptr.end()) {
    *out = it->second;
    return cudaSuccess;
  }
  void* p = nullptr;
  e = cudaGetSymbolAddress(&p, g_iou_scratch);
  if (e != cudaSuccess) return e;
  g_scratch_ptr[dev] = p;
  *out = p;
  return cudaSuccess;
}

}  // namespace
}  // namespace augk

extern "C" aug_status iou_loss_fwd_bwd_noalloc(const aug_volume_desc* d_descs, int n_vols,
                                               const float* d_p, int n_classes, float* d_loss,
                                               float* d_grad_p, int* d_status,
                                               aug_stream_t stream) {
  using namespace augk;
  if (d_descs == nullptr || d_p == nullptr || d_loss == nullptr) return AUG_ERR_INVALID_ARG;
  if (n_vols < 1 || n_vols > kStaticMaxVols) return AUG_ERR_INVALID_ARG;
  if (n_classes < 1 || n_classes > kStaticMaxClasses) return AUG_ERR_UNSUPPORTED;
  cudaStream_t st = (cudaStream_t)stream;
  void* base = nullptr;
  if (scratch_address(&base) != cudaSuccess) return AUG_ERR_CUDA;
  WsHeader* ws = (WsHeader*)base;
  VolConst* tab = (VolConst*)((char*)base + sizeof(WsHeader));
  double* partials = (double*)((char*)tab + kStaticTableBytes);
  float2* coefs = (float2*)((char*)partials + kStaticPartialBytes);
  // The status word keeps the previous call's value: clear it first.
  if (cudaMemsetAsync(ws, 0, 2 * sizeof(int), st) != cudaSuccess) return AUG_ERR_CUDA;

  const int variant = aug_get_variant(2);
  const IouVariant& iv = kIou[variant < 0 ? 0 : variant];
  const int block = iv.nw * 32;
  const int C = n_classes;
  const PassK ks = iv.sums[C - 1];
  int grid = persistent_grid((const void*)ks, block, 0);
  if (grid <= 0) return AUG_ERR_CUDA;
  if (grid > kStaticMaxCtas) grid = kStaticMaxCtas;
  if (launch_prepare(d_descs, n_vols, NEED_IMAGE_NEVER, false, nullptr, nullptr, true, tab, ws,
                     st) != cudaSuccess)
    return AUG_ERR_CUDA;
  // Every CTA writes all of its partial slots (zero where it has no tile), so
  // the previous call's partial sums need no clearing.
  ks<<<grid, block, 0, st>>>(d_descs, n_vols, tab, d_p, nullptr, nullptr, partials);
  if (cudaGetLastError() != cudaSuccess) return AUG_ERR_CUDA;
  kIouFin[C - 1]<<<n_vols, 256, 0, st>>>(partials, grid, n_vols, d_loss,
                                         d_grad_p ? coefs : nullptr);
  if (cudaGetLastError() != cudaSuccess) return AUG_ERR_CUDA;
  if (d_grad_p) {
    const PassK kg = iv.grad[C - 1];
    const int g2 = grid;  // any grid works for the write pass; keep the same
    kg<<<g2, block, 0, st>>>(d_descs, n_vols, tab, d_p, d_grad_p, coefs, nullptr);
    if (cudaGetLastError() != cudaSuccess) return AUG_ERR_CUDA;
  }
  if (d_status != nullptr &&
      cudaMemcpyAsync(d_status, ws, 2 * sizeof(int), cudaMemcpyDeviceToDevice, st) !=
          cudaSuccess)
    return AUG_ERR_CUDA;
  return AUG_OK;
}
