// Overlap losses of Sec. 5.C: launcher, finalize table and the plain-probability
// pass kernels (the kernels themselves are in iou.cuh).
#include <cuda.h>

#include <map>
#include <mutex>
#include <utility>

#include "iou.cuh"

namespace augk {

template const IouPasses& iou_passes<0>(int);

namespace {
using FinK = void (*)(const double*, int, int, int, float*, float2*);
const FinK kIouFin[8] = {k_iou_finalize<1>, k_iou_finalize<2>, k_iou_finalize<3>,
                         k_iou_finalize<4>, k_iou_finalize<5>, k_iou_finalize<6>,
                         k_iou_finalize<7>, k_iou_finalize<8>};
const char* kIouNames[kIouVariants] = {"tile32x8x16", "tile32x4x16", "tile32x8x32",
                                       "tile32x4x32"};

const IouPasses& passes_for(int variant, int xf) {
  switch (xf) {
    case XF_POW: return iou_passes<XF_POW>(variant);
    case XF_LOGITS: return iou_passes<XF_LOGITS>(variant);
    case XF_LOGITS | XF_POW: return iou_passes<XF_LOGITS | XF_POW>(variant);
    default: return iou_passes<0>(variant);
  }
}
}  // namespace

int iou_num_variants() { return kIouVariants; }
const char* iou_variant_name(int v) { return kIouNames[v]; }

cudaError_t launch_iou(int variant, const aug_volume_desc* d, int n, const float* p, int C,
                       int kind, float power, bool logits, float* loss, float* gp,
                       VolConst* tab, double* partials, float2* coefs, WsHeader* ws,
                       cudaStream_t st, int max_grid) {
  const int xf = (power != 1.0f ? XF_POW : 0) | (logits ? XF_LOGITS : 0);
  const IouPasses& iv = passes_for(variant, xf);
  const int block = iv.nw * 32;
  const IouPassK ks = iv.sums[C - 1];
  int grid = persistent_grid((const void*)ks, block, 0);
  if (grid <= 0) return cudaErrorInvalidConfiguration;
  if (max_grid > 0 && grid > max_grid) grid = max_grid;
  cudaError_t e = launch_prepare(d, n, NEED_IMAGE_NEVER, false, nullptr, nullptr, true, tab, ws,
                                 st);
  if (e != cudaSuccess) return e;
  ks<<<grid, block, 0, st>>>(d, n, tab, p, nullptr, nullptr, partials, power);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  kIouFin[C - 1]<<<n, 256, 0, st>>>(partials, grid, n, kind, loss, gp ? coefs : nullptr);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  if (gp) {
    const IouPassK kg = iv.grad[C - 1];
    int g2 = persistent_grid((const void*)kg, block, 0);
    if (g2 <= 0) return cudaErrorInvalidConfiguration;
    if (max_grid > 0 && g2 > max_grid) g2 = max_grid;
    kg<<<g2, block, 0, st>>>(d, n, tab, p, gp, coefs, nullptr, power);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
  }
  return cudaSuccess;
}

// Batch mean of the per-volume losses (Sec. 5.C averages over the batch): one
// warp, each lane a fixed stride of volumes in double, then a fixed-order
// shuffle tree, so the result is reproducible.
__global__ void k_batch_mean(const float* __restrict__ x, int n, float* out) {
  double s = 0.0;
  for (int b = threadIdx.x; b < n; b += 32) s += (double)x[b];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(FULL_MASK, s, o);
  if (threadIdx.x == 0) *out = (float)(s / (double)n);
}

cudaError_t launch_batch_mean(const float* x, int n, float* out, cudaStream_t st) {
  k_batch_mean<<<1, 32, 0, st>>>(x, n, out);
  return cudaGetLastError();
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

// Driver calls for the identity of the current context, fetched through the
// runtime (no link-time dependency on the driver library).
using CtxGetCurrentFn = CUresult (*)(CUcontext*);
using CtxGetIdFn = CUresult (*)(CUcontext, unsigned long long*);

std::mutex g_scratch_mu;
// (device, context id) -> device address of g_iou_scratch in that context.
std::map<std::pair<int, unsigned long long>, void*> g_scratch_ptr;

// Identity of the current context: unique within the process, so a context
// created after cudaDeviceReset (whose module copy of the array may sit at
// another address) never matches an address looked up in an earlier one.
cudaError_t current_context_id(unsigned long long* id) {
  static std::once_flag once;
  static CtxGetCurrentFn get_current = nullptr;
  static CtxGetIdFn get_id = nullptr;
  std::call_once(once, [] {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &p, 12000, cudaEnableDefault, &q) ==
            cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      get_current = (CtxGetCurrentFn)p;
    if (cudaGetDriverEntryPointByVersion("cuCtxGetId", &p, 12000, cudaEnableDefault, &q) ==
            cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      get_id = (CtxGetIdFn)p;
  });
  if (get_current == nullptr || get_id == nullptr) return cudaErrorNotSupported;
  CUcontext ctx = nullptr;
  if (get_current(&ctx) != CUDA_SUCCESS) return cudaErrorDeviceUninitialized;
  if (ctx == nullptr) {
    // No runtime call has made the device's context current on this thread
    // yet: cudaFree(NULL) does (and is otherwise a no-op).
    const cudaError_t e = cudaFree(nullptr);
    if (e != cudaSuccess) return e;
    if (get_current(&ctx) != CUDA_SUCCESS || ctx == nullptr) return cudaErrorDeviceUninitialized;
  }
  return get_id(ctx, id) == CUDA_SUCCESS ? cudaSuccess : cudaErrorDeviceUninitialized;
}

// Device address of the scratch array in the current context.  The host-side
// symbol is only a stand-in, never a device pointer, so the address is looked
// up with cudaGetSymbolAddress, once per device and context.
cudaError_t scratch_address(void** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  unsigned long long ctx = 0;
  if ((e = current_context_id(&ctx)) != cudaSuccess) return e;
  std::lock_guard<std::mutex> lk(g_scratch_mu);
  const auto key = std::make_pair(dev, ctx);
  auto it = g_scratch_ptr.find(key);
  if (it != g_scratch_ptr.end()) {
    *out = it->second;
    return cudaSuccess;
  }
  void* p = nullptr;
  e = cudaGetSymbolAddress(&p, g_iou_scratch);
  if (e != cudaSuccess) return e;
  g_scratch_ptr[key] = p;
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
  // The status words keep the previous call's values: status 0, bad volume -1
  // (the convention of aug_read_device_status when no descriptor is invalid).
  if (cudaMemsetAsync(&ws->status, 0, sizeof(int), st) != cudaSuccess ||
      cudaMemsetAsync(&ws->bad_volume, 0xff, sizeof(int), st) != cudaSuccess)
    return AUG_ERR_CUDA;
  // The same launcher as iou_loss_fwd_bwd, with its grids capped to the
  // partial-sum slots the array holds.  Every CTA of the sums pass writes all
  // of its partial slots (zero where it has no tile), so the previous call's
  // partial sums need no clearing.
  const int variant = aug_get_variant(2);
  if (launch_iou(variant < 0 ? 0 : variant, d_descs, n_vols, d_p, n_classes, AUG_LOSS_IOU, 1.0f,
                 false, d_loss, d_grad_p, tab, partials, coefs, ws, st,
                 kStaticMaxCtas) != cudaSuccess)
    return AUG_ERR_CUDA;
  if (d_status != nullptr &&
      cudaMemcpyAsync(d_status, ws, 2 * sizeof(int), cudaMemcpyDeviceToDevice, st) !=
          cudaSuccess)
    return AUG_ERR_CUDA;
  return AUG_OK;
}
