// Overlap losses of Sec. 5.C: launcher, finalize table and the plain-probability
// pass kernels (the kernels themselves are in iou.cuh).
#include <map>
#include <mutex>

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
                       cudaStream_t st) {
  const int xf = (power != 1.0f ? XF_POW : 0) | (logits ? XF_LOGITS : 0);
  const IouPasses& iv = passes_for(variant, xf);
  const int block = iv.nw * 32;
  const IouPassK ks = iv.sums[C - 1];
  const int grid = persistent_grid((const void*)ks, block, 0);
  if (grid <= 0) return cudaErrorInvalidConfiguration;
  cudaError_t e = launch_prepare(d, n, NEED_IMAGE_NEVER, false, nullptr, nullptr, true, tab, ws,
                                 st);
  if (e != cudaSuccess) return e;
  ks<<<grid, block, 0, st>>>(d, n, tab, p, nullptr, nullptr, partials, power);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  kIouFin[C - 1]<<<n, 256, 0, st>>>(partials, grid, n, kind, loss, gp ? coefs : nullptr);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  if (gp) {
    const IouPassK kg = iv.grad[C - 1];
    const int g2 = persistent_grid((const void*)kg, block, 0);
    if (g2 <= 0) return cudaErrorInvalidConfiguration;
    kg<<<g2, block, 0, st>>>(d, n, tab, p, gp, coefs, nullptr, power);
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
  const IouPasses& iv = iou_passes<0>(variant < 0 ? 0 : variant);
  const int block = iv.nw * 32;
  const int C = n_classes;
  const IouPassK ks = iv.sums[C - 1];
  int grid = persistent_grid((const void*)ks, block, 0);
  if (grid <= 0) return AUG_ERR_CUDA;
  if (grid > kStaticMaxCtas) grid = kStaticMaxCtas;
  if (launch_prepare(d_descs, n_vols, NEED_IMAGE_NEVER, false, nullptr, nullptr, true, tab, ws,
                     st) != cudaSuccess)
    return AUG_ERR_CUDA;
  // Every CTA writes all of its partial slots (zero where it has no tile), so
  // the previous call's partial sums need no clearing.
  ks<<<grid, block, 0, st>>>(d_descs, n_vols, tab, d_p, nullptr, nullptr, partials, 1.0f);
  if (cudaGetLastError() != cudaSuccess) return AUG_ERR_CUDA;
  kIouFin[C - 1]<<<n_vols, 256, 0, st>>>(partials, grid, n_vols, AUG_LOSS_IOU, d_loss,
                                         d_grad_p ? coefs : nullptr);
  if (cudaGetLastError() != cudaSuccess) return AUG_ERR_CUDA;
  if (d_grad_p) {
    const IouPassK kg = iv.grad[C - 1];
    const int g2 = grid;  // any grid works for the write pass; keep the same
    kg<<<g2, block, 0, st>>>(d_descs, n_vols, tab, d_p, d_grad_p, coefs, nullptr, 1.0f);
    if (cudaGetLastError() != cudaSuccess) return AUG_ERR_CUDA;
  }
  if (d_status != nullptr &&
      cudaMemcpyAsync(d_status, ws, 2 * sizeof(int), cudaMemcpyDeviceToDevice, st) !=
          cudaSuccess)
    return AUG_ERR_CUDA;
  return AUG_OK;
}
