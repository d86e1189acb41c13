// C ABI of the augmentation library: argument checks, workspace layout,
// launch-shape selection (persistent grids sized from occupancy and the SM
// count), kernel variants and the autotuner.
#include <math.h>
#include <stddef.h>
#include <stdint.h>

#include <map>
#include <mutex>
#include <tuple>

#include "kernels.h"

namespace augk {
namespace {

std::mutex g_mu;
std::map<int, int> g_sms;                                            // device -> SMs
std::map<std::tuple<int, const void*, int, size_t>, int> g_occ;     // -> CTAs per SM
int g_variant[3] = {-1, -1, -1};
// Defaults: the variants measured fastest on the 64-volume forward batch, the
// 8 x 128^3 adjoint and the 8 x 120x120x160 loss (6 classes).
const int kDefaultVariant[3] = {33, 13, 3};

int current_device() {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return -1;
  return dev;
}

}  // namespace

int device_sm_count() {
  const int dev = current_device();
  if (dev < 0) return 0;
  std::lock_guard<std::mutex> lk(g_mu);
  auto it = g_sms.find(dev);
  if (it != g_sms.end()) return it->second;
  int sms = 0;
  if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return 0;
  g_sms[dev] = sms;
  return sms;
}

int persistent_grid(const void* kernel, int block, size_t smem, int cap) {
  const int sms = device_sm_count();
  if (sms <= 0) return 0;
  const int dev = current_device();
  int per_sm = 0;
  {
    std::lock_guard<std::mutex> lk(g_mu);
    const auto key = std::make_tuple(dev, kernel, block, smem);
    auto it = g_occ.find(key);
    if (it != g_occ.end()) {
      per_sm = it->second;
    } else {
      if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, block, smem) !=
          cudaSuccess)
        per_sm = 0;
      g_occ[key] = per_sm;
    }
  }
  if (per_sm > cap) per_sm = cap;
  return per_sm * sms;
}

__global__ void k_prepare(const aug_volume_desc* __restrict__ descs, int n_vols, int need,
                          int f32_only, const float* const* gout, float* const* gin,
                          int need_label, unsigned forbid_flags, VolConst* __restrict__ tab,
                          WsHeader* ws, unsigned long long tile_next0) {
  const int v = blockIdx.x * blockDim.x + threadIdx.x;
  // First tile index that the dynamic schedule of the next kernel hands out.
  if (v == 0 && ws != nullptr) ws->tile_next = tile_next0;
  if (v >= n_vols) return;
  const aug_volume_desc d = descs[v];
  bool ok = desc_valid(d, needs_image(d, need), f32_only != 0);
  ok &= (d.flags & forbid_flags) == 0u;
  if (gout != nullptr) ok &= gout[v] != nullptr;
  if (gin != nullptr) ok &= gin[v] != nullptr;
  if (need_label) ok &= d.label != nullptr;
  VolConst vc;
  make_volconst(d, ok, vc, need == NEED_IMAGE_ALWAYS);
  tab[v] = vc;
  if (!ok) record_error(ws, AUG_ERR_DESCRIPTOR, v);
}

cudaError_t launch_prepare(const aug_volume_desc* d, int n, int need, bool f32_only,
                           const float* const* gout, float* const* gin, bool need_label,
                           VolConst* tab, WsHeader* ws, cudaStream_t st,
                           unsigned long long tile_next0) {
  // The adjoint (need == NEED_IMAGE_ALWAYS) has no adjoint of the window clamp.
  const unsigned forbid = need == NEED_IMAGE_ALWAYS ? (unsigned)AUG_FLAG_WINDOW : 0u;
  k_prepare<<<(n + 127) / 128, 128, 0, st>>>(d, n, need, f32_only ? 1 : 0, gout, gin,
                                              need_label ? 1 : 0, forbid, tab, ws, tile_next0);
  return cudaGetLastError();
}

__global__ void k_philox(const uint32_t* __restrict__ ctr, long long n, unsigned k0,
                         unsigned k1, uint32_t* __restrict__ out) {
  for (long long m = (long long)blockIdx.x * blockDim.x + threadIdx.x; m < n;
       m += (long long)gridDim.x * blockDim.x) {
    const uint4 c = make_uint4(ctr[4 * m], ctr[4 * m + 1], ctr[4 * m + 2], ctr[4 * m + 3]);
    const uint4 r = philox4x32_10(c, k0, k1);
    out[4 * m] = r.x;
    out[4 * m + 1] = r.y;
    out[4 * m + 2] = r.z;
    out[4 * m + 3] = r.w;
  }
}

cudaError_t launch_philox(const uint32_t* ctr, long long n, unsigned k0, unsigned k1,
                          uint32_t* out, cudaStream_t st) {
  if (n <= 0) return cudaSuccess;
  long long blocks = (n + 255) / 256;
  if (blocks > 4096) blocks = 4096;
  k_philox<<<(unsigned)blocks, 256, 0, st>>>(ctr, n, k0, k1, out);
  return cudaGetLastError();
}

}  // namespace augk

using namespace augk;

namespace {

constexpr int kMaxVols = 65535;
constexpr int kMaxClasses = 8;

size_t align256(size_t v) { return (v + 255) & ~(size_t)255; }

size_t partial_bytes(int n_vols, int n_classes) {
  const size_t per = (size_t)((3 * n_classes > 12) ? 3 * n_classes : 12);
  return align256((size_t)device_sm_count() * kMaxCtasPerSm * (size_t)n_vols * per *
                  sizeof(double));
}

size_t table_bytes(int n_vols) { return align256((size_t)n_vols * sizeof(VolConst)); }

// Workspace: [header 256 B][per-volume constant table][per-CTA partials][class coefficients]
size_t ws_size(int n_vols, int n_classes) {
  if (n_vols < 1 || n_vols > kMaxVols || n_classes < 0 || n_classes > kMaxClasses) return 0;
  if (device_sm_count() <= 0) return 0;
  return sizeof(WsHeader) + table_bytes(n_vols) + partial_bytes(n_vols, n_classes) +
         align256((size_t)n_vols * kMaxClasses * sizeof(float2));
}

VolConst* ws_table(void* ws) { return (VolConst*)((char*)ws + sizeof(WsHeader)); }
double* ws_partials(void* ws, int n_vols) {
  return (double*)((char*)ws + sizeof(WsHeader) + table_bytes(n_vols));
}

aug_status check_ws(void* ws, size_t bytes, int n_vols, int n_classes) {
  if (ws == nullptr || (((uintptr_t)ws) & 255) != 0) return AUG_ERR_WORKSPACE;
  const size_t need = ws_size(n_vols, n_classes);
  if (need == 0 || bytes < need) return AUG_ERR_WORKSPACE;
  return AUG_OK;
}

int variant_of(int op) {
  std::lock_guard<std::mutex> lk(g_mu);
  return g_variant[op] >= 0 ? g_variant[op] : kDefaultVariant[op];
}

int n_variants(int op) {
  switch (op) {
    case 0: return fwd_num_variants();
    case 1: return bwd_num_variants();
    case 2: return iou_num_variants();
    default: return 0;
  }
}

aug_status from_cuda(cudaError_t e) { return e == cudaSuccess ? AUG_OK : AUG_ERR_CUDA; }

void split_seed(uint64_t seed, unsigned* k0, unsigned* k1) {
  *k0 = (unsigned)(seed & 0xffffffffu);
  *k1 = (unsigned)(seed >> 32);
}

// Host mirror of the device descriptor checks (for descriptors in host memory).
bool host_desc_ok(const aug_volume_desc& d) {
  auto dim_ok = [](int v) { return v >= 1 && v <= MAX_DIM; };
  if (!dim_ok(d.in_nx) || !dim_ok(d.in_ny) || !dim_ok(d.in_nz)) return false;
  if (!dim_ok(d.out_nx) || !dim_ok(d.out_ny) || !dim_ok(d.out_nz)) return false;
  if ((long long)d.in_nx * d.in_ny * d.in_nz >= (1LL << 31)) return false;
  if ((long long)d.out_nx * d.out_ny * d.out_nz >= (1LL << 31)) return false;
  if (d.fill_label < 0 || d.fill_label > 255) return false;
  for (int m = 0; m < 12; ++m) {
    const float t = d.affine[m];
    if (!isfinite(t) || fabsf(t) > (((m & 3) < 3) ? 64.0f : 1048576.0f)) return false;
  }
  if (!isfinite(d.photo_a) || !isfinite(d.photo_b) || !isfinite(d.noise_sigma) ||
      d.noise_sigma < 0.0f || !isfinite(d.fill_image))
    return false;
  if (d.flags & ~(unsigned)(AUG_FLAG_WINDOW | AUG_FLAG_OCCLUDE)) return false;
  if (!isfinite(d.occ_z0) || !isfinite(d.occ_dz) || d.occ_dz < 0.0f) return false;
  if (d.out_image != nullptr &&
      (d.image == nullptr || (d.image_dtype != AUG_F32 && d.image_dtype != AUG_I16)))
    return false;
  if (d.out_image != nullptr &&
      ((uintptr_t)d.image & (d.image_dtype == AUG_I16 ? 1u : 3u)) != 0u)
    return false;
  if (d.out_label != nullptr && d.label == nullptr) return false;
  return true;
}

// Checks of a parameter-sampling spec (see aug_sample_params).
bool spec_ok(const aug_param_spec& p) {
  const float* f = (const float*)&p;
  for (size_t i = 0; i < offsetof(aug_param_spec, draw) / sizeof(float); ++i)
    if (!isfinite(f[i])) return false;
  auto range = [](const float* r) { return r[0] <= r[1]; };
  for (int r = 0; r < 3; ++r) {
    if (p.rot_max[r] < 0.0f || p.shift_max[r] < 0.0f) return false;
    if (p.scale_min[r] <= 0.0f || p.scale_min[r] > p.scale_max[r]) return false;
    if (!(p.reflect_prob[r] >= 0.0f && p.reflect_prob[r] <= 1.0f)) return false;
  }
  if (p.shear_max < 0.0f || p.generic_max < 0.0f) return false;
  if (!range(p.photo_a) || !range(p.photo_b) || !range(p.sigma) || p.sigma[0] < 0.0f)
    return false;
  if (!range(p.window_lo) || !range(p.window_hi) || !(p.window_lo[1] < p.window_hi[0]))
    return false;
  if (!(p.occ_max_frac >= 0.0f && p.occ_max_frac <= 1.0f)) return false;
  if (p.draw & ~(unsigned)(AUG_DRAW_AFFINE | AUG_DRAW_PHOTO | AUG_DRAW_WINDOW | AUG_DRAW_OCCLUDE))
    return false;
  return true;
}

aug_status run_fwd(int variant, const aug_volume_desc* d, int n, uint64_t seed, void* ws,
                   cudaStream_t st) {
  unsigned k0, k1;
  split_seed(seed, &k0, &k1);
  return from_cuda(launch_fwd_batched(variant, d, n, k0, k1, ws_table(ws), (WsHeader*)ws, st));
}

aug_status run_bwd(int variant, const aug_volume_desc* d, int n, const float* const* gout,
                   float* const* gin, float* gaff, void* ws, cudaStream_t st) {
  return from_cuda(launch_bwd(variant, d, n, gout, gin, gaff, ws_table(ws), ws_partials(ws, n),
                              (WsHeader*)ws, st));
}

aug_status run_iou(int variant, const aug_volume_desc* d, int n, const float* p, int C,
                   float* loss, float* gp, void* ws, cudaStream_t st, int kind = AUG_LOSS_IOU,
                   float power = 1.0f, bool logits = false) {
  double* partials = ws_partials(ws, n);
  float2* coefs = (float2*)((char*)partials + partial_bytes(n, C));
  return from_cuda(launch_iou(variant, d, n, p, C, kind, power, logits, loss, gp, ws_table(ws),
                              partials, coefs, (WsHeader*)ws, st));
}

}  // namespace

namespace augk {
cudaError_t fwd_on_device(const aug_volume_desc* d, int n, uint64_t seed, void* ws,
                          cudaStream_t st) {
  unsigned k0, k1;
  split_seed(seed, &k0, &k1);
  return launch_fwd_batched(variant_of(0), d, n, k0, k1, ws_table(ws), (WsHeader*)ws, st);
}
size_t fwd_workspace_bytes(int n_vols) { return ws_size(n_vols, 0); }
}  // namespace augk

extern "C" {

size_t aug_workspace_size(int n_vols, int n_classes) { return ws_size(n_vols, n_classes); }

aug_status aug_read_device_status(void* d_workspace, aug_stream_t stream, int clear,
                                  int* bad_volume) {
  if (bad_volume) *bad_volume = -1;
  if (d_workspace == nullptr || (((uintptr_t)d_workspace) & 255) != 0) return AUG_ERR_WORKSPACE;
  cudaStream_t st = (cudaStream_t)stream;
  int h[2] = {0, -1};
  cudaError_t e = cudaMemcpyAsync(h, d_workspace, sizeof(h), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return AUG_ERR_CUDA;
  if (clear && h[0] != 0) {
    const int z[2] = {0, 0};
    e = cudaMemcpyAsync(d_workspace, z, sizeof(z), cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return AUG_ERR_CUDA;
  }
  if (bad_volume) *bad_volume = h[0] ? h[1] : -1;
  return (aug_status)h[0];
}

aug_status aug_warp_fwd_host(const aug_volume_desc* h_descs, int n_vols, uint64_t seed,
                             int chunk_vols, aug_stream_t stream) {
  if (h_descs == nullptr || n_vols < 1 || n_vols > kMaxVols || chunk_vols < 1)
    return AUG_ERR_INVALID_ARG;
  for (int b = 0; b < n_vols; ++b)
    if (!host_desc_ok(h_descs[b])) return AUG_ERR_DESCRIPTOR;
  return fwd_host_pipeline(h_descs, n_vols, seed, std::min(chunk_vols, n_vols),
                           (cudaStream_t)stream);
}

aug_status aug_warp_fwd(const aug_volume_desc* d_descs, int n_vols, uint64_t seed,
                        void* d_workspace, size_t workspace_bytes, aug_stream_t stream) {
  if (n_vols < 1 || n_vols > kMaxVols || d_descs == nullptr) return AUG_ERR_INVALID_ARG;
  const aug_status s = check_ws(d_workspace, workspace_bytes, n_vols, 0);
  if (s != AUG_OK) return s;
  return run_fwd(variant_of(0), d_descs, n_vols, seed, d_workspace, (cudaStream_t)stream);
}

aug_status aug_warp_fwd_volume(const aug_volume_desc* h_desc, uint64_t seed,
                               aug_stream_t stream) {
  if (h_desc == nullptr) return AUG_ERR_INVALID_ARG;
  if (!host_desc_ok(*h_desc)) return AUG_ERR_DESCRIPTOR;
  if (h_desc->out_image == nullptr && h_desc->out_label == nullptr) return AUG_OK;
  unsigned k0, k1;
  split_seed(seed, &k0, &k1);
  return from_cuda(launch_fwd_volume(variant_of(0), *h_desc, k0, k1, (cudaStream_t)stream));
}

aug_status aug_warp_bwd(const aug_volume_desc* d_descs, int n_vols,
                        const float* const* d_grad_out, float* const* d_grad_in,
                        float* d_grad_affine, void* d_workspace, size_t workspace_bytes,
                        aug_stream_t stream) {
  if (n_vols < 1 || n_vols > kMaxVols || d_descs == nullptr || d_grad_out == nullptr)
    return AUG_ERR_INVALID_ARG;
  const aug_status s = check_ws(d_workspace, workspace_bytes, n_vols, 0);
  if (s != AUG_OK) return s;
  return run_bwd(variant_of(1), d_descs, n_vols, d_grad_out, d_grad_in, d_grad_affine,
                 d_workspace, (cudaStream_t)stream);
}

aug_status iou_loss_fwd_bwd(const aug_volume_desc* d_descs, int n_vols, const float* d_p,
                            int n_classes, float* d_loss, float* d_grad_p, void* d_workspace,
                            size_t workspace_bytes, aug_stream_t stream) {
  if (n_vols < 1 || n_vols > kMaxVols || d_descs == nullptr || d_p == nullptr ||
      d_loss == nullptr)
    return AUG_ERR_INVALID_ARG;
  if (n_classes < 1 || n_classes > kMaxClasses) return AUG_ERR_UNSUPPORTED;
  const aug_status s = check_ws(d_workspace, workspace_bytes, n_vols, n_classes);
  if (s != AUG_OK) return s;
  return run_iou(variant_of(2), d_descs, n_vols, d_p, n_classes, d_loss, d_grad_p, d_workspace,
                 (cudaStream_t)stream);
}

aug_status seg_loss_fwd_bwd(const aug_volume_desc* d_descs, int n_vols, const float* d_x,
                            int n_classes, int kind, float power, int logits, float* d_loss,
                            float* d_grad_x, void* d_workspace, size_t workspace_bytes,
                            aug_stream_t stream) {
  if (n_vols < 1 || n_vols > kMaxVols || d_descs == nullptr || d_x == nullptr ||
      d_loss == nullptr)
    return AUG_ERR_INVALID_ARG;
  if (kind != AUG_LOSS_IOU && kind != AUG_LOSS_DICE) return AUG_ERR_INVALID_ARG;
  if (!(power > 0.0f) || !isfinite(power)) return AUG_ERR_INVALID_ARG;
  if (n_classes < 1 || n_classes > kMaxClasses) return AUG_ERR_UNSUPPORTED;
  const aug_status s = check_ws(d_workspace, workspace_bytes, n_vols, n_classes);
  if (s != AUG_OK) return s;
  return run_iou(variant_of(2), d_descs, n_vols, d_x, n_classes, d_loss, d_grad_x, d_workspace,
                 (cudaStream_t)stream, kind, power, logits != 0);
}

aug_status aug_loss_batch_mean(const float* d_loss, int n_vols, float* d_mean,
                               aug_stream_t stream) {
  if (d_loss == nullptr || d_mean == nullptr || n_vols < 1 || n_vols > kMaxVols)
    return AUG_ERR_INVALID_ARG;
  return from_cuda(launch_batch_mean(d_loss, n_vols, d_mean, (cudaStream_t)stream));
}

aug_status aug_sample_params(aug_volume_desc* d_descs, int n_vols, const aug_param_spec* spec,
                             uint64_t seed, uint64_t draw, uint64_t* d_counter,
                             aug_stream_t stream) {
  if (d_descs == nullptr || spec == nullptr || n_vols < 1 || n_vols > kMaxVols)
    return AUG_ERR_INVALID_ARG;
  if (!spec_ok(*spec)) return AUG_ERR_INVALID_ARG;
  unsigned k0, k1;
  split_seed(seed, &k0, &k1);
  return from_cuda(launch_sample_params(d_descs, n_vols, *spec, k0, k1, draw,
                                        (unsigned long long*)d_counter,
                                        (cudaStream_t)stream));
}

aug_status aug_smooth(const aug_smooth_desc* h_descs, int n_vols, aug_stream_t stream) {
  if (h_descs == nullptr || n_vols < 1 || n_vols > kMaxVols) return AUG_ERR_INVALID_ARG;
  for (int b = 0; b < n_vols; ++b) {
    const aug_smooth_desc& d = h_descs[b];
    auto dim_ok = [](int v) { return v >= 1 && v <= MAX_DIM; };
    if (d.image == nullptr || d.out == nullptr) return AUG_ERR_INVALID_ARG;
    if (!dim_ok(d.nx) || !dim_ok(d.ny) || !dim_ok(d.nz)) return AUG_ERR_INVALID_ARG;
    const long long nvox = (long long)d.nx * d.ny * d.nz;
    if (nvox >= (1LL << 31)) return AUG_ERR_INVALID_ARG;
    if (d.image_dtype != AUG_F32 && d.image_dtype != AUG_I16) return AUG_ERR_INVALID_ARG;
    if (!isfinite(d.fill)) return AUG_ERR_INVALID_ARG;
    const char* i0 = (const char*)d.image;
    const char* i1 = i0 + nvox * (d.image_dtype == AUG_I16 ? 2 : 4);
    const char* o0 = (const char*)d.out;
    if (o0 < i1 && i0 < o0 + nvox * 4) return AUG_ERR_INVALID_ARG;
    for (int r = 0; r < 3; ++r) {
      if (!isfinite(d.sigma[r]) || d.sigma[r] < 0.0f) return AUG_ERR_INVALID_ARG;
      if (gauss_radius(d.sigma[r]) > smooth_max_radius()) return AUG_ERR_UNSUPPORTED;
    }
  }
  return from_cuda(launch_smooth(h_descs, n_vols, (cudaStream_t)stream));
}

aug_status aug_test_smooth_wait_timeout(const aug_smooth_desc* h_descs, int n_vols,
                                        aug_stream_t stream) {
  if (h_descs == nullptr || n_vols < 1 || n_vols > 4) return AUG_ERR_INVALID_ARG;
  return from_cuda(launch_smooth(h_descs, n_vols, (cudaStream_t)stream, true));
}

aug_status aug_smooth_status(int* status) {
  if (status == nullptr) return AUG_ERR_INVALID_ARG;
  int* word = nullptr;
  if (smooth_status_word(&word) != cudaSuccess) return AUG_ERR_CUDA;
  if (cudaDeviceSynchronize() != cudaSuccess) return AUG_ERR_CUDA;
  if (cudaMemcpy(status, word, sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess)
    return AUG_ERR_CUDA;
  if (cudaMemset(word, 0, sizeof(int)) != cudaSuccess) return AUG_ERR_CUDA;
  return AUG_OK;
}

float aug_antialias_sigma(float r, float u) {
  const double t = (double)r / (double)u - 1.0;
  return (float)((t > 0.0 ? t : 0.0) / 3.0);
}

aug_status aug_tex_create(const aug_volume_desc* h_descs, int n_vols, void** handle) {
  if (h_descs == nullptr || handle == nullptr || n_vols < 1 || n_vols > kMaxVols)
    return AUG_ERR_INVALID_ARG;
  for (int b = 0; b < n_vols; ++b) {
    if (!host_desc_ok(h_descs[b])) return AUG_ERR_DESCRIPTOR;
    if (h_descs[b].flags != 0) return AUG_ERR_UNSUPPORTED;
    if (h_descs[b].out_image != nullptr && h_descs[b].image_dtype != AUG_F32)
      return AUG_ERR_UNSUPPORTED;
  }
  return tex_create(h_descs, n_vols, handle);
}

aug_status aug_tex_warp_fwd(void* handle, uint64_t seed, aug_stream_t stream) {
  if (handle == nullptr) return AUG_ERR_INVALID_ARG;
  return tex_warp_fwd(handle, seed, (cudaStream_t)stream);
}

aug_status aug_tex_destroy(void* handle) { return tex_destroy(handle); }

int aug_num_variants(int op) { return n_variants(op); }

const char* aug_variant_name(int op, int variant) {
  if (variant < 0 || variant >= n_variants(op)) return "invalid";
  switch (op) {
    case 0: return fwd_variant_name(variant);
    case 1: return bwd_variant_name(variant);
    default: return iou_variant_name(variant);
  }
}

aug_status aug_set_variant(int op, int variant) {
  if (op < 0 || op > 2 || variant < -1 || variant >= n_variants(op)) return AUG_ERR_INVALID_ARG;
  std::lock_guard<std::mutex> lk(g_mu);
  g_variant[op] = variant;
  return AUG_OK;
}

int aug_get_variant(int op) {
  if (op < 0 || op > 2) return -1;
  return variant_of(op);
}

aug_status aug_autotune(int op, const aug_volume_desc* d_descs, int n_vols, uint64_t seed,
                        const float* const* d_grad_out, float* const* d_grad_in,
                        float* d_grad_affine, const float* d_p, int n_classes, float* d_loss,
                        float* d_grad_p, void* d_workspace, size_t workspace_bytes,
                        aug_stream_t stream, int reps, int* best, float* best_ms) {
  if (op < 0 || op > 2 || reps < 1 || n_vols < 1 || n_vols > kMaxVols || d_descs == nullptr)
    return AUG_ERR_INVALID_ARG;
  if (op == 1 && d_grad_out == nullptr) return AUG_ERR_INVALID_ARG;
  if (op == 2 && (d_p == nullptr || d_loss == nullptr)) return AUG_ERR_INVALID_ARG;
  if (op == 2 && (n_classes < 1 || n_classes > kMaxClasses)) return AUG_ERR_UNSUPPORTED;
  const aug_status s = check_ws(d_workspace, workspace_bytes, n_vols, op == 2 ? n_classes : 0);
  if (s != AUG_OK) return s;
  cudaStream_t st = (cudaStream_t)stream;
  cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
  if (cudaStreamIsCapturing(st, &cap) != cudaSuccess || cap != cudaStreamCaptureStatusNone)
    return AUG_ERR_INVALID_ARG;
  auto run = [&](int v) -> aug_status {
    switch (op) {
      case 0: return run_fwd(v, d_descs, n_vols, seed, d_workspace, st);
      case 1:
        return run_bwd(v, d_descs, n_vols, d_grad_out, d_grad_in, d_grad_affine, d_workspace,
                       st);
      default:
        return run_iou(v, d_descs, n_vols, d_p, n_classes, d_loss, d_grad_p, d_workspace, st);
    }
  };
  cudaEvent_t e0, e1;
  if (cudaEventCreate(&e0) != cudaSuccess) return AUG_ERR_CUDA;
  if (cudaEventCreate(&e1) != cudaSuccess) {
    cudaEventDestroy(e0);
    return AUG_ERR_CUDA;
  }
  int best_v = -1;
  float best_t = 0.0f;
  aug_status result = AUG_OK;
  for (int v = 0; v < n_variants(op) && result == AUG_OK; ++v) {
    if ((result = run(v)) != AUG_OK) break;  // warm-up
    if (cudaEventRecord(e0, st) != cudaSuccess) {
      result = AUG_ERR_CUDA;
      break;
    }
    for (int r = 0; r < reps && result == AUG_OK; ++r) result = run(v);
    if (result != AUG_OK) break;
    if (cudaEventRecord(e1, st) != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess) {
      result = AUG_ERR_CUDA;
      break;
    }
    float ms = 0.0f;
    cudaEventElapsedTime(&ms, e0, e1);
    ms /= (float)reps;
    if (best_v < 0 || ms < best_t) {
      best_v = v;
      best_t = ms;
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (result != AUG_OK) return result;
  aug_set_variant(op, best_v);
  if (best) *best = best_v;
  if (best_ms) *best_ms = best_t;
  return AUG_OK;
}

aug_status aug_philox4x32_10(const uint32_t* d_ctr, int64_t n, uint64_t seed, uint32_t* d_out,
                             aug_stream_t stream) {
  if (n < 0 || (n > 0 && (d_ctr == nullptr || d_out == nullptr))) return AUG_ERR_INVALID_ARG;
  unsigned k0, k1;
  split_seed(seed, &k0, &k1);
  return from_cuda(launch_philox(d_ctr, (long long)n, k0, k1, d_out, (cudaStream_t)stream));
}

const char* aug_status_string(int status) {
  switch (status) {
    case AUG_OK: return "ok";
    case AUG_ERR_INVALID_ARG: return "invalid argument";
    case AUG_ERR_CUDA: return "CUDA runtime error";
    case AUG_ERR_WORKSPACE: return "workspace missing, misaligned or too small";
    case AUG_ERR_DESCRIPTOR: return "invalid volume descriptor";
    case AUG_ERR_UNSUPPORTED: return "unsupported request";
    case AUG_ERR_TIMEOUT: return "a bounded device wait for a copy ran out";
    default: return "unknown status";
  }
}

int aug_version(void) { return 10000; }

}  // extern "C"
