// Internal host-side interface between the C ABI (api.cu) and the kernel
// translation units.  Not installed; not part of the public ABI.
#pragma once

#include <cuda_runtime.h>

#include "augwarp.h"
#include "common.cuh"
#include "sched.cuh"

namespace augk {

// Grid of a persistent launch: (resident CTAs per SM, capped at cap) * SM
// count of the current device.  Cached per kernel.  The default cap,
// kMaxCtasPerSm, also sizes the workspace's per-CTA partial sums; kernels
// that keep none may pass a higher one (at most 32, the SM's CTA limit).
int persistent_grid(const void* kernel, int block, size_t smem, int cap = kMaxCtasPerSm);
int device_sm_count();

int fwd_num_variants();
const char* fwd_variant_name(int v);
// Prologue of each batched call (k_prepare): per-volume constant table.
cudaError_t launch_prepare(const aug_volume_desc* d, int n, int need, bool f32_only,
                           const float* const* gout, float* const* gin, bool need_label,
                           VolConst* tab, WsHeader* ws, cudaStream_t st,
                           unsigned long long tile_next0 = 0ull);

cudaError_t launch_fwd_batched(int variant, const aug_volume_desc* d, int n, unsigned k0,
                               unsigned k1, VolConst* tab, WsHeader* ws, cudaStream_t st);
cudaError_t launch_fwd_volume(int variant, const aug_volume_desc& h, unsigned k0, unsigned k1,
                              cudaStream_t st);
// Shared-memory brick forward (fwd_brick.cu): its own variant numbering.
int fwd_brick_num_variants();
const char* fwd_brick_variant_name(int v);
cudaError_t launch_fwd_brick(int variant, const aug_volume_desc* d, int n, unsigned k0,
                             unsigned k1, VolConst* tab, WsHeader* ws, cudaStream_t st);

int bwd_num_variants();
const char* bwd_variant_name(int v);
cudaError_t launch_bwd(int variant, const aug_volume_desc* d, int n, const float* const* gout,
                       float* const* gin, float* gaff, VolConst* tab, double* partials,
                       WsHeader* ws, cudaStream_t st);

// Brick adjoint (bwd_brick.cu): its own variant numbering; the kernel only
// (launch_bwd issues the prologue, the zeroing and the finalize).
int bwd_brick_num_variants();
const char* bwd_brick_variant_name(int v);
cudaError_t launch_bwd_brick(int variant, const aug_volume_desc* d, int n,
                             const float* const* gout, float* const* gin, bool want_gt,
                             VolConst* tab, double* partials, WsHeader* ws, cudaStream_t st,
                             int* grid_out);

// Input-driven gather adjoint for grad_in (bwd_gather.cu); the affine gradient
// then comes from the output-driven pass of a bwd.cu variant.
int bwd_gather_num_variants();
const char* bwd_gather_variant_name(int v);
cudaError_t launch_bwd_gather(int variant, const aug_volume_desc* d, int n,
                              const float* const* gout, float* const* gin, VolConst* tab,
                              WsHeader* ws, cudaStream_t st);

int iou_num_variants();
const char* iou_variant_name(int v);
// Overlap loss `kind` (aug_loss_kind) on q = (logits ? softmax(p) : p)^power.
// max_grid > 0 caps the CTAs of both passes (partial-sum slots of a fixed
// scratch array).
cudaError_t launch_iou(int variant, const aug_volume_desc* d, int n, const float* p, int C,
                       int kind, float power, bool logits, float* loss, float* gp,
                       VolConst* tab, double* partials, float2* coefs, WsHeader* ws,
                       cudaStream_t st, int max_grid = 0);

// out[0] = mean of x[0..n-1] (fixed summation order).
cudaError_t launch_batch_mean(const float* x, int n, float* out, cudaStream_t st);

// Per-volume random parameters into the descriptors (one CTA).
cudaError_t launch_sample_params(aug_volume_desc* d, int n, const aug_param_spec& sp,
                                 unsigned k0, unsigned k1, unsigned long long draw,
                                 unsigned long long* counter, cudaStream_t st);

// Anti-aliasing Gaussian (host descriptors; grouped launches).
int gauss_radius(float sigma);
int smooth_max_radius();
// no_copies: the test of the bounded waits (no tile copy is issued).
cudaError_t launch_smooth(const aug_smooth_desc* h, int n, cudaStream_t st,
                          bool no_copies = false);
cudaError_t smooth_status_word(int** p);

// Batched forward on device descriptors with the default variant (the C ABI's
// aug_warp_fwd without its argument checks), its workspace size, and the
// pipelined forward from host buffers built on it.
cudaError_t fwd_on_device(const aug_volume_desc* d, int n, uint64_t seed, void* ws,
                          cudaStream_t st);
size_t fwd_workspace_bytes(int n_vols);
aug_status fwd_host_pipeline(const aug_volume_desc* h, int n, uint64_t seed, int chunk,
                             cudaStream_t stream);

// Hardware-texture alternative of the forward (measured comparison).
aug_status tex_create(const aug_volume_desc* h, int n, void** handle);
aug_status tex_warp_fwd(void* handle, uint64_t seed, cudaStream_t st);
aug_status tex_destroy(void* handle);

cudaError_t launch_philox(const uint32_t* ctr, long long n, unsigned k0, unsigned k1,
                          uint32_t* out, cudaStream_t st);

}  // namespace augk
