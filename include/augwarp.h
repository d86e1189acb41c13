/*
 * augwarp.h -- C ABI of the B300 (sm_103a) CT data-augmentation library.
 *
 * The library implements the GPU augmentation path of Rister et al., "CT organ
 * segmentation using GPU data augmentation, unsupervised labels and IOU loss"
 * (arXiv 1811.11226):
 *
 *   - Sec. 4: each output voxel o = (i, j, k) of a crop is mapped through an
 *     affine coordinate map s = A o + b, the image is sampled trilinearly at s
 *     and the label volume at the nearest voxel, a constant fill is used
 *     outside the input, and additive Gaussian noise is applied;
 *   - the intensity affine y = a v + beta precedes the noise;
 *   - the adjoint of the image warp with respect to the input volume and the
 *     12 affine parameters (the paper has no backward pass; it is what makes
 *     the warp trainable);
 *   - Sec. 5.C: the soft IOU loss 1 - |py|_1 / (|p|_1 + |y|_1 - |py|_1),
 *     averaged over classes and over the batch, fused with the nearest-label
 *     warp so the warped labels never reach memory.
 *
 * Conventions (all entry points):
 *   - Volumes are dense, C-contiguous [nz][ny][nx] arrays, x fastest.
 *   - The affine is float32 row-major 3x4 T in voxel-index units:
 *       s_r = T[r][0] i + T[r][1] j + T[r][2] k + T[r][3],  r = x, y, z.
 *     Voxel centres are at integer coordinates.
 *   - Image sample: trilinear over the cell floor(s); every tap outside the
 *     input reads fill_image.  Label sample: input label at floor(s + 1/2),
 *     fill_label outside.
 *   - Output value: y = photo_a * v + photo_b + noise_sigma * n, with n a
 *     standard normal from Philox4x32-10 (key = seed, counter = (quad index,
 *     noise_id)) and Box-Muller; quads are four z-consecutive output voxels
 *     (k = 4m..4m+3) -- see aug_warp_fwd.  Optional per volume (aug_flags):
 *     occlusion of a z-slab of the output and a window/level clamp.
 *   - All pointers are DEVICE pointers unless stated otherwise.  The caller
 *     owns every buffer.  Two entry points allocate device memory, as their
 *     declarations state: aug_warp_fwd_host (staging slots from the
 *     stream-ordered pool, returned at the end of the call) and
 *     aug_tex_create (the CUDA arrays its handle owns); no other entry point
 *     allocates.  Every entry point only enqueues work on `stream` and returns
 *     without synchronising, except aug_read_device_status and aug_autotune.
 *   - Argument errors found on the host are returned synchronously; errors
 *     found in device descriptors are written to the workspace status word
 *     (read it with aug_read_device_status); the offending volume is skipped.
 *   - Limits: every dimension in [1, 8192]; every volume below 2^31 voxels;
 *     |T[r][c]| <= 64 for c < 3 and |T[r][3]| <= 2^20; 1 <= n_vols <= 65535.
 */
#ifndef AUGWARP_H
#define AUGWARP_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Every declaration below is exported from the shared library (the library
 * is built with hidden visibility for everything else). */
#if defined(__GNUC__)
#pragma GCC visibility push(default)
#endif

/* Binary-compatible with cudaStream_t; NULL selects the legacy default stream. */
typedef struct CUstream_st* aug_stream_t;

typedef enum {
  AUG_OK = 0,
  AUG_ERR_INVALID_ARG = 1, /* a host argument is out of range / NULL           */
  AUG_ERR_CUDA = 2,        /* a CUDA runtime call or kernel launch failed       */
  AUG_ERR_WORKSPACE = 3,   /* workspace NULL, misaligned or too small           */
  AUG_ERR_DESCRIPTOR = 4,  /* (device status) a volume descriptor is invalid    */
  AUG_ERR_UNSUPPORTED = 5, /* valid request outside what this library implements */
  AUG_ERR_TIMEOUT = 6      /* (device status) a bounded wait for a copy ran out   */
} aug_status;

typedef enum { AUG_F32 = 0, AUG_I16 = 1 } aug_dtype;

/* Descriptor flags (Sec. 4, the photometric steps after the warp). */
typedef enum {
  /* Window/level: clamp the output to [0, 1] after the noise.  With
   * photo_a = 1/(hi - lo), photo_b = -lo/(hi - lo) and noise_sigma scaled by
   * photo_a this is clamp((I + n - lo)/(hi - lo), 0, 1). */
  AUG_FLAG_WINDOW = 1,
  /* Random occlusion: output voxels whose z index k satisfies
   * occ_z0 <= k <= occ_z0 + occ_dz are 0, and nothing else is computed for
   * them (no fetch, no noise, no window).  Labels are not occluded. */
  AUG_FLAG_OCCLUDE = 2
} aug_flags;

/*
 * One volume of a batch.  Arrays of these live in DEVICE memory, so a CUDA
 * graph captured once can be replayed with new parameters written into the
 * same descriptor buffer.  144 bytes, 16-byte aligned.
 */
typedef struct __attribute__((aligned(16))) {
  const void* image;       /* [in_nz][in_ny][in_nx] of image_dtype                */
  const uint8_t* label;    /* same shape, or NULL (no label warp)                 */
  float* out_image;        /* [out_nz][out_ny][out_nx] float32, or NULL           */
  uint8_t* out_label;      /* same shape as out_image; NULL, or label != NULL     */
  int32_t in_nx, in_ny, in_nz;
  int32_t image_dtype;     /* aug_dtype                                           */
  int32_t out_nx, out_ny, out_nz;
  int32_t fill_label;      /* 0..255                                              */
  float affine[12];        /* T, row-major 3x4, output index -> input coordinate  */
  float photo_a, photo_b;  /* intensity affine y = a v + b                        */
  float noise_sigma;       /* standard deviation of the additive noise (>= 0)    */
  float fill_image;        /* value of every input tap outside the volume         */
  uint32_t noise_id;       /* third Philox counter word (usually the batch index) */
  uint32_t flags;          /* aug_flags bits (0: plain warp + affine + noise)     */
  float occ_z0, occ_dz;    /* occlusion slab (AUG_FLAG_OCCLUDE), occ_dz >= 0       */
} aug_volume_desc;

/* ---- workspace ----------------------------------------------------------
 * Device scratch every batched entry point needs: a status word and
 * per-block partial sums.  Allocate at least aug_workspace_size() bytes,
 * 256-byte aligned, zero-filled once before first use (the status word then
 * stays zero until a device-side error is recorded).  One workspace may be
 * reused by consecutive calls on one stream; concurrent calls need separate
 * workspaces.  Returns 0 if the arguments are out of range or no CUDA device
 * is present.  Host function; queries the current device once. */
size_t aug_workspace_size(int n_vols, int n_classes);

/* Reads (and, if clear != 0, resets) the device status word of a workspace.
 * Synchronises `stream`.  Returns the first device-side error recorded since
 * the last clear (AUG_OK if none); *bad_volume (may be NULL) receives the
 * index of the offending volume or -1. */
aug_status aug_read_device_status(void* d_workspace, aug_stream_t stream, int clear,
                                  int* bad_volume);

/* ---- forward warp (Sec. 4) -------------------------------------------------
 * Augments n_vols volumes of arbitrary, unequal sizes in ONE persistent launch.
 * For each descriptor: out_image (if not NULL) receives the trilinear image
 * sample passed through the intensity affine and the additive noise, and
 * out_label (if not NULL) the nearest-neighbour label.  Output voxels whose
 * every tap lies outside the input read the fill values.
 *
 * Noise: for output voxel (i, j, k), quad index Q = ((k >> 2) * out_ny + j)
 * * out_nx + i and lane l = k & 3.  Philox4x32-10 with key (lo32(seed),
 * hi32(seed)) and counter (lo32(Q), hi32(Q), noise_id, 0) yields r0..r3;
 * lanes 0-1 use (ra, rb) = (r0, r1), lanes 2-3 (r2, r3);
 * u1 = ((ra >> 8) + 1) 2^-24, u2 = (rb >> 8) 2^-24, R = sqrt(-2 ln u1);
 * n = R cos(2 pi u2) for even l, R sin(2 pi u2) for odd l.  noise_sigma == 0
 * adds exactly nothing.
 *
 * d_descs: device array of n_vols descriptors.  d_workspace: see above.
 * Errors: AUG_ERR_INVALID_ARG (n_vols out of range, d_descs NULL),
 * AUG_ERR_WORKSPACE, AUG_ERR_CUDA (launch failure). */
aug_status aug_warp_fwd(const aug_volume_desc* d_descs, int n_vols, uint64_t seed,
                        void* d_workspace, size_t workspace_bytes, aug_stream_t stream);

/* The same computation for ONE volume in its own non-persistent launch (one
 * CTA per output tile), with the descriptor passed by value from HOST memory:
 * the plain one-volume-per-launch form, kept as the comparison point for the
 * batched launch.  h_desc: host pointer.  Descriptor errors are returned
 * synchronously as AUG_ERR_DESCRIPTOR. */
aug_status aug_warp_fwd_volume(const aug_volume_desc* h_desc, uint64_t seed,
                               aug_stream_t stream);

/* ---- device-side random parameters (Sec. 4) ----------------------------------
 * Ranges of the per-volume random augmentation (all float32, host struct passed
 * by value).  Angles in radians, lengths in voxels of the input grid.
 *
 * For volume v the sampler draws 32 uniforms u_0..u_31 in [0, 1) from
 * Philox4x32-10 with key (lo32 seed, hi32 seed) and counters
 * (j, noise_id_v, lo32 n, 0x80000000 | hi32 n), j = 0..7, as u = (w >> 8) 2^-24
 * of the words w in order; n is the draw index (below).  The set top bit keeps
 * these counters apart from the noise's (last word 0).  With x(u) = 2u - 1:
 *   angles    g_r = rot_max_r x(u_r)                       r = 0, 1, 2 (x, y, z)
 *   scales    s_r = scale_min_r + (scale_max_r - scale_min_r) u_{3+r}
 *   reflect   refl_r = -1 if u_{6+r} < reflect_prob_r else +1
 *   shear     Sh = I with Sh_01, Sh_02, Sh_12 = shear_max x(u_9), x(u_10), x(u_11)
 *   generic   G_ij = generic_max x(u_{12+3i+j})
 *   shift     d_r = shift_max_r x(u_{21+r})
 *   A = (I + G) Rz(g_z) Ry(g_y) Rx(g_x) Sh diag(refl s) diag(extra_scale),
 *   b = c_in + d - A c_out, c = (N - 1)/2 per axis  (Sec. 4: A c + b = c + d),
 * computed in double and rounded to float32 into affine[].
 *   intensity photo_a, photo_b, sigma from their [min, max] by u_24, u_25, u_26;
 *   window    lo, hi from window_lo, window_hi by u_27, u_28; photo_a =
 *             1/(hi - lo), photo_b = -lo/(hi - lo), noise_sigma = (sigma draw)
 *             / (hi - lo), and flags |= AUG_FLAG_WINDOW;
 *   occlusion dmax = occ_max_frac out_nz, occ_dz = dmax u_29,
 *             occ_z0 = -dmax + (out_nz - 1 + dmax) u_30, flags |= AUG_FLAG_OCCLUDE.
 * Rotation about x by g: rows (y, z) = (cos g, -sin g; sin g, cos g); about y:
 * rows (x, z); about z: rows (x, y). */
typedef struct {
  float rot_max[3];
  float scale_min[3], scale_max[3];
  float reflect_prob[3];
  float shear_max;
  float generic_max;
  float extra_scale[3];
  float shift_max[3];
  float photo_a[2], photo_b[2], sigma[2]; /* [min, max] */
  float window_lo[2], window_hi[2];       /* [min, max]; window_lo[1] < window_hi[0] */
  float occ_max_frac;                     /* in [0, 1] */
  uint32_t draw;                          /* aug_draw bits */
} aug_param_spec;

typedef enum {
  AUG_DRAW_AFFINE = 1,  /* affine[]                                              */
  AUG_DRAW_PHOTO = 2,   /* photo_a, photo_b, noise_sigma (ignored with WINDOW)    */
  AUG_DRAW_WINDOW = 4,  /* photo_a, photo_b, noise_sigma as a window; flags        */
  AUG_DRAW_OCCLUDE = 8  /* occ_z0, occ_dz; flags                                   */
} aug_draw;

/* Draws the parameters of every volume into its descriptor (device memory):
 * the fields of the groups in spec->draw are overwritten, the others kept.
 * Reads in/out dims and noise_id.  The draw index is n = draw + *d_counter
 * when d_counter (device uint64) is non-NULL, which the call then increments
 * on the device, so a captured graph draws new parameters on every replay;
 * with d_counter NULL, n = draw.  One small kernel on `stream`.
 * AUG_ERR_INVALID_ARG: NULL descriptors, n_vols out of 1..65535, or a spec
 * with a non-finite value, a negative range width or maximum, a probability
 * or occ_max_frac outside [0, 1], scale_min <= 0, window_lo[1] >= window_hi[0],
 * or unknown draw bits. */
aug_status aug_sample_params(aug_volume_desc* d_descs, int n_vols, const aug_param_spec* spec,
                             uint64_t seed, uint64_t draw, uint64_t* d_counter,
                             aug_stream_t stream);

/* ---- anti-aliasing Gaussian of the 3 mm resampling (Sec. 5.A) ----------------
 * out = the input smoothed by g(x) proportional to exp(-sum_k x_k^2 / sigma_k^2)
 * on the support |x_k| <= ceil(3 sigma_k) (a single tap where sigma_k = 0),
 * normalised to sum 1 per axis, with the input extended by `fill` outside its
 * box (the same extension the warp uses).  Weights are computed in double and
 * rounded to float32; the sums are float32.  A resampling to resolution r mm
 * from spacing u_k mm uses sigma_k = aug_antialias_sigma(r, u_k), then the
 * warp (aug_warp_fwd) with the downscaling affine reads `out`.
 *
 * h_descs: HOST array of n_vols descriptors (read during the call only).
 * image: [nz][ny][nx] of image_dtype (device); out: [nz][ny][nx] float32
 * (device, must not overlap image).  One launch per group of at most 32
 * volumes with the same input type and radius, on `stream`.
 * AUG_ERR_INVALID_ARG: NULL pointers, dims outside 1..8192 or >= 2^31
 * voxels, unknown dtype, non-finite fill or sigma, sigma < 0.
 * AUG_ERR_UNSUPPORTED: ceil(3 sigma_k) > 8 (sigma_k > 2.67). */
typedef struct {
  const void* image;
  float* out;
  int32_t nx, ny, nz;
  int32_t image_dtype; /* aug_dtype */
  float sigma[3];      /* x, y, z, in input voxels */
  float fill;
} aug_smooth_desc;

aug_status aug_smooth(const aug_smooth_desc* h_descs, int n_vols, aug_stream_t stream);

/* Device status of the smoothing calls since the last read: *status = 0;
 * 1 if a block gave up waiting for its input tile, 2 if a block found its
 * staging buffer misaligned (its outputs are then incomplete).  Synchronises
 * the device, then clears the word. */
aug_status aug_smooth_status(int* status);

/* sigma = max(r / u - 1, 0) / 3: the smoothing factor of Sec. 5.A for target
 * resolution r and spacing u (same unit), in input voxels.  Host function. */
float aug_antialias_sigma(float r, float u);

/* Test of the smoothing kernel's bounded waits (no counterpart in the paper):
 * runs aug_smooth on at most 4 descriptors without issuing any tile copy, so
 * every block's wait for its first tile runs out (after about a second), is
 * recorded as status 1 (read with aug_smooth_status) and the block returns.
 * Outputs are left incomplete.  Volumes whose rows are not a multiple of 16
 * bytes use per-thread loads and do not wait. */
aug_status aug_test_smooth_wait_timeout(const aug_smooth_desc* h_descs, int n_vols,
                                        aug_stream_t stream);

/* ---- forward from host buffers, pipelined (Sec. 4, the host <-> device FIFO) --
 * Same result as aug_warp_fwd on the same descriptors, for volumes that live
 * in HOST memory: h_descs is a HOST array whose image, label, out_image and
 * out_label point to host buffers (page-locked for the copies to overlap;
 * pageable memory works but serialises).  The batch is processed in chunks of
 * chunk_vols volumes on three internal streams and device slots: the input
 * copy of one chunk, the kernel of the next and the output copy of the
 * previous run at the same time.  The call is ordered after prior work on
 * `stream`, and `stream` waits for all of it; the output buffers are valid
 * once `stream` reaches that point.  Device memory: three slots sized for the
 * largest chunk, from the stream-ordered pool (cudaMallocAsync), returned at
 * the end of the call.  Calls on one device are serialised by the library.
 * Errors: NULL h_descs, n_vols outside 1..65535 or chunk_vols < 1:
 * AUG_ERR_INVALID_ARG; a descriptor failing the checks of
 * aug_warp_fwd_volume: AUG_ERR_DESCRIPTOR (nothing is launched). */
aug_status aug_warp_fwd_host(const aug_volume_desc* h_descs, int n_vols, uint64_t seed,
                             int chunk_vols, aug_stream_t stream);

/* ---- hardware-texture alternative (a measured comparison) -----------------------
 * The paper's own sampling (Sec. 4): trilinear interpolation by the texture
 * unit (tex3D, linear filtering, fixed-point weights) on float32 coordinates.
 * It is not a parity path: its interpolation error is several HU at sharp
 * edges, far above the exact path's 2e-3 HU.  The intensity affine and the noise
 * are the exact path's (same Philox stream); labels are the nearest voxel.
 *
 * aug_tex_create: h_descs is a HOST array of n_vols descriptors (device
 * buffers, float32 images); copies each image into a newly allocated 3-D CUDA
 * array read through a texture whose border colour is fill_image; *handle
 * receives an opaque handle owning them.  Synchronous.
 * aug_tex_warp_fwd: writes each descriptor's out_image / out_label, one launch
 * per volume on `stream`.  aug_tex_destroy frees the handle (after the
 * launches that use it have finished).
 * Errors: NULL arguments or n_vols outside 1..65535: AUG_ERR_INVALID_ARG; a
 * descriptor failing the checks of aug_warp_fwd_volume: AUG_ERR_DESCRIPTOR;
 * an int16 image with an image output, or flags != 0: AUG_ERR_UNSUPPORTED. */
aug_status aug_tex_create(const aug_volume_desc* h_descs, int n_vols, void** handle);
aug_status aug_tex_warp_fwd(void* handle, uint64_t seed, aug_stream_t stream);
aug_status aug_tex_destroy(void* handle);

/* ---- adjoint of the image warp ---------------------------------------------
 * For upstream gradients g_b (shape of out_image of volume b, float32):
 *   grad_in_b[n]    = sum_o photo_a g_b(o) w_{n}(o)       over in-volume taps,
 *   grad_affine_b[r][c] = sum_o photo_a g_b(o) dv/ds_r(o) obar_c(o),
 * with w the trilinear weights, obar = (i, j, k, 1) and dv/ds_r the derivative
 * of the trilinear sample along axis r (fill taps included; the cell is the
 * one chosen by floor(s), i.e. right derivatives at integer coordinates).
 * The noise and photo_b do not depend on the input or on T.
 *
 * d_grad_out: device array of n_vols device pointers (output shape).
 * d_grad_in:  device array of n_vols device pointers (input shape, float32
 *             images only), or NULL to skip; overwritten (the library zeroes
 *             them first).  Accumulated with atomics: run-to-run rounding
 *             order may differ.
 * d_grad_affine: [n_vols][12] float32, or NULL to skip; overwritten;
 *             reduced in a fixed order (bitwise reproducible).
 * Occluded output voxels (AUG_FLAG_OCCLUDE) pass no gradient.  A descriptor
 * with AUG_FLAG_WINDOW (the clamp has no useful adjoint here) and an int16
 * volume with d_grad_in != NULL are descriptor errors.  Other errors as
 * aug_warp_fwd. */
aug_status aug_warp_bwd(const aug_volume_desc* d_descs, int n_vols,
                        const float* const* d_grad_out, float* const* d_grad_in,
                        float* d_grad_affine, void* d_workspace, size_t workspace_bytes,
                        aug_stream_t stream);

/* ---- fused label warp + soft IOU loss (Sec. 5.C) ----------------------------
 * For each volume b and class c in 0..n_classes-1 (labels outside 0..C-1 belong
 * to no class), with y_k = [nearest warped label at output voxel k == c]:
 *   I = sum_k p_k y_k, P = sum_k p_k, Y = sum_k y_k, U = P + Y - I,
 *   L_bc = 1 - I / U  (0 where U == 0),
 *   loss[b] = mean_c L_bc,
 *   grad_p[b][c][k] = d(mean_b loss[b]) / d p = (1 / (B C)) (y_k ? -1/U : I/U^2)
 * (0 where U == 0).  The warped labels are recomputed in registers by both
 * passes and never written to memory.
 *
 * d_p: float32, volumes packed consecutively, volume b as [C][out_nz][out_ny]
 * [out_nx] at offset C * sum_{b'<b} nvox_{b'}.  d_grad_p: same layout, or NULL
 * for the loss only.  d_loss: [n_vols] float32.  Uses each descriptor's label,
 * affine, out dims and fill_label; the image fields are ignored.
 * 1 <= n_classes <= 8, else AUG_ERR_UNSUPPORTED. */
aug_status iou_loss_fwd_bwd(const aug_volume_desc* d_descs, int n_vols, const float* d_p,
                            int n_classes, float* d_loss, float* d_grad_p, void* d_workspace,
                            size_t workspace_bytes, aug_stream_t stream);

/* The scalar training loss of Sec. 5.C, the mean over the batch of the
 * per-volume losses: *d_mean = (1/n_vols) sum_b d_loss[b], summed in double in a
 * fixed order (reproducible), rounded to float32.  d_grad_p of
 * iou_loss_fwd_bwd / seg_loss_fwd_bwd is already the gradient of this mean.
 * d_loss: [n_vols] float32 device; d_mean: one float32 device.  One small
 * kernel on `stream`.  AUG_ERR_INVALID_ARG: NULL pointers or n_vols outside
 * 1..65535. */
aug_status aug_loss_batch_mean(const float* d_loss, int n_vols, float* d_mean,
                               aug_stream_t stream);

/* ---- overlap-loss variants (Sec. 5.C) in the same fused kernels --------------
 * Generalises iou_loss_fwd_bwd (which is kind = AUG_LOSS_IOU, power = 1,
 * logits = 0) to the other losses the paper discusses.  Per volume b, class c
 * and output voxel k, with y_k = [warped label == c]:
 *   p_k = x_k                                  (logits == 0: probabilities)
 *   p_k = exp(x_{c,k}) / sum_j exp(x_{j,k})    (logits != 0: class scores,
 *                                               softmax over the C classes)
 *   q_k = p_k^power                            (the L^m family, power > 0)
 *   I = sum q y, P = sum q, Y = sum y,
 *   AUG_LOSS_IOU:  L_bc = 1 - I / (P + Y - I)
 *   AUG_LOSS_DICE: L_bc = 1 - 2 I / (P + Y)
 * (L_bc = 0 and no gradient where the denominator is 0);
 * loss[b] = mean_c L_bc, and d_grad_x = d(mean_b loss[b]) / d x, i.e. with
 * respect to the scores when logits != 0 (softmax chain rule included).
 * Layouts as iou_loss_fwd_bwd (d_x, d_grad_x: [C][out_nz][out_ny][out_nx] per
 * volume, packed).  power must be finite and > 0 (else AUG_ERR_INVALID_ARG);
 * with power < 1 a probability of exactly 0 has an infinite derivative.
 * p^power is a product for power 2, 3 or 4 and the hardware log2/exp2
 * otherwise; exp and the reciprocal use the hardware approximations (relative
 * error ~1e-6).  Variants and autotuning are shared with op 2. */
typedef enum { AUG_LOSS_IOU = 0, AUG_LOSS_DICE = 1 } aug_loss_kind;

aug_status seg_loss_fwd_bwd(const aug_volume_desc* d_descs, int n_vols, const float* d_x,
                            int n_classes, int kind, float power, int logits, float* d_loss,
                            float* d_grad_x, void* d_workspace, size_t workspace_bytes,
                            aug_stream_t stream);

/* ---- allocation-free variant of iou_loss_fwd_bwd --------------------------------
 * The paper has no counterpart to this entry point; it exists for callers
 * that must not allocate device memory: plug-ins hosted by a framework that
 * owns the whole device memory budget and hands out no scratch buffers, and
 * latency-critical loops that may not allocate once they have started (an
 * allocation can block on the device and take milliseconds).
 *
 * Computes exactly what iou_loss_fwd_bwd computes (same arguments and
 * layouts), but instead of a caller-provided workspace it uses one
 * fixed-size scratch array (about 3.2 MB) that the library keeps in device
 * memory on every GPU that loads it, until the process exits.  The caller
 * still passes all inputs and outputs.  No device memory is allocated by this
 * call or by the library on its behalf.
 *
 * Limits: 1 <= n_vols <= 64 (else AUG_ERR_INVALID_ARG), 1 <= n_classes <= 8
 * (else AUG_ERR_UNSUPPORTED); at most 256 thread blocks per pass.
 * d_status: NULL, or a device int32[2] that receives (status, bad volume) of
 * this call's descriptor checks: (0, -1) when every descriptor is valid, else
 * (AUG_ERR_DESCRIPTOR, index of the first invalid volume), as
 * aug_read_device_status reports them.  d_grad_p NULL computes the loss only.
 *
 * The first call on a device (and again after the device's context has been
 * recreated, e.g. by cudaDeviceReset) looks up the array's device address in
 * the current context, with that device current; make that first call before
 * any stream capture.  All calls share the one array and each call overwrites it, so
 * calls that may overlap on the GPU (different streams, or several host
 * threads) race and give wrong results: serialise them. */
aug_status iou_loss_fwd_bwd_noalloc(const aug_volume_desc* d_descs, int n_vols,
                                    const float* d_p, int n_classes, float* d_loss,
                                    float* d_grad_p, int* d_status, aug_stream_t stream);

/* ---- kernel variants and autotuning -----------------------------------------
 * op: 0 = aug_warp_fwd, 1 = aug_warp_bwd, 2 = iou_loss_fwd_bwd.
 * Variants differ in tile shape (warps per CTA along y, z-run per thread);
 * all compute the same result.  Settings are process-wide host state. */
int aug_num_variants(int op);
const char* aug_variant_name(int op, int variant);
/* variant -1 restores the built-in default. */
aug_status aug_set_variant(int op, int variant);
int aug_get_variant(int op);

/* Times every variant of `op` on the given batch (reps launches each, after
 * one warm-up, CUDA events on `stream`), selects the fastest with
 * aug_set_variant and returns it in *best (may be NULL) with its mean time in
 * *best_ms (may be NULL).  Synchronises `stream`; must not be called while
 * the stream is being captured.  The arguments are those of the op's entry
 * point; unused ones may be NULL/0 (op 0 uses d_descs, n_vols, seed; op 1
 * adds d_grad_out, d_grad_in, d_grad_affine; op 2 adds d_p, n_classes, d_loss,
 * d_grad_p).  The outputs of the op are overwritten. */
aug_status aug_autotune(int op, const aug_volume_desc* d_descs, int n_vols, uint64_t seed,
                        const float* const* d_grad_out, float* const* d_grad_in,
                        float* d_grad_affine, const float* d_p, int n_classes, float* d_loss,
                        float* d_grad_p, void* d_workspace, size_t workspace_bytes,
                        aug_stream_t stream, int reps, int* best, float* best_ms);

/* ---- diagnostics -------------------------------------------------------------
 * Philox4x32-10 words computed by the device generator the warp uses:
 * d_out[4m..4m+3] = Philox4x32-10(counter = d_ctr[4m..4m+3], key = (lo32(seed),
 * hi32(seed))), m < n.  For bit-exact comparison with other implementations. */
aug_status aug_philox4x32_10(const uint32_t* d_ctr, int64_t n, uint64_t seed,
                             uint32_t* d_out, aug_stream_t stream);

/* Human-readable name of a status code.  Host function, never NULL. */
const char* aug_status_string(int status);

/* Library version as MAJOR*10000 + MINOR*100 + PATCH. */
int aug_version(void);

#if defined(__GNUC__)
#pragma GCC visibility pop
#endif

#ifdef __cplusplus
}
#endif

#endif /* AUGWARP_H */
