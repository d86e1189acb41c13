"""Python binding of libaugwarp.so (include/augwarp.h).

Argument marshalling only: every step of the augmentation runs in the CUDA
library.  PyTorch supplies device memory and the current stream.  The names
mirror the C entry points (``aug_warp_fwd``, ``aug_warp_bwd``,
``iou_loss_fwd_bwd`` ...); on top sit :class:`VolumeBatch` (descriptor
packing) and the autograd functions :class:`AugWarp` and :class:`IouLoss`.

If the compiled library is missing this module raises at import time: there
is no CPU fallback.
"""
from __future__ import annotations

import ctypes as C
import os
from typing import Optional, Sequence

import numpy as np
import torch

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libaugwarp.so")

AUG_OK, AUG_ERR_INVALID_ARG, AUG_ERR_CUDA, AUG_ERR_WORKSPACE, AUG_ERR_DESCRIPTOR, \
    AUG_ERR_UNSUPPORTED, AUG_ERR_TIMEOUT = range(7)
AUG_F32, AUG_I16 = 0, 1
AUG_FLAG_WINDOW, AUG_FLAG_OCCLUDE = 1, 2
OP_FWD, OP_BWD, OP_IOU = 0, 1, 2
AUG_LOSS_IOU, AUG_LOSS_DICE = 0, 1
AUG_DRAW_AFFINE, AUG_DRAW_PHOTO, AUG_DRAW_WINDOW, AUG_DRAW_OCCLUDE = 1, 2, 4, 8

# Layout of aug_volume_desc (144 bytes, 16-byte aligned).
DESC_DTYPE = np.dtype({
    "names": ["image", "label", "out_image", "out_label", "in_nx", "in_ny", "in_nz",
              "image_dtype", "out_nx", "out_ny", "out_nz", "fill_label", "affine", "photo_a",
              "photo_b", "noise_sigma", "fill_image", "noise_id", "flags", "occ_z0", "occ_dz"],
    "formats": ["<u8", "<u8", "<u8", "<u8", "<i4", "<i4", "<i4", "<i4", "<i4", "<i4", "<i4",
                "<i4", ("<f4", (12,)), "<f4", "<f4", "<f4", "<f4", "<u4", "<u4", "<f4", "<f4"],
    "offsets": [0, 8, 16, 24, 32, 36, 40, 44, 48, 52, 56, 60, 64, 112, 116, 120, 124, 128, 132,
                136, 140],
    "itemsize": 144,
})


class AugError(RuntimeError):
    def __init__(self, status: int, where: str):
        self.status = status
        super().__init__(f"{where}: {status_string(status)} (status {status})")


def _load():
    if not os.path.exists(LIB_PATH):
        raise ImportError(
            f"{LIB_PATH} is missing: build it with `python -m paper_1811_11226_b300.build` "
            "(nvcc, sm_103a). There is no CPU fallback.")
    L = C.CDLL(LIB_PATH)
    vp, i32, i64, u64, sz, f32p = C.c_void_p, C.c_int, C.c_int64, C.c_uint64, C.c_size_t, \
        C.POINTER(C.c_float)
    L.aug_workspace_size.argtypes = [i32, i32]
    L.aug_workspace_size.restype = sz
    L.aug_read_device_status.argtypes = [vp, vp, i32, C.POINTER(C.c_int)]
    L.aug_read_device_status.restype = i32
    L.aug_warp_fwd.argtypes = [vp, i32, u64, vp, sz, vp]
    L.aug_warp_fwd.restype = i32
    L.aug_warp_fwd_volume.argtypes = [vp, u64, vp]
    L.aug_warp_fwd_volume.restype = i32
    L.aug_warp_bwd.argtypes = [vp, i32, vp, vp, vp, vp, sz, vp]
    L.aug_warp_bwd.restype = i32
    L.iou_loss_fwd_bwd.argtypes = [vp, i32, vp, i32, vp, vp, vp, sz, vp]
    L.iou_loss_fwd_bwd.restype = i32
    L.seg_loss_fwd_bwd.argtypes = [vp, i32, vp, i32, i32, C.c_float, i32, vp, vp, vp, sz, vp]
    L.seg_loss_fwd_bwd.restype = i32
    L.aug_sample_params.argtypes = [vp, i32, vp, u64, u64, vp, vp]
    L.aug_sample_params.restype = i32
    L.aug_warp_fwd_host.argtypes = [vp, i32, u64, i32, vp]
    L.aug_warp_fwd_host.restype = i32
    L.aug_tex_create.argtypes = [vp, i32, C.POINTER(vp)]
    L.aug_tex_create.restype = i32
    L.aug_tex_warp_fwd.argtypes = [vp, u64, vp]
    L.aug_tex_warp_fwd.restype = i32
    L.aug_tex_destroy.argtypes = [vp]
    L.aug_tex_destroy.restype = i32
    L.aug_smooth.argtypes = [vp, i32, vp]
    L.aug_smooth.restype = i32
    L.aug_test_smooth_wait_timeout.argtypes = [vp, i32, vp]
    L.aug_test_smooth_wait_timeout.restype = i32
    L.aug_smooth_status.argtypes = [vp]
    L.aug_smooth_status.restype = i32
    L.aug_antialias_sigma.argtypes = [C.c_float, C.c_float]
    L.aug_antialias_sigma.restype = C.c_float
    L.aug_loss_batch_mean.argtypes = [vp, i32, vp, vp]
    L.aug_loss_batch_mean.restype = i32
    L.iou_loss_fwd_bwd_noalloc.argtypes = [vp, i32, vp, i32, vp, vp, vp, vp]
    L.iou_loss_fwd_bwd_noalloc.restype = i32
    L.aug_num_variants.argtypes = [i32]
    L.aug_num_variants.restype = i32
    L.aug_variant_name.argtypes = [i32, i32]
    L.aug_variant_name.restype = C.c_char_p
    L.aug_set_variant.argtypes = [i32, i32]
    L.aug_set_variant.restype = i32
    L.aug_get_variant.argtypes = [i32]
    L.aug_get_variant.restype = i32
    L.aug_autotune.argtypes = [i32, vp, i32, u64, vp, vp, vp, vp, i32, vp, vp, vp, sz, vp, i32,
                               C.POINTER(C.c_int), f32p]
    L.aug_autotune.restype = i32
    L.aug_philox4x32_10.argtypes = [vp, i64, u64, vp, vp]
    L.aug_philox4x32_10.restype = i32
    L.aug_status_string.argtypes = [i32]
    L.aug_status_string.restype = C.c_char_p
    L.aug_version.argtypes = []
    L.aug_version.restype = i32
    return L


_L = _load()


def lib():
    return _L


def status_string(status: int) -> str:
    return _L.aug_status_string(int(status)).decode()


def _check(status: int, where: str):
    if status != AUG_OK:
        raise AugError(status, where)


def _ptr(t: Optional[torch.Tensor]):
    return None if t is None else C.c_void_p(t.data_ptr())


def _stream(stream=None):
    s = torch.cuda.current_stream() if stream is None else stream
    return C.c_void_p(s.cuda_stream)


def _seed(seed: int) -> int:
    return int(seed) & 0xFFFFFFFFFFFFFFFF


# ---- workspace ----------------------------------------------------------------------
def aug_workspace_size(n_vols: int, n_classes: int = 0) -> int:
    return int(_L.aug_workspace_size(int(n_vols), int(n_classes)))


def make_workspace(n_vols: int, n_classes: int = 0, device=None) -> torch.Tensor:
    n = aug_workspace_size(n_vols, n_classes)
    if n == 0:
        raise AugError(AUG_ERR_INVALID_ARG, "aug_workspace_size")
    ws = torch.zeros(n + 256, dtype=torch.uint8, device=device or "cuda")
    off = (-ws.data_ptr()) % 256
    return ws[off: off + n]


def aug_read_device_status(workspace: torch.Tensor, clear: bool = True, stream=None):
    bad = C.c_int(-1)
    st = _L.aug_read_device_status(_ptr(workspace), _stream(stream), int(clear), C.byref(bad))
    return int(st), int(bad.value)


# ---- raw entry points (device descriptor arrays) ----------------------------------------
def aug_warp_fwd(d_descs: torch.Tensor, n_vols: int, seed: int, workspace: torch.Tensor,
                 stream=None):
    _check(_L.aug_warp_fwd(_ptr(d_descs), int(n_vols), _seed(seed), _ptr(workspace),
                           workspace.numel(), _stream(stream)), "aug_warp_fwd")


def aug_warp_fwd_volume(h_desc: np.ndarray, seed: int, stream=None):
    h = np.ascontiguousarray(h_desc, dtype=DESC_DTYPE).reshape(1)
    _check(_L.aug_warp_fwd_volume(h.ctypes.data_as(C.c_void_p), _seed(seed), _stream(stream)),
           "aug_warp_fwd_volume")


def aug_warp_fwd_host(h_descs: np.ndarray, seed: int, chunk_vols: int = 8, stream=None):
    """Forward from HOST buffers (descriptor pointers are host addresses, ideally
    page-locked), pipelined over chunks of volumes; ordered on ``stream``."""
    h = np.ascontiguousarray(h_descs, dtype=DESC_DTYPE)
    _check(_L.aug_warp_fwd_host(h.ctypes.data_as(C.c_void_p), len(h), _seed(seed),
                                int(chunk_vols), _stream(stream)), "aug_warp_fwd_host")


def host_descriptors(images, affines, out_shapes, labels=None, out_images=None, out_labels=None,
                     photo_a=None, photo_b=None, noise_sigma=None, fill_image=-1000.0,
                     fill_label=0, noise_ids=None):
    """Descriptor array for aug_warp_fwd_host from CPU tensors (page-locked for
    overlap): the same fields as VolumeBatch, with host addresses."""
    B = len(out_shapes)
    h = np.zeros(B, DESC_DTYPE)
    h["affine"] = np.asarray(affines.detach().cpu() if torch.is_tensor(affines) else affines,
                             np.float32).reshape(B, 12)
    h["photo_a"] = 1.0 if photo_a is None else np.asarray(photo_a, np.float32)
    h["photo_b"] = 0.0 if photo_b is None else np.asarray(photo_b, np.float32)
    h["noise_sigma"] = 0.0 if noise_sigma is None else np.asarray(noise_sigma, np.float32)
    h["fill_image"] = fill_image
    h["fill_label"] = fill_label
    h["noise_id"] = np.arange(B, dtype=np.uint32) if noise_ids is None else np.asarray(
        noise_ids, np.uint32)
    for b in range(B):
        img = images[b]
        assert not img.is_cuda and img.is_contiguous() and img.dim() == 3
        h["image"][b] = img.data_ptr()
        h["image_dtype"][b] = _dtype_code(img)
        h["in_nz"][b], h["in_ny"][b], h["in_nx"][b] = img.shape
        onx, ony, onz = (int(v) for v in out_shapes[b])
        h["out_nx"][b], h["out_ny"][b], h["out_nz"][b] = onx, ony, onz
        if labels is not None and labels[b] is not None:
            assert not labels[b].is_cuda and labels[b].dtype == torch.uint8
            h["label"][b] = labels[b].data_ptr()
        if out_images is not None and out_images[b] is not None:
            assert not out_images[b].is_cuda and tuple(out_images[b].shape) == (onz, ony, onx)
            h["out_image"][b] = out_images[b].data_ptr()
        if out_labels is not None and out_labels[b] is not None:
            assert not out_labels[b].is_cuda and tuple(out_labels[b].shape) == (onz, ony, onx)
            h["out_label"][b] = out_labels[b].data_ptr()
    return h


class TexWarp:
    """The hardware-texture alternative of the forward (tex3D linear filtering,
    a measured comparison, not a parity path): built from host descriptors
    (device buffers, float32 images), run with ``run(seed)``, freed by
    ``close()``."""

    def __init__(self, h_descs: np.ndarray):
        self._h = np.ascontiguousarray(h_descs, dtype=DESC_DTYPE)
        self._handle = C.c_void_p()
        _check(_L.aug_tex_create(self._h.ctypes.data_as(C.c_void_p), len(self._h),
                                 C.byref(self._handle)), "aug_tex_create")

    def run(self, seed: int, stream=None):
        _check(_L.aug_tex_warp_fwd(self._handle, _seed(seed), _stream(stream)),
               "aug_tex_warp_fwd")

    def close(self):
        if self._handle:
            torch.cuda.synchronize()
            _L.aug_tex_destroy(self._handle)
            self._handle = C.c_void_p()


def aug_warp_bwd(d_descs: torch.Tensor, n_vols: int, d_grad_out_ptrs: torch.Tensor,
                 d_grad_in_ptrs: Optional[torch.Tensor], grad_affine: Optional[torch.Tensor],
                 workspace: torch.Tensor, stream=None):
    _check(_L.aug_warp_bwd(_ptr(d_descs), int(n_vols), _ptr(d_grad_out_ptrs),
                           _ptr(d_grad_in_ptrs), _ptr(grad_affine), _ptr(workspace),
                           workspace.numel(), _stream(stream)), "aug_warp_bwd")


def iou_loss_fwd_bwd(d_descs: torch.Tensor, n_vols: int, p: torch.Tensor, n_classes: int,
                     loss: torch.Tensor, grad_p: Optional[torch.Tensor],
                     workspace: torch.Tensor, stream=None):
    _check(_L.iou_loss_fwd_bwd(_ptr(d_descs), int(n_vols), _ptr(p), int(n_classes),
                               _ptr(loss), _ptr(grad_p), _ptr(workspace), workspace.numel(),
                               _stream(stream)), "iou_loss_fwd_bwd")


def seg_loss_fwd_bwd(d_descs: torch.Tensor, n_vols: int, x: torch.Tensor, n_classes: int,
                     loss: torch.Tensor, grad_x: Optional[torch.Tensor],
                     workspace: torch.Tensor, kind: int = AUG_LOSS_IOU, power: float = 1.0,
                     logits: bool = False, stream=None):
    """Overlap loss ``kind`` (IOU or Dice) of q = p^power, p = x or, with
    ``logits``, the softmax of x over the classes; grad_x is with respect to x."""
    _check(_L.seg_loss_fwd_bwd(_ptr(d_descs), int(n_vols), _ptr(x), int(n_classes), int(kind),
                               float(power), int(bool(logits)), _ptr(loss), _ptr(grad_x),
                               _ptr(workspace), workspace.numel(), _stream(stream)),
           "seg_loss_fwd_bwd")


class ParamSpec(C.Structure):
    """Ranges of the device-side parameter draw (aug_param_spec): angles in
    radians, lengths in input voxels, [min, max] pairs; ``draw`` is a mask of
    AUG_DRAW_* bits."""
    _fields_ = [("rot_max", C.c_float * 3), ("scale_min", C.c_float * 3),
                ("scale_max", C.c_float * 3), ("reflect_prob", C.c_float * 3),
                ("shear_max", C.c_float), ("generic_max", C.c_float),
                ("extra_scale", C.c_float * 3), ("shift_max", C.c_float * 3),
                ("photo_a", C.c_float * 2), ("photo_b", C.c_float * 2), ("sigma", C.c_float * 2),
                ("window_lo", C.c_float * 2), ("window_hi", C.c_float * 2),
                ("occ_max_frac", C.c_float), ("draw", C.c_uint32)]

    def __init__(self, **kw):
        base = dict(rot_max=(0.0, 0.0, 0.0), scale_min=(1.0, 1.0, 1.0),
                    scale_max=(1.0, 1.0, 1.0), reflect_prob=(0.0, 0.0, 0.0), shear_max=0.0,
                    generic_max=0.0, extra_scale=(1.0, 1.0, 1.0), shift_max=(0.0, 0.0, 0.0),
                    photo_a=(1.0, 1.0), photo_b=(0.0, 0.0), sigma=(0.0, 0.0),
                    window_lo=(-1000.0, -1000.0), window_hi=(1000.0, 1000.0),
                    occ_max_frac=0.0, draw=AUG_DRAW_AFFINE)
        base.update(kw)
        super().__init__()
        for name, _ in self._fields_:
            v = base[name]
            if isinstance(v, (tuple, list, np.ndarray)):
                getattr(self, name)[:] = [float(x) for x in v]
            else:
                setattr(self, name, v)


def aug_sample_params(d_descs: torch.Tensor, n_vols: int, spec: ParamSpec, seed: int,
                      draw: int = 0, counter: Optional[torch.Tensor] = None, stream=None):
    """Draws every volume's parameters into the device descriptors.  ``counter``:
    optional int64 CUDA tensor of one element, added to ``draw`` and advanced
    by the call (so graph replays draw new parameters)."""
    if counter is not None:
        assert counter.is_cuda and counter.dtype == torch.int64 and counter.numel() == 1
    _check(_L.aug_sample_params(_ptr(d_descs), int(n_vols), C.byref(spec), _seed(seed),
                                _seed(draw), _ptr(counter), _stream(stream)),
           "aug_sample_params")


SMOOTH_DTYPE = np.dtype([("image", "<u8"), ("out", "<u8"), ("nx", "<i4"), ("ny", "<i4"),
                         ("nz", "<i4"), ("image_dtype", "<i4"), ("sigma", "<f4", 3),
                         ("fill", "<f4")])


def aug_smooth_status() -> int:
    """0, or 1 if a smoothing block gave up waiting for its input since the last
    read (synchronises the device; clears the word)."""
    st = C.c_int(0)
    _check(_L.aug_smooth_status(C.byref(st)), "aug_smooth_status")
    return st.value


def aug_antialias_sigma(r: float, u: float) -> float:
    """max(r/u - 1, 0)/3: Gaussian factor of the resampling of Sec. 5.A."""
    return float(_L.aug_antialias_sigma(float(r), float(u)))


def _smooth_descs(images, outs, sigmas, fill):
    n = len(images)
    h = np.zeros(n, SMOOTH_DTYPE)
    fl = np.broadcast_to(np.asarray(fill, np.float32), (n,))
    for b, (img, out) in enumerate(zip(images, outs)):
        assert img.is_cuda and img.is_contiguous() and img.dim() == 3
        assert out.is_cuda and out.is_contiguous() and out.dtype == torch.float32
        assert tuple(out.shape) == tuple(img.shape)
        h["image"][b], h["out"][b] = img.data_ptr(), out.data_ptr()
        h["nz"][b], h["ny"][b], h["nx"][b] = img.shape
        h["image_dtype"][b] = _dtype_code(img)
        h["sigma"][b] = np.asarray(sigmas[b], np.float32)
        h["fill"][b] = fl[b]
    return h


def aug_test_smooth_wait_timeout(images, outs, sigmas, fill=-1000.0, stream=None):
    """The smoothing kernel with no tile copies issued: every wait runs out and
    is recorded in the smoothing status (a test of the bounded waits)."""
    h = _smooth_descs(images, outs, sigmas, fill)
    _check(_L.aug_test_smooth_wait_timeout(h.ctypes.data_as(C.c_void_p), len(h),
                                           _stream(stream)), "aug_test_smooth_wait_timeout")


def aug_smooth(images: Sequence[torch.Tensor], outs: Sequence[torch.Tensor], sigmas,
               fill=-1000.0, stream=None):
    """Anti-aliasing Gaussian of each [nz, ny, nx] float32/int16 CUDA volume into
    the float32 volume of the same shape; ``sigmas``: per volume (sx, sy, sz)."""
    h = _smooth_descs(images, outs, sigmas, fill)
    _check(_L.aug_smooth(h.ctypes.data_as(C.c_void_p), len(h), _stream(stream)), "aug_smooth")


def aug_loss_batch_mean(loss: torch.Tensor, stream=None) -> torch.Tensor:
    """Mean over the batch of per-volume losses (Sec. 5.C), computed on the
    device: returns a 0-dim float32 tensor."""
    out = torch.empty((), dtype=torch.float32, device=loss.device)
    _check(_L.aug_loss_batch_mean(_ptr(loss), int(loss.numel()), _ptr(out), _stream(stream)),
           "aug_loss_batch_mean")
    return out


def iou_loss_fwd_bwd_noalloc(d_descs: torch.Tensor, n_vols: int, p: torch.Tensor,
                             n_classes: int, loss: torch.Tensor, grad_p: Optional[torch.Tensor],
                             status: Optional[torch.Tensor] = None, stream=None):
    """iou_loss_fwd_bwd without a caller workspace: the library's own fixed
    scratch array is used (at most 64 volumes, 8 classes).  ``status``: optional
    int32[2] CUDA tensor receiving (device status, bad volume)."""
    _check(_L.iou_loss_fwd_bwd_noalloc(_ptr(d_descs), int(n_vols), _ptr(p), int(n_classes),
                                       _ptr(loss), _ptr(grad_p), _ptr(status), _stream(stream)),
           "iou_loss_fwd_bwd_noalloc")


def aug_philox4x32_10(ctr: torch.Tensor, seed: int, stream=None) -> torch.Tensor:
    """Device Philox4x32-10 words for counters ``ctr`` ([n, 4] int32/uint32 on cuda)."""
    ctr = ctr.contiguous()
    out = torch.empty_like(ctr)
    _check(_L.aug_philox4x32_10(_ptr(ctr), ctr.numel() // 4, _seed(seed), _ptr(out),
                                _stream(stream)), "aug_philox4x32_10")
    return out


def aug_num_variants(op: int) -> int:
    return int(_L.aug_num_variants(op))


def aug_variant_name(op: int, v: int) -> str:
    return _L.aug_variant_name(op, v).decode()


def aug_set_variant(op: int, v: int):
    _check(_L.aug_set_variant(op, v), "aug_set_variant")


def aug_get_variant(op: int) -> int:
    return int(_L.aug_get_variant(op))


def aug_autotune(op: int, batch: "VolumeBatch", workspace: torch.Tensor, *, seed: int = 0,
                 grad_out_ptrs=None, grad_in_ptrs=None, grad_affine=None, p=None,
                 n_classes: int = 0, loss=None, grad_p=None, reps: int = 5, stream=None):
    best, ms = C.c_int(-1), C.c_float(0.0)
    _check(_L.aug_autotune(op, _ptr(batch.d_descs), batch.n, _seed(seed), _ptr(grad_out_ptrs),
                           _ptr(grad_in_ptrs), _ptr(grad_affine), _ptr(p), int(n_classes),
                           _ptr(loss), _ptr(grad_p), _ptr(workspace), workspace.numel(),
                           _stream(stream), int(reps), C.byref(best), C.byref(ms)),
           "aug_autotune")
    return int(best.value), float(ms.value)


def aug_version() -> int:
    return int(_L.aug_version())


# ---- descriptor packing ------------------------------------------------------------------
def _dtype_code(t: torch.Tensor) -> int:
    if t.dtype == torch.float32:
        return AUG_F32
    if t.dtype == torch.int16:
        return AUG_I16
    raise TypeError(f"image dtype must be float32 or int16, got {t.dtype}")


class VolumeBatch:
    """A batch of volume descriptors (host copy + device copy).

    ``images``/``labels``: per volume ``[nz, ny, nx]`` contiguous CUDA tensors
    (labels uint8 or None).  ``out_images``/``out_labels``: per volume output
    tensors ``[onz, ony, onx]`` (float32 / uint8) or None.  ``affines``:
    ``[B, 3, 4]`` float32 (output index -> input coordinate).  The batch keeps
    references to every tensor it points to.
    """

    def __init__(self, images: Sequence[Optional[torch.Tensor]], affines, out_shapes,
                 labels=None, out_images=None, out_labels=None, photo_a=None, photo_b=None,
                 noise_sigma=None, fill_image=-1000.0, fill_label=0, noise_ids=None,
                 flags=None, occ_z0=None, occ_dz=None, device=None):
        B = len(out_shapes)
        self.n = B
        h = np.zeros(B, DESC_DTYPE)
        aff = np.asarray(affines.detach().cpu() if torch.is_tensor(affines) else affines,
                         np.float32).reshape(B, 12)
        labels = labels if labels is not None else [None] * B
        out_images = out_images if out_images is not None else [None] * B
        out_labels = out_labels if out_labels is not None else [None] * B
        pa = np.ones(B, np.float32) if photo_a is None else np.asarray(photo_a, np.float32)
        pb = np.zeros(B, np.float32) if photo_b is None else np.asarray(photo_b, np.float32)
        ns = np.zeros(B, np.float32) if noise_sigma is None else np.asarray(noise_sigma,
                                                                              np.float32)
        fi = np.broadcast_to(np.asarray(fill_image, np.float32), (B,))
        fl = np.broadcast_to(np.asarray(fill_label, np.int32), (B,))
        nid = np.arange(B, dtype=np.uint32) if noise_ids is None else np.asarray(noise_ids,
                                                                                  np.uint32)
        self._keep = []
        for b in range(B):
            img, lab, oi, ol = images[b], labels[b], out_images[b], out_labels[b]
            if img is not None:
                assert img.is_cuda and img.is_contiguous() and img.dim() == 3
                h["image"][b] = img.data_ptr()
                h["image_dtype"][b] = _dtype_code(img)
                h["in_nz"][b], h["in_ny"][b], h["in_nx"][b] = img.shape
            if lab is not None:
                assert lab.is_cuda and lab.is_contiguous() and lab.dtype == torch.uint8
                if img is not None:
                    assert tuple(lab.shape) == tuple(img.shape)
                else:
                    h["in_nz"][b], h["in_ny"][b], h["in_nx"][b] = lab.shape
                h["label"][b] = lab.data_ptr()
            onx, ony, onz = (int(v) for v in out_shapes[b])
            h["out_nx"][b], h["out_ny"][b], h["out_nz"][b] = onx, ony, onz
            if oi is not None:
                assert oi.is_cuda and oi.is_contiguous() and oi.dtype == torch.float32
                assert tuple(oi.shape) == (onz, ony, onx)
                h["out_image"][b] = oi.data_ptr()
            if ol is not None:
                assert ol.is_cuda and ol.is_contiguous() and ol.dtype == torch.uint8
                assert tuple(ol.shape) == (onz, ony, onx)
                h["out_label"][b] = ol.data_ptr()
            self._keep += [img, lab, oi, ol]
        h["affine"] = aff
        h["photo_a"], h["photo_b"], h["noise_sigma"] = pa, pb, ns
        h["fill_image"], h["fill_label"], h["noise_id"] = fi, fl, nid
        if flags is not None:
            h["flags"] = np.asarray(flags, np.uint32)
        if occ_z0 is not None:
            h["occ_z0"] = np.asarray(occ_z0, np.float32)
        if occ_dz is not None:
            h["occ_dz"] = np.asarray(occ_dz, np.float32)
        self.h_descs = h
        dev = device or (images[0].device if images[0] is not None else torch.device("cuda"))
        self.d_descs = torch.from_numpy(h.view(np.uint8).copy()).to(dev)

    def upload(self):
        """Re-copy the host descriptors to the device (e.g. after editing
        ``h_descs`` between CUDA-graph replays)."""
        self.d_descs.copy_(torch.from_numpy(self.h_descs.view(np.uint8).copy()))

    def download(self):
        """Refresh the host descriptors from the device (e.g. after
        aug_sample_params wrote new parameters there)."""
        self.h_descs = self.d_descs.cpu().numpy().view(DESC_DTYPE).copy()
        return self.h_descs

    def out_voxels(self):
        return [int(self.h_descs["out_nx"][b]) * int(self.h_descs["out_ny"][b]) *
                int(self.h_descs["out_nz"][b]) for b in range(self.n)]


def pointer_array(tensors: Sequence[Optional[torch.Tensor]], device) -> torch.Tensor:
    """Device array of raw pointers (int64) for the adjoint's per-volume buffers."""
    return torch.tensor([0 if t is None else t.data_ptr() for t in tensors], dtype=torch.int64,
                        device=device)


# ---- autograd wrappers ----------------------------------------------------------------------
class AugWarp(torch.autograd.Function):
    """Differentiable warp of a batch of equal-shape float32 volumes.

    forward(image [B, D, H, W], affine [B, 3, 4], out_shape (onx, ony, onz),
    photo [B, 2] (a, b) or None, sigma [B] or None, seed, fill) ->
    out [B, onz, ony, onx].  backward returns the gradients with respect to
    ``image`` and ``affine`` (aug_warp_bwd)."""

    @staticmethod
    def forward(ctx, image, affine, out_shape, photo=None, sigma=None, seed=0, fill=-1000.0):
        B = image.shape[0]
        onx, ony, onz = (int(v) for v in out_shape)
        image = image.contiguous()
        out = torch.empty((B, onz, ony, onx), dtype=torch.float32, device=image.device)
        pa = None if photo is None else photo[:, 0].detach().cpu().numpy()
        pb = None if photo is None else photo[:, 1].detach().cpu().numpy()
        sg = None if sigma is None else sigma.detach().cpu().numpy()
        batch = VolumeBatch([image[b] for b in range(B)], affine, [(onx, ony, onz)] * B,
                            out_images=[out[b] for b in range(B)], photo_a=pa, photo_b=pb,
                            noise_sigma=sg, fill_image=fill)
        ws = make_workspace(B, 0, image.device)
        aug_warp_fwd(batch.d_descs, B, seed, ws)
        ctx.save_for_backward(image, affine)
        ctx.batch, ctx.ws = batch, ws
        ctx.needs = (ctx.needs_input_grad[0], ctx.needs_input_grad[1])
        return out

    @staticmethod
    def backward(ctx, grad_out):
        image, affine = ctx.saved_tensors
        B = image.shape[0]
        g = grad_out.contiguous()
        gptr = pointer_array([g[b] for b in range(B)], image.device)
        gin = torch.empty_like(image) if ctx.needs[0] else None
        giptr = pointer_array([gin[b] for b in range(B)], image.device) if ctx.needs[0] else None
        gaff = torch.empty((B, 3, 4), dtype=torch.float32, device=image.device) \
            if ctx.needs[1] else None
        aug_warp_bwd(ctx.batch.d_descs, B, gptr, giptr, gaff, ctx.ws)
        return gin, gaff, None, None, None, None, None


class IouLoss(torch.autograd.Function):
    """Soft IOU loss of class probabilities against nearest-warped labels,
    mean over classes and batch (Sec. 5.C).  forward(p [B, C, onz, ony, onx],
    labels [B, D, H, W] uint8, affine [B, 3, 4]) -> scalar; the gradient with
    respect to p comes from the same fused call."""

    @staticmethod
    def forward(ctx, p, labels, affine):
        B, Cn = p.shape[0], p.shape[1]
        onz, ony, onx = p.shape[2:]
        p = p.contiguous()
        batch = VolumeBatch([None] * B, affine, [(onx, ony, onz)] * B,
                            labels=[labels[b] for b in range(B)], device=p.device)
        ws = make_workspace(B, Cn, p.device)
        loss = torch.empty(B, dtype=torch.float32, device=p.device)
        gp = torch.empty_like(p) if ctx.needs_input_grad[0] else None
        iou_loss_fwd_bwd(batch.d_descs, B, p, Cn, loss, gp, ws)
        ctx.gp = gp
        return aug_loss_batch_mean(loss)

    @staticmethod
    def backward(ctx, grad):
        return ctx.gp * grad, None, None


class SegLoss(torch.autograd.Function):
    """Overlap loss of Sec. 5.C against nearest-warped labels, mean over classes
    and batch: forward(x [B, C, onz, ony, onx], labels [B, D, H, W] uint8,
    affine [B, 3, 4], kind, power, logits) -> scalar, with kind AUG_LOSS_IOU or
    AUG_LOSS_DICE, p replaced by p^power, and x class scores (softmax fused)
    when ``logits``; the gradient comes from the same fused call."""

    @staticmethod
    def forward(ctx, x, labels, affine, kind=AUG_LOSS_IOU, power=1.0, logits=False):
        B, Cn = x.shape[0], x.shape[1]
        onz, ony, onx = x.shape[2:]
        x = x.contiguous()
        batch = VolumeBatch([None] * B, affine, [(onx, ony, onz)] * B,
                            labels=[labels[b] for b in range(B)], device=x.device)
        ws = make_workspace(B, Cn, x.device)
        loss = torch.empty(B, dtype=torch.float32, device=x.device)
        gx = torch.empty_like(x) if ctx.needs_input_grad[0] else None
        seg_loss_fwd_bwd(batch.d_descs, B, x, Cn, loss, gx, ws, kind, power, logits)
        ctx.gx = gx
        return aug_loss_batch_mean(loss)

    @staticmethod
    def backward(ctx, grad):
        return ctx.gx * grad, None, None, None, None, None
