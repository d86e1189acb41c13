"""Python entry points of the FP64 oracle (ctypes over liboracle.so).

TEST INFRASTRUCTURE ONLY -- used by tests, ``smoke()`` and the benchmark's
CPU baseline, never by the product path.

Inputs are numpy arrays (torch tensors are converted with ``.cpu().numpy()``);
volume records are any object with the fields of ``synth.workloads.VolumeCase``.
"""
from __future__ import annotations

import ctypes as C
import threading

import numpy as np

from . import build as _build

_lib = None
_lock = threading.Lock()

_i64, _u64, _u32, _f32, _int = C.c_int64, C.c_uint64, C.c_uint32, C.c_float, C.c_int
_vp = C.c_void_p


def lib():
    global _lib
    with _lock:
        if _lib is None:
            path = _build.build()
            L = C.CDLL(path)
            L.oracle_philox4x32_10.argtypes = [_vp, _vp, _vp]
            L.oracle_philox_many.argtypes = [_u64, _vp, _i64, _vp]
            L.oracle_noise.argtypes = [_u64, _u32, _i64, _i64, _vp, _i64, _vp]
            fwd_args = [_vp, _int, _vp, _i64, _i64, _i64, _i64, _i64, _i64, _vp, _f32, _f32,
                        _f32, _f32, _int, _u64, _u32, _int, _f32, _f32]
            L.oracle_warp_fwd.argtypes = fwd_args + [_vp, _vp, _vp]
            L.oracle_warp_fwd.restype = _i64
            L.oracle_warp_fwd_points.argtypes = fwd_args + [_vp, _i64, _vp, _vp, _vp]
            L.oracle_warp_bwd.argtypes = [_vp, _int, _i64, _i64, _i64, _i64, _i64, _i64, _vp,
                                          _f32, _f32, _int, _f32, _f32, _vp, _vp, _vp, _vp]
            L.oracle_iou.argtypes = [_vp, _vp, _int, _i64, C.c_double, _vp, _vp, _vp]
            L.oracle_sample_params.argtypes = [_vp, C.c_uint32, _u64, _u64, C.c_uint32, _vp,
                                               _vp, _vp, _vp, _vp, _vp, _vp, _vp]
            L.oracle_antialias_sigma.argtypes = [C.c_double, C.c_double]
            L.oracle_antialias_sigma.restype = C.c_double
            L.oracle_gauss_radius.argtypes = [C.c_double]
            L.oracle_gauss_radius.restype = _int
            L.oracle_gauss_weights.argtypes = [C.c_double, _vp]
            L.oracle_smooth.argtypes = [_vp, _int, _i64, _i64, _i64, _vp, C.c_double, _vp]
            L.oracle_smooth_points.argtypes = [_vp, _int, _i64, _i64, _i64, _vp, C.c_double, _vp,
                                               _i64, _vp]
            L.oracle_loss.argtypes = [_vp, _vp, _int, _i64, _int, C.c_double, _int,
                                      C.c_double, _vp, _vp, _vp]
            _lib = L
    return _lib


def _np(x, dtype=None):
    if x is None:
        return None
    if hasattr(x, "detach"):
        x = x.detach().cpu().numpy()
    x = np.ascontiguousarray(x)
    if dtype is not None and x.dtype != dtype:
        raise TypeError(f"expected {dtype}, got {x.dtype}")
    return x


def _ptr(a):
    return None if a is None else a.ctypes.data_as(_vp)


def philox(ctrs, seed: int):
    """Philox4x32-10 words for counters ``ctrs`` ([n, 4] uint32), key from ``seed``."""
    c = _np(np.asarray(ctrs, dtype=np.uint32).reshape(-1, 4), np.uint32)
    out = np.empty_like(c)
    lib().oracle_philox_many(_u64(seed), _ptr(c), c.shape[0], _ptr(out))
    return out


def noise(seed: int, noise_id: int, onx: int, ony: int, q):
    """Standard normals of the flattened output indices ``q``."""
    q = _np(np.asarray(q, dtype=np.int64), np.int64)
    z = np.empty(q.shape, dtype=np.float64)
    lib().oracle_noise(_u64(seed), _u32(noise_id), onx, ony, _ptr(q), q.size, _ptr(z))
    return z


def _extra(v):
    """Optional window/level and occlusion fields (flags, occ_z0, occ_dz)."""
    return [int(getattr(v, "flags", 0)), _f32(getattr(v, "occ_z0", 0.0)),
            _f32(getattr(v, "occ_dz", 0.0))]


def _vol_args(v, seed):
    img = _np(v.image)
    if img.dtype not in (np.float32, np.int16):
        raise TypeError("image must be float32 or int16")
    lab = _np(v.label, np.uint8) if v.label is not None else None
    nz, ny, nx = img.shape
    onx, ony, onz = v.out_shape
    T = np.ascontiguousarray(np.asarray(v.T, dtype=np.float32).reshape(12))
    keep = (img, lab, T)
    args = [_ptr(img), int(img.dtype == np.int16), _ptr(lab), nx, ny, nz, onx, ony, onz,
            _ptr(T), _f32(v.photo_a), _f32(v.photo_b), _f32(v.sigma), _f32(v.fill_image),
            int(v.fill_label), _u64(seed), _u32(v.noise_id), *_extra(v)]
    return args, keep


def warp_fwd(v, seed: int, want_image=True, want_label=True):
    """Whole-grid forward warp of one volume.

    Returns ``(image f64 [onz, ony, onx] or None, label u8 or None,
    tie u8 flags, n_ties)``."""
    args, keep = _vol_args(v, seed)
    onx, ony, onz = v.out_shape
    out = np.empty((onz, ony, onx), np.float64) if want_image else None
    lab = (np.empty((onz, ony, onx), np.uint8)
           if (want_label and v.label is not None) else None)
    tie = np.empty((onz, ony, onx), np.uint8)
    n = lib().oracle_warp_fwd(*args, _ptr(out), _ptr(lab), _ptr(tie))
    del keep
    return out, lab, tie, int(n)


def warp_fwd_points(v, seed: int, q):
    """Forward warp at flattened output indices ``q``: (values f64, labels u8, ties u8)."""
    args, keep = _vol_args(v, seed)
    q = _np(np.asarray(q, dtype=np.int64), np.int64)
    vals = np.empty(q.shape, np.float64)
    labs = np.empty(q.shape, np.uint8) if v.label is not None else None
    ties = np.empty(q.shape, np.uint8)
    lib().oracle_warp_fwd_points(*args, _ptr(q), q.size, _ptr(vals), _ptr(labs), _ptr(ties))
    del keep
    return vals, labs, ties


def warp_bwd(v, g, want_grad_in=True, want_dvds=False):
    """Adjoint of the image warp of one volume for upstream gradient ``g``
    (output shape).  Returns ``(grad_in f64 or None, grad_T f64 [3, 4],
    dvds f64 [onz, ony, onx, 3] or None)``."""
    img = _np(v.image)
    nz, ny, nx = img.shape
    onx, ony, onz = v.out_shape
    g = _np(g, np.float32)
    assert g.size == onx * ony * onz
    T = np.ascontiguousarray(np.asarray(v.T, dtype=np.float32).reshape(12))
    gi = np.empty((nz, ny, nx), np.float64) if want_grad_in else None
    gt = np.empty(12, np.float64)
    dv = np.empty((onz, ony, onx, 3), np.float64) if want_dvds else None
    lib().oracle_warp_bwd(_ptr(img), int(img.dtype == np.int16), nx, ny, nz, onx, ony, onz,
                          _ptr(T), _f32(v.photo_a), _f32(v.fill_image), *_extra(v), _ptr(g),
                          _ptr(gi), _ptr(gt), _ptr(dv))
    return gi, gt.reshape(3, 4), dv


def iou(p, y, n_classes: int, grad_scale: float = 1.0, want_grad=True):
    """Soft IOU loss of one volume.  ``p``: [C, nvox] float32, ``y``: [nvox]
    uint8.  Returns ``(loss_c [C], sums [C, 3] = (I, P, Y), grad [C, nvox] or None)``."""
    p = _np(p, np.float32).reshape(n_classes, -1)
    y = _np(y, np.uint8).reshape(-1)
    nvox = y.size
    assert p.shape[1] == nvox
    loss = np.empty(n_classes, np.float64)
    sums = np.empty((n_classes, 3), np.float64)
    grad = np.empty((n_classes, nvox), np.float64) if want_grad else None
    lib().oracle_iou(_ptr(p), _ptr(y), n_classes, nvox, C.c_double(grad_scale), _ptr(loss),
                     _ptr(sums), _ptr(grad))
    return loss, sums, grad


def warp_iou(vols, p_packed, n_classes: int, want_grad=True):
    """Label warp followed by the IOU loss, batch-averaged (Sec. 5.C: mean over
    classes, then over the batch).  ``p_packed`` holds per volume
    ``[C][onz][ony][onx]`` consecutively.  Returns ``(loss [B], grad packed f64
    or None, sums [B, C, 3])`` where ``grad`` is the gradient of the batch mean."""
    p = _np(p_packed, np.float32).reshape(-1)
    B = len(vols)
    scale = 1.0 / (B * n_classes)
    losses, sums, grads = [], [], []
    off = 0
    for v in vols:
        nvox = v.n_out
        _, lab, _, _ = warp_fwd(v, 0, want_image=False, want_label=True)
        pc = p[off: off + n_classes * nvox].reshape(n_classes, nvox)
        lc, sc, gc = iou(pc, lab.reshape(-1), n_classes, scale, want_grad)
        losses.append(lc.mean())
        sums.append(sc)
        if want_grad:
            grads.append(gc.reshape(-1))
        off += n_classes * nvox
    grad = np.concatenate(grads) if want_grad else None
    return np.asarray(losses), grad, np.asarray(sums)


LOSS_IOU, LOSS_DICE = 0, 1


def loss(x, y, n_classes: int, kind: int = LOSS_IOU, m: float = 1.0, logits: bool = False,
         grad_scale: float = 1.0, want_grad=True):
    """Loss `kind` (IOU or Dice) of one volume with p replaced by p^m, on
    probabilities or (``logits``) on class scores through a softmax; the
    gradient is with respect to the input x.  Layout as iou()."""
    x = _np(x, np.float32).reshape(n_classes, -1)
    y = _np(y, np.uint8).reshape(-1)
    nvox = y.size
    lossc = np.empty(n_classes, np.float64)
    sums = np.empty((n_classes, 3), np.float64)
    grad = np.empty((n_classes, nvox), np.float64) if want_grad else None
    lib().oracle_loss(_ptr(x), _ptr(y), n_classes, nvox, int(kind), C.c_double(m), int(logits),
                      C.c_double(grad_scale), _ptr(lossc), _ptr(sums), _ptr(grad))
    return lossc, sums, grad


def warp_loss(vols, x_packed, n_classes: int, kind: int = LOSS_IOU, m: float = 1.0,
              logits: bool = False, want_grad=True):
    """Label warp + loss variant, batch-averaged (as warp_iou, same return
    triple); with ``logits`` the gradient is with respect to the class scores."""
    x = _np(x_packed, np.float32).reshape(-1)
    B = len(vols)
    scale = 1.0 / (B * n_classes)
    losses, sums, grads = [], [], []
    off = 0
    for v in vols:
        nvox = v.n_out
        _, lab, _, _ = warp_fwd(v, 0, want_image=False, want_label=True)
        xc = x[off: off + n_classes * nvox].reshape(n_classes, nvox)
        lc, sc, gc = loss(xc, lab.reshape(-1), n_classes, kind, m, logits, scale, want_grad)
        losses.append(lc.mean())
        sums.append(sc)
        if want_grad:
            grads.append(gc.reshape(-1))
        off += n_classes * nvox
    return (np.asarray(losses), (np.concatenate(grads) if want_grad else None),
            np.stack(sums))


# Fields of a parameter-sampling spec, in the oracle's float order (Sec. 4).
SPEC_FIELDS = (("rot_max", 3), ("scale_min", 3), ("scale_max", 3), ("reflect_prob", 3),
               ("shear_max", 1), ("generic_max", 1), ("extra_scale", 3), ("shift_max", 3),
               ("photo_a", 2), ("photo_b", 2), ("sigma", 2), ("window_lo", 2),
               ("window_hi", 2), ("occ_max_frac", 1))
DRAW_AFFINE, DRAW_PHOTO, DRAW_WINDOW, DRAW_OCCLUDE = 1, 2, 4, 8


def spec_floats(spec: dict) -> np.ndarray:
    out = []
    for name, n in SPEC_FIELDS:
        v = np.atleast_1d(np.asarray(spec[name], np.float32))
        assert v.size == n, name
        out.extend(v.tolist())
    return np.asarray(out, np.float32)


def sample_params(spec: dict, draw_mask: int, seed: int, draw: int, noise_id: int, in_dims,
                  out_dims, T=None, photo=(1.0, 0.0, 0.0), flags=0, occ=(0.0, 0.0)):
    """Parameters of one volume drawn as in oracle_sample_params; fields that
    are not drawn keep the values passed in.  Returns a dict with T [3, 4]
    float32, photo_a, photo_b, sigma, flags, occ_z0, occ_dz (float32) and the
    FP64 displacement d and matrix A (NaN where not drawn)."""
    Tv = np.zeros(12, np.float32) if T is None else np.asarray(T, np.float32).reshape(12).copy()
    ph = np.asarray(photo, np.float32).copy()
    fl = np.asarray([flags], np.int32)
    oc = np.asarray(occ, np.float32).copy()
    d = np.full(3, np.nan)
    A = np.full(9, np.nan)
    sp = spec_floats(spec)
    lib().oracle_sample_params(_ptr(sp), int(draw_mask), _u64(seed), _u64(draw), int(noise_id),
                               _ptr(np.asarray(in_dims, np.int64)),
                               _ptr(np.asarray(out_dims, np.int64)), _ptr(Tv), _ptr(ph), _ptr(fl),
                               _ptr(oc), _ptr(d), _ptr(A))
    return dict(T=Tv.reshape(3, 4), photo_a=ph[0], photo_b=ph[1], sigma=ph[2], flags=int(fl[0]),
                occ_z0=oc[0], occ_dz=oc[1], d=d, A=A.reshape(3, 3))


def antialias_sigma(r: float, u: float) -> float:
    """Smoothing factor of the 3 mm resampling (Sec. 5.A), in input voxels."""
    return float(lib().oracle_antialias_sigma(float(r), float(u)))


def gauss_radius(sigma: float) -> int:
    return int(lib().oracle_gauss_radius(float(sigma)))


def gauss_weights(sigma: float) -> np.ndarray:
    R = gauss_radius(sigma)
    w = np.empty(2 * R + 1, np.float64)
    lib().oracle_gauss_weights(float(sigma), _ptr(w))
    return w


def smooth(image, sigma_xyz, fill: float) -> np.ndarray:
    """Anti-aliasing Gaussian of a [nz, ny, nx] float32 / int16 volume (FP64 out)."""
    img = _np(image)
    nz, ny, nx = img.shape
    out = np.empty(img.shape, np.float64)
    lib().oracle_smooth(_ptr(img), int(img.dtype == np.int16), nx, ny, nz,
                        _ptr(np.asarray(sigma_xyz, np.float64)), float(fill), _ptr(out))
    return out


def smooth_points(image, sigma_xyz, fill: float, q) -> np.ndarray:
    img = _np(image)
    nz, ny, nx = img.shape
    q = np.ascontiguousarray(q, np.int64)
    out = np.empty(q.shape, np.float64)
    lib().oracle_smooth_points(_ptr(img), int(img.dtype == np.int16), nx, ny, nz,
                               _ptr(np.asarray(sigma_xyz, np.float64)), float(fill), _ptr(q),
                               q.size, _ptr(out))
    return out
