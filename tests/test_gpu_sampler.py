"""GPU parity of the device-side parameter sampler (Sec. 4) with the FP64
oracle: every drawn descriptor field of a mixed batch (float32 results equal,
up to a last-bit difference of sin/cos counted and bounded), the draw counter
(each call and each CUDA-graph replay draws the next index), a graph of
sampler + forward whose every replay matches the oracle warp with the drawn
parameters, groups that are not drawn left as they were, and spec errors."""
import numpy as np
import pytest
import torch

from oracle import ref
from synth.workloads import make_case

import _gpu as G

pytestmark = pytest.mark.gpu

FULL = dict(rot_max=(0.3, 0.2, 0.26), scale_min=(0.9, 0.85, 0.9), scale_max=(1.1, 1.2, 1.1),
            reflect_prob=(0.5, 0.3, 0.1), shear_max=0.05, generic_max=0.02,
            extra_scale=(1.0, 1.0, 1.5), shift_max=(10.0, 8.0, 5.0), photo_a=(0.9, 1.1),
            photo_b=(-50.0, 50.0), sigma=(0.0, 50.0), window_lo=(-1000.0, -150.0),
            window_hi=(230.0, 1500.0), occ_max_frac=0.3)


def _batch(n, seed0=0):
    rng = np.random.default_rng(seed0)
    cases = []
    for b in range(n):
        si = tuple(int(v) for v in rng.integers(4, 40, 3))
        so = tuple(int(v) for v in rng.integers(3, 36, 3))
        cases.append(make_case(si, so, seed=seed0 + b, noise_id=int(rng.integers(0, 2 ** 32))))
    cases = G.to_device(cases)
    batch, oi, ol = G.batch_for(cases)
    return cases, batch, oi, ol


def _ulps(a, b):
    a = np.asarray(a, np.float32).reshape(-1)
    b = np.asarray(b, np.float32).reshape(-1)
    ia, ib = a.view(np.int32).astype(np.int64), b.view(np.int32).astype(np.int64)
    ia = np.where(ia < 0, -(ia & 0x7FFFFFFF), ia)
    ib = np.where(ib < 0, -(ib & 0x7FFFFFFF), ib)
    return np.abs(ia - ib)


def _expected(h, b, mask, seed, draw, before):
    d = h[b]
    return ref.sample_params(FULL, mask, seed, draw, int(d["noise_id"]),
                             (d["in_nx"], d["in_ny"], d["in_nz"]),
                             (d["out_nx"], d["out_ny"], d["out_nz"]),
                             T=before["affine"][b].reshape(3, 4),
                             photo=(before["photo_a"][b], before["photo_b"][b],
                                    before["noise_sigma"][b]),
                             flags=int(before["flags"][b]),
                             occ=(before["occ_z0"][b], before["occ_dz"][b]))


def _compare(h, b, e):
    d = h[b]
    worst = int(_ulps(d["affine"], e["T"]).max())
    for f, k in (("photo_a", "photo_a"), ("photo_b", "photo_b"), ("noise_sigma", "sigma"),
                 ("occ_z0", "occ_z0"), ("occ_dz", "occ_dz")):
        worst = max(worst, int(_ulps(d[f], e[k]).max()))
    assert int(d["flags"]) == e["flags"]
    return worst


@pytest.mark.parametrize("mask", [ref.DRAW_AFFINE | ref.DRAW_WINDOW | ref.DRAW_OCCLUDE,
                                  ref.DRAW_AFFINE | ref.DRAW_PHOTO, ref.DRAW_OCCLUDE])
def test_drawn_fields_match_oracle(mask):
    A = G.aw()
    cases, batch, _, _ = _batch(300, seed0=100 + mask)
    before = batch.h_descs.copy()
    seed, draw = 0xDEADBEEF12345678, (3 << 32) + 99
    A.aug_sample_params(batch.d_descs, batch.n, A.ParamSpec(**FULL, draw=mask), seed, draw)
    h = batch.download()
    worst, off = 0, 0
    for b in range(batch.n):
        w = _compare(h, b, _expected(h, b, mask, seed, draw, before))
        worst = max(worst, w)
        off += w > 0
    # Double-precision sin/cos may differ in the last bit; after rounding to
    # float32 that moves a result by at most one float32 ulp, and rarely.
    assert worst <= 1 and off <= 3, (worst, off)
    if not mask & ref.DRAW_AFFINE:
        assert np.array_equal(h["affine"], before["affine"])


def test_counter_advances_per_call_and_per_graph_replay():
    A = G.aw()
    cases, batch, _, _ = _batch(5, seed0=7)
    before = batch.h_descs.copy()
    spec = A.ParamSpec(**FULL, draw=A.AUG_DRAW_AFFINE)
    counter = torch.zeros(1, dtype=torch.int64, device="cuda")
    for expect in range(3):
        A.aug_sample_params(batch.d_descs, batch.n, spec, 5, draw=40, counter=counter)
        h = batch.download()
        for b in range(batch.n):
            assert _compare(h, b, _expected(h, b, 1, 5, 40 + expect, before)) <= 1
    assert int(counter.item()) == 3
    stream = torch.cuda.Stream()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.stream(stream):
        with torch.cuda.graph(g, stream=stream):
            A.aug_sample_params(batch.d_descs, batch.n, spec, 5, draw=40, counter=counter)
    torch.cuda.synchronize()
    assert int(counter.item()) == 3       # capture does not run the kernel
    for expect in range(3, 6):
        with torch.cuda.stream(stream):
            g.replay()
        torch.cuda.synchronize()
        h = batch.download()
        for b in range(batch.n):
            assert _compare(h, b, _expected(h, b, 1, 5, 40 + expect, before)) <= 1
    assert int(counter.item()) == 6


def test_graph_of_sampler_and_forward_matches_oracle_every_replay():
    A = G.aw()
    cases, batch, oi, ol = _batch(6, seed0=31)
    spec = A.ParamSpec(**FULL, draw=A.AUG_DRAW_AFFINE | A.AUG_DRAW_WINDOW | A.AUG_DRAW_OCCLUDE)
    ws = A.make_workspace(batch.n)
    counter = torch.zeros(1, dtype=torch.int64, device="cuda")
    stream = torch.cuda.Stream()
    with torch.cuda.stream(stream):
        A.aug_warp_fwd(batch.d_descs, batch.n, 11, ws)     # first call outside capture
        torch.cuda.synchronize()
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g, stream=stream):
            A.aug_sample_params(batch.d_descs, batch.n, spec, 21, counter=counter)
            A.aug_warp_fwd(batch.d_descs, batch.n, 11, ws)
    for rep in range(3):
        with torch.cuda.stream(stream):
            g.replay()
        torch.cuda.synchronize()
        assert A.aug_read_device_status(ws)[0] == 0
        h = batch.download()
        for b, v in enumerate(cases):
            d = h[b]
            v.T = d["affine"].reshape(3, 4).copy()
            v.photo_a, v.photo_b, v.sigma = d["photo_a"], d["photo_b"], d["noise_sigma"]
            v.flags, v.occ_z0, v.occ_dz = int(d["flags"]), d["occ_z0"], d["occ_dz"]
            img, lab, tie, _ = ref.warp_fwd(v, 11)
            G.check_image(oi[b].cpu().numpy(), img, f"replay {rep} vol {b}",
                          tol=G.IMG_TOL * float(v.photo_a))
            G.check_labels(ol[b].cpu().numpy(), lab, tie)
    assert int(counter.item()) == 3


def test_spec_errors():
    A = G.aw()
    cases, batch, _, _ = _batch(2, seed0=3)
    bad = [dict(rot_max=(-0.1, 0.0, 0.0)), dict(scale_min=(0.0, 1.0, 1.0)),
           dict(scale_min=(1.2, 1.0, 1.0), scale_max=(1.1, 1.0, 1.0)),
           dict(reflect_prob=(1.5, 0.0, 0.0)), dict(window_lo=(-10.0, 300.0)),
           dict(occ_max_frac=1.5), dict(shear_max=float("nan")), dict(draw=16),
           dict(sigma=(-1.0, 0.0))]
    for kw in bad:
        with pytest.raises(A.AugError) as e:
            A.aug_sample_params(batch.d_descs, batch.n, A.ParamSpec(**{**FULL, **kw}), 1)
        assert e.value.status == A.AUG_ERR_INVALID_ARG, kw
