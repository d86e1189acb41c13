"""GPU parity of the forward warp (Sec. 4) against the FP64 oracle, through
the C ABI.  Small cases compare every voxel (several tiles, ragged x/y/z
tails, odd shapes, volumes mostly or entirely outside the input, int16
input); the full-size batched workload compares sampled voxels in the launch
configuration the benchmark times."""
import numpy as np
import pytest
import torch

from oracle import ref
from synth import workloads
from synth.params import AffineSpec
from synth.workloads import VolumeCase, make_case

import _gpu as G

pytestmark = pytest.mark.gpu


def _small_cases():
    rng = np.random.default_rng(1234)
    wild = AffineSpec(max_rot_deg=45.0, scale_range=(0.6, 1.6), max_shift_vox=4.0,
                      max_shear=0.25, reflect_prob=(0.3, 0.3, 0.3))
    shapes = [((37, 29, 23), (45, 21, 19)), ((8, 8, 8), (8, 8, 8)), ((1, 1, 1), (5, 3, 7)),
              ((64, 33, 17), (33, 65, 10)), ((16, 16, 40), (70, 9, 13))]
    cases = []
    for n, (si, so) in enumerate(shapes):
        dtype = "int16" if n == 3 else "float32"
        cases.append(make_case(si, so, seed=500 + n, dtype=dtype, spec=wild, noise_id=n))
    # Entirely outside the input: every voxel is fill (+ photometric + noise).
    far = make_case((20, 20, 20), (33, 7, 9), seed=600, noise_id=9)
    far.T = far.T.copy()
    far.T[:, 3] += np.float32(500.0)
    cases.append(far)
    return cases


@pytest.fixture(scope="module")
def small():
    return G.to_device(_small_cases())


@pytest.mark.parametrize("batched", [True, False])
def test_small_cases_match_oracle_every_voxel(small, batched):
    seed = 0x1234_5678_9ABC
    gi, gl = G.run_fwd(small, seed, batched=batched)
    for b, v in enumerate(small):
        img, lab, tie, _ = ref.warp_fwd(v, seed)
        G.check_image(gi[b], img, f"case {b}")
        G.check_labels(gl[b], lab, tie, f"case {b}")


def test_all_variants_agree_bitwise(small):
    A = G.aw()
    seed = 99
    base_i, base_l = G.run_fwd(small, seed, variant=0)
    for v in range(1, A.aug_num_variants(A.OP_FWD)):
        gi, gl = G.run_fwd(small, seed, variant=v)
        for b in range(len(small)):
            assert np.array_equal(gi[b], base_i[b]), (v, b)
            assert np.array_equal(gl[b], base_l[b]), (v, b)


def test_one_volume_launches_agree_bitwise(small):
    """The one-volume-per-launch form of every direct variant (flat or box
    tiles) gives the batched output bit for bit."""
    A = G.aw()
    seed = 99
    base_i, base_l = G.run_fwd(small, seed, variant=0)
    names = [A.aug_variant_name(A.OP_FWD, v) for v in range(A.aug_num_variants(A.OP_FWD))]
    direct = [v for v, nm in enumerate(names) if nm.startswith(("t32", "b8", "b16"))]
    assert any(names[v].startswith("b8") for v in direct)
    for v in direct:
        gi, gl = G.run_fwd(small, seed, batched=False, variant=v)
        for b in range(len(small)):
            assert np.array_equal(gi[b], base_i[b]), (names[v], b)
            assert np.array_equal(gl[b], base_l[b]), (names[v], b)


@pytest.mark.parametrize("dtype", ["float32", "int16"])
def test_identity_and_integer_shift_are_exact(dtype):
    from synth.phantom import make_phantom
    img, lab = make_phantom((41, 35, 18), seed=3, dtype=dtype, device="cuda")
    T = np.zeros((3, 4), np.float32)
    T[:, :3] = np.eye(3)
    ident = VolumeCase(image=img, label=lab, out_shape=(41, 35, 18), T=T)
    Ts = T.copy()
    Ts[:, 3] = (3, -2, 5)
    shift = VolumeCase(image=img, label=lab, out_shape=(30, 40, 20), T=Ts,
                       fill_image=np.float32(-7.0))
    gi, gl = G.run_fwd([ident, shift], seed=5)
    host = img.cpu().numpy().astype(np.float32)
    hl = lab.cpu().numpy()
    assert np.array_equal(gi[0], host) and np.array_equal(gl[0], hl)
    pad = 30
    big = np.pad(host, pad, constant_values=-7.0)
    bigl = np.pad(hl, pad, constant_values=0)
    sl = (slice(pad + 5, pad + 25), slice(pad - 2, pad + 38), slice(pad + 3, pad + 33))
    assert np.array_equal(gi[1], big[sl]) and np.array_equal(gl[1], bigl[sl])


def test_config0_full_grid():
    w = workloads.config0(device="cuda")
    gi, gl = G.run_fwd(w.vols, w.seed)
    img, lab, tie, nt = ref.warp_fwd(w.vols[0], w.seed)
    worst = G.check_image(gi[0], img, "config 0")
    ties, tie_mismatch = G.check_labels(gl[0], lab, tie, "config 0")
    print(f"config0: max err {worst:.2e} HU, label ties {ties} (mismatched {tie_mismatch})")


def test_config1_full_size_sampled():
    """The full batched workload (64 uneven volumes -> 120x120x160), one
    persistent launch as timed by the benchmark; 20k random voxels per volume
    checked against the oracle evaluated point by point."""
    w = workloads.config1(device="cuda")
    gi, gl = G.run_fwd(w.vols, w.seed)
    rng = np.random.default_rng(5)
    ties = 0
    for b, v in enumerate(w.vols):
        q = rng.integers(0, v.n_out, 20000)
        vals, labs, tie = ref.warp_fwd_points(v, w.seed, q)
        G.check_image(gi[b].reshape(-1)[q], vals, f"config1 vol {b}")
        t, _ = G.check_labels(gl[b].reshape(-1)[q], labs, tie, f"config1 vol {b}")
        ties += t
        assert np.all(np.isfinite(gi[b]))
    print(f"config1: sampled 64 x 20000 voxels, label ties {ties}")


def test_config1_full_grid_four_volumes():
    """Every voxel of four of the 64 volumes (the smallest and the largest
    inputs and two others) of the full batched launch against the oracle."""
    w = workloads.config1(device="cuda")
    gi, gl = G.run_fwd(w.vols, w.seed)
    sizes = [v.image.numel() for v in w.vols]
    pick = sorted({int(np.argmin(sizes)), int(np.argmax(sizes)), 17, 42})
    for b in pick:
        img, lab, tie, _ = ref.warp_fwd(w.vols[b], w.seed)
        G.check_image(gi[b], img, f"config1 vol {b}")
        G.check_labels(gl[b], lab, tie, f"config1 vol {b}")
    print(f"config1: every voxel of volumes {pick}")


def test_config4_int16_downscale_sampled():
    w = workloads.config4(device="cuda", n_vols=2)
    gi, gl = G.run_fwd(w.vols, w.seed)
    rng = np.random.default_rng(6)
    for b, v in enumerate(w.vols):
        q = rng.integers(0, v.n_out, 50000)
        vals, labs, tie = ref.warp_fwd_points(v, w.seed, q)
        G.check_image(gi[b].reshape(-1)[q], vals, f"config4 vol {b}")
        G.check_labels(gl[b].reshape(-1)[q], labs, tie, f"config4 vol {b}")


def test_philox_words_bitexact():
    A = G.aw()
    rng = np.random.default_rng(7)
    ctr = rng.integers(0, 2 ** 32, (1 << 20, 4), dtype=np.uint64).astype(np.uint32)
    seed = 0xDEADBEEF_0BADF00D
    dev = torch.from_numpy(ctr.view(np.int32)).cuda()
    got = A.aug_philox4x32_10(dev, seed).cpu().numpy().view(np.uint32)
    assert np.array_equal(got, ref.philox(ctr, seed))


def test_noise_stream_matches_oracle_and_moments():
    """a = 0, b = 0, sigma = 1 on a constant image: the output is the noise."""
    img = torch.zeros((8, 8, 8), dtype=torch.float32, device="cuda")
    T = np.zeros((3, 4), np.float32)
    T[:, :3] = np.eye(3)
    v = VolumeCase(image=img, label=None, out_shape=(256, 128, 130), T=T,
                   photo_a=np.float32(0.0), photo_b=np.float32(0.0), sigma=np.float32(1.0),
                   noise_id=3)
    gi, _ = G.run_fwd([v], seed=2024)
    z = gi[0].reshape(-1).astype(np.float64)
    q = np.arange(z.size, dtype=np.int64)
    zr = ref.noise(2024, 3, 256, 128, q)
    assert np.max(np.abs(z - zr)) < 2e-5
    n = z.size
    assert abs(z.mean()) < 5 / np.sqrt(n)
    assert abs(z.var() - 1) < 5 * np.sqrt(2 / n)


def test_bad_descriptor_is_reported_and_skipped():
    A = G.aw()
    cases = G.to_device([make_case((12, 12, 12), (10, 10, 10), seed=1),
                         make_case((12, 12, 12), (10, 10, 10), seed=2, noise_id=1)])
    batch, oi, ol = G.batch_for(cases)
    batch.h_descs["affine"][0][0] = np.nan
    batch.upload()
    ws = A.make_workspace(2)
    A.aug_warp_fwd(batch.d_descs, 2, 0, ws)
    st, bad = A.aug_read_device_status(ws)
    assert st == A.AUG_ERR_DESCRIPTOR and bad == 0
    assert torch.isnan(oi[0]).all()          # skipped
    img, _, _, _ = ref.warp_fwd(cases[1], 0)
    G.check_image(oi[1].cpu().numpy(), img)
    assert A.aug_read_device_status(ws)[0] == 0   # cleared
