"""Host logic of bench.py without a GPU: kernel variants given by index or by
name, the kernel each forward variant launches (the label of the roofline
objects), and the profile record lookup keyed by source hash and variant."""
import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)


@pytest.fixture(scope="module")
def aw():
    from paper_1811_11226_b300 import build
    build.build()
    from paper_1811_11226_b300 import augwarp
    return augwarp


def test_variant_index_by_index_and_name(aw):
    import bench
    for op in (aw.OP_FWD, aw.OP_BWD, aw.OP_IOU):
        n = aw.aug_num_variants(op)
        assert n >= 2
        for v in range(n):
            assert bench.variant_index(aw, op, str(v)) == v
            assert bench.variant_index(aw, op, aw.aug_variant_name(op, v)) == v
        assert bench.variant_index(aw, op, "-1") == -1
        with pytest.raises(SystemExit):
            bench.variant_index(aw, op, "no_such_variant")


def test_every_forward_variant_names_a_kernel(aw):
    import bench
    kinds = set()
    for v in range(aw.aug_num_variants(aw.OP_FWD)):
        name = aw.aug_variant_name(aw.OP_FWD, v)
        k = bench.fwd_kernel_name(name)
        assert k in ("k_fwd_batched", "k_fwd_batched_box", "k_fwd_brick", "k_fwd_brick_bulk"), name
        kinds.add(k)
        if name.startswith("t32"):
            assert k == "k_fwd_batched"
    assert kinds == {"k_fwd_batched", "k_fwd_batched_box", "k_fwd_brick", "k_fwd_brick_bulk"}
    default = aw.aug_variant_name(aw.OP_FWD, aw.aug_get_variant(aw.OP_FWD))
    assert bench.fwd_kernel_name(default) == "k_fwd_batched_box"


def test_profile_record_is_keyed_by_variant_and_source_hash(aw):
    import re
    import bench
    text = open(os.path.join(ROOT, "profiles", "fwd_batched_config1.md")).read()
    rec_hash = re.search(r"^- csrc_hash: (\w+)", text, re.M).group(1)
    rec_variant = re.search(r"^- variant: (\w+)", text, re.M).group(1)
    traffic = bench.profile_traffic("fwd_batched_config1", rec_variant)
    inst = bench.profile_record("fwd_batched_config1", "warp_inst_per_launch", rec_variant)
    if rec_hash == bench.kernel_source_hash():
        # A record of the current sources is used, with plausible figures.
        assert traffic is not None and traffic > 1.0e9
        assert inst is not None and inst > 1.0e8
    else:
        # A record of other sources is never used.
        assert traffic is None and inst is None
    # Nor is a record of another variant.
    other = next(aw.aug_variant_name(aw.OP_FWD, v) for v in range(aw.aug_num_variants(aw.OP_FWD))
                 if aw.aug_variant_name(aw.OP_FWD, v) != rec_variant)
    assert bench.profile_traffic("fwd_batched_config1", other) is None
