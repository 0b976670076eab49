"""Coarse-labelling variants of Sec. 4.2 (C2FL, RC2FL, CC2FL, NC2FL): the
coarse labelling only changes how much merging the refinement has to do, so
every variant must give the canonical labels of the oracle, and the counters
must show the refinement doing more work as coarse labelling is removed."""
import numpy as np
import pytest

import oracle
from paper_1712_09789_gb300 import ccl, synth


def _run(img, conn, variant, counters=False):
    import torch

    d = torch.from_numpy(np.ascontiguousarray(img)).cuda()
    out = ccl.ccl_label_variant(d, conn, variant, counters=counters)
    assert ccl.ccl_get_device_status() == ccl.CCL_OK
    if counters:
        lab, cnt = out
        return lab.cpu().numpy(), cnt
    return out.cpu().numpy()


@pytest.mark.gpu
@pytest.mark.parametrize("conn", (4, 8))
@pytest.mark.parametrize("variant", (0, 1, 2, 3))
def test_every_variant_is_exact(conn, variant):
    g = np.random.default_rng(100 + variant)
    imgs = [synth.bernoulli(int(g.integers(1, 300)), int(g.integers(1, 1400)), float(g.uniform(0.1, 0.9)), i)
            for i in range(6)]
    imgs += [synth.spiral(257), synth.comb(70, 1100), np.ones((65, 513), np.uint8),
             synth.granular(300, 700, 0.5, 4, 3)]
    y, x = np.mgrid[0:64, 0:512]
    imgs += [((x + y) % 2 == 0).astype(np.uint8), ((x // 2 + y) % 2 == 0).astype(np.uint8)]
    for i, img in enumerate(imgs):
        got = _run(img, conn, variant)
        want = oracle.label(img, conn)
        assert np.array_equal(got, want), f"variant {variant} conn {conn} image {i} {img.shape}"


@pytest.mark.gpu
@pytest.mark.parametrize("conn", (4, 8))
def test_refinement_work_grows_without_coarse_labelling(conn):
    img = synth.bernoulli(1024, 1024, 0.5, 0)
    counts = [_run(img, conn, v, counters=True)[1] for v in range(4)]
    merges = [c["merges"] for c in counts]
    # C2FL merges least; dropping coarse labelling along columns (RC2FL) or
    # along rows (CC2FL), or both (NC2FL), leaves more to the refinement
    assert merges[0] < merges[1] <= merges[3]
    assert merges[0] < merges[2] <= merges[3]
    assert all(c["find_steps"] >= c["merges"] for c in counts)
