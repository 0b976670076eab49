"""Component statistics (ccl_component_stats) against the oracle's
per-component area, bounding box and coordinate sums, exact integers."""
import numpy as np
import pytest

import oracle
from paper_1712_09789_gb300 import ccl, synth


def _stats(img, conn):
    import torch

    lab = ccl.ccl_label(torch.from_numpy(np.ascontiguousarray(img)).cuda(), conn)
    got = ccl.ccl_component_stats(lab)
    want = oracle.component_stats(oracle.label(img, conn))
    return got, want


def _as_rows(st):
    return np.stack([st[f].astype(np.int64) for f in ("label", "area", "x0", "y0", "x1", "y1", "sum_x", "sum_y")],
                    axis=1) if st.size else np.zeros((0, 8), np.int64)


@pytest.mark.gpu
@pytest.mark.parametrize("conn", (4, 8))
def test_stats_match_the_oracle(conn):
    g = np.random.default_rng(5)
    imgs = [synth.bernoulli(int(g.integers(1, 400)), int(g.integers(1, 1500)), float(g.uniform(0.1, 0.9)), i)
            for i in range(5)]
    y, x = np.mgrid[0:70, 0:600]
    imgs += [synth.spiral(301), synth.comb(66, 700), np.ones((100, 1030), np.uint8), np.zeros((9, 9), np.uint8),
             ((x + y) % 2 == 0).astype(np.uint8), synth.smoothed(600, 900, 6.0, 0.5, 3)]
    for i, img in enumerate(imgs):
        got, want = _stats(img, conn)
        np.testing.assert_array_equal(_as_rows(got), want, err_msg=f"image {i} {img.shape}")


@pytest.mark.gpu
def test_stats_of_a_large_noise_image_and_capacity():
    import torch

    img = synth.bernoulli(2048, 2048, 0.5, 1)
    lab = ccl.ccl_label(torch.from_numpy(img).cuda(), 8)
    want = oracle.component_stats(oracle.label(img, 8))
    np.testing.assert_array_equal(_as_rows(ccl.ccl_component_stats(lab)), want)
    # too little room: the count is still the full count, the first records fill
    part = ccl.ccl_component_stats(lab, capacity=10)
    np.testing.assert_array_equal(_as_rows(part), want[:10])
    # labels that are not canonical are refused
    bad = lab.clone()
    bad[0, 0] = 12345678
    with pytest.raises(ccl.CclError) as e:
        ccl.ccl_component_stats(bad, capacity=4)
    assert e.value.status == ccl.CCL_ERR_INVALID_ARG
