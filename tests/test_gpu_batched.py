"""Batched path (ccl_label_batched): many images of uneven size in one
launch sequence of persistent kernels, replayed as a CUDA graph, with the
block shape picked by the autotuner.  Every image is compared bit-exactly
against the CPU oracle."""
import os

import numpy as np
import pytest

import oracle
from paper_1712_09789_gb300 import build as ccl_build
from paper_1712_09789_gb300 import ccl, synth


def _torch():
    import torch

    return torch


def uneven_batch(n, seed, lo=1, hi=700):
    g = np.random.default_rng(seed)
    out = []
    for i in range(n):
        H, W = int(g.integers(lo, hi + 1)), int(g.integers(lo, hi + 1))
        d = float(g.uniform(0.1, 0.9))
        kind = i % 3
        if kind == 0:
            img = synth.bernoulli(H, W, d, seed * 1000 + i)
        elif kind == 1 and min(H, W) >= 8:
            img = synth.smoothed(H, W, 3.0, d, seed * 1000 + i)
        else:
            img = synth.granular(H, W, d, int(g.integers(2, 6)), seed * 1000 + i)
        out.append(img)
    return out


def run_batched(imgs, conn, tile=None, stream=None):
    torch = _torch()
    pairs = []
    for img in imgs:
        d = torch.from_numpy(np.ascontiguousarray(img)).cuda()
        pairs.append((d, torch.full(img.shape, -5, dtype=torch.int32, device="cuda")))
    ccl.ccl_label_batched(pairs, conn, stream=stream, tile=tile)
    assert ccl.ccl_get_device_status(stream) == ccl.CCL_OK
    return [lab.cpu().numpy() for _, lab in pairs]


def check_all(imgs, outs, conn, tag):
    for i, (img, got) in enumerate(zip(imgs, outs)):
        want = oracle.label(img, conn)
        if not np.array_equal(got, want):
            bad = int((got != want).sum())
            raise AssertionError(f"{tag} image {i} shape={img.shape} conn={conn}: {bad} mismatches")


def test_batched_argument_checks_without_gpu():
    ccl_build.build()
    lib = ccl.load()
    arr = (ccl.CclImage * 2)()
    arr[0] = ccl.CclImage(0x1000, 0x900000, 4, 4, 4)
    arr[1] = ccl.CclImage(0x2000, 0x990000, 4, 8, 4)  # pitch < W
    assert lib.ccl_label_batched(arr, 2, 8, None) == ccl.CCL_ERR_INVALID_ARG
    assert lib.ccl_label_batched(arr, 1, 6, None) == ccl.CCL_ERR_INVALID_ARG
    assert lib.ccl_label_batched(None, 0, 8, None) == ccl.CCL_OK
    assert lib.ccl_label_batched_tile(arr, 1, 8, 99, None) == ccl.CCL_ERR_INVALID_ARG
    assert ccl.ccl_tile_names() == ["512x64", "256x64", "1024x32", "512x64x8", "512x64p", "256x32p"]


@pytest.mark.gpu
@pytest.mark.parametrize("conn", (4, 8))
@pytest.mark.parametrize("tile", (0, 1, 2, 3, 4, 5))
def test_uneven_batch_every_tile(conn, tile):
    imgs = uneven_batch(24, seed=tile * 10 + conn)
    imgs += [np.zeros((0, 7), np.uint8), np.ones((1, 1), np.uint8), synth.spiral(301),
             synth.comb(70, 1500), np.ones((513, 3), np.uint8)]
    outs = run_batched(imgs, conn, tile=tile)
    check_all(imgs, outs, conn, f"tile={tile}")


@pytest.mark.gpu
def test_graph_replay_and_capacity_growth():
    # several calls on one stream with batches that grow and shrink: ring
    # slots are reused, graphs are replayed and rebuilt on growth
    for k, (n, hi) in enumerate(((5, 200), (30, 400), (3, 100), (60, 900), (10, 300), (10, 300))):
        imgs = uneven_batch(n, seed=100 + k, hi=hi)
        conn = 8 if k % 2 == 0 else 4
        check_all(imgs, run_batched(imgs, conn, tile=0), conn, f"call {k}")


@pytest.mark.gpu
def test_pitched_views_and_stream():
    torch = _torch()
    g = np.random.default_rng(9)
    imgs, pairs = [], []
    for i in range(8):
        H, W = int(g.integers(10, 600)), int(g.integers(10, 600))
        img = synth.bernoulli(H, W, 0.45, 500 + i)
        off = int(g.integers(0, 5))
        buf = np.full((H, W + off + int(g.integers(0, 40))), 255, np.uint8)
        buf[:, off:off + W] = img
        dev = torch.from_numpy(buf).cuda()[:, off:off + W]
        imgs.append(img)
        pairs.append((dev, torch.empty((H, W), dtype=torch.int32, device="cuda")))
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        ccl.ccl_label_batched(pairs, 8, stream=s, tile=1)
    s.synchronize()
    check_all(imgs, [lab.cpu().numpy() for _, lab in pairs], 8, "pitched")


@pytest.mark.gpu
def test_autotune_and_cache(tmp_path, monkeypatch):
    monkeypatch.setenv("CCL_AUTOTUNE_CACHE", str(tmp_path / "tune.txt"))
    monkeypatch.delenv("CCL_TILE", raising=False)
    torch = _torch()
    imgs = uneven_batch(12, seed=77, lo=300, hi=900)
    pairs = [(torch.from_numpy(im).cuda(), torch.empty(im.shape, dtype=torch.int32, device="cuda"))
             for im in imgs]
    tile = ccl.ccl_autotune_batched(pairs, 8)
    assert 0 <= tile < len(ccl.ccl_tile_names())
    assert ccl.ccl_batched_tile(pairs, 8) == tile
    check_all(imgs, [lab.cpu().numpy() for _, lab in pairs], 8, "autotuned")
    assert (tmp_path / "tune.txt").read_text().strip().endswith(str(tile))
    # the automatic path uses the tuned shape
    for _, lab in pairs:
        lab.fill_(-1)
    ccl.ccl_label_batched(pairs, 8)
    check_all(imgs, [lab.cpu().numpy() for _, lab in pairs], 8, "auto")
    # an explicit override wins
    monkeypatch.setenv("CCL_TILE", "1024x32")
    assert ccl.ccl_batched_tile(pairs, 8) == 2


@pytest.mark.gpu
def test_uneven_256_batch_full_size():
    """The 256-image batch (H, W uniform in [64, 2048], density uniform in
    [0.2, 0.8], half Bernoulli, half smoothed noise), 8-connectivity."""
    imgs = synth.batch_uneven(256, seed=0)
    for tile in (0, 4, 5):
        outs = run_batched(imgs, 8, tile=tile)
        check_all(imgs, outs, 8, f"batch256 tile={tile}")
