"""GPU parity: the CUDA path, called through the C ABI, against the CPU oracle.

Labels are integers, so the bar is bit-exact equality.  Cases span several
32x128 tiles with ragged tails, the tiny exhaustive set, the paper-shaped
workloads at their full sizes (512x512; the 4096x4096 density sweep and
granular noise; the 8192x8192 structured stress images), odd pitches and
alignments, nonzero bytes other than 1, the maximum image size and the
failure-detection hook.
"""
import numpy as np
import pytest

import oracle
from paper_1712_09789_gb300 import ccl, synth

pytestmark = pytest.mark.gpu
CONNS = (4, 8)


def _torch():
    import torch

    return torch


def run_gpu(img: np.ndarray, conn: int) -> np.ndarray:
    torch = _torch()
    d = torch.from_numpy(np.ascontiguousarray(img)).cuda()
    lab = ccl.ccl_label(d, conn)
    assert ccl.ccl_get_device_status() == ccl.CCL_OK
    return lab.cpu().numpy()


def assert_parity(img, conn, tag=""):
    got = run_gpu(img, conn)
    want = oracle.label(img, conn)
    if not np.array_equal(got, want):
        bad = np.argwhere(got != want)
        y, x = bad[0]
        raise AssertionError(f"{tag} conn={conn} shape={img.shape}: {len(bad)} mismatches, "
                             f"first at (y={y}, x={x}) got {got[y, x]} want {want[y, x]}")


@pytest.mark.parametrize("conn", CONNS)
@pytest.mark.parametrize("H,W", [(1, 1), (1, 200), (200, 1), (31, 127), (32, 128), (33, 129),
                                 (64, 256), (65, 257), (100, 300), (257, 385), (96, 1000)])
@pytest.mark.parametrize("p", [0.1, 0.5, 0.9])
def test_random_ragged(conn, H, W, p):
    for seed in range(3):
        assert_parity(synth.bernoulli(H, W, p, seed), conn, f"bernoulli p={p} seed={seed}")


@pytest.mark.parametrize("conn", CONNS)
def test_exhaustive_tiny(conn):
    torch = _torch()
    for H, W in ((1, 4), (4, 1), (2, 3), (3, 3), (4, 4)):
        n = H * W
        codes = np.arange(2 ** n)
        imgs = ((codes[:, None] >> np.arange(n)[None, :]) & 1).astype(np.uint8).reshape(-1, H, W)
        want = np.stack([oracle.label(im, conn) for im in imgs])
        dev = torch.from_numpy(imgs).cuda()
        out = torch.empty((len(imgs), H, W), dtype=torch.int32, device="cuda")
        for i in range(len(imgs)):
            ccl.ccl_label(dev[i], conn, labels=out[i])
        assert ccl.ccl_get_device_status() == ccl.CCL_OK
        got = out.cpu().numpy()
        bad = np.nonzero((got != want).reshape(len(imgs), -1).any(1))[0]
        assert len(bad) == 0, f"{H}x{W} conn={conn}: image {bad[0]}\n{imgs[bad[0]]}\n{got[bad[0]]}"


@pytest.mark.parametrize("conn", CONNS)
def test_structured_medium(conn):
    for img, tag in ((synth.spiral(1001), "spiral"), (synth.rings(777), "rings"),
                     (synth.comb(300, 1025), "comb"), (synth.smoothed(700, 900, 8.0, 0.5, 1), "smoothed"),
                     (synth.granular(513, 700, 0.5, 4, 2), "granular4"),
                     (synth.granular(513, 700, 0.5, 16, 2), "granular16")):
        assert_parity(img, conn, tag)


@pytest.mark.parametrize("conn", CONNS)
def test_closed_forms(conn):
    for H, W in ((1, 1), (33, 129), (64, 512), (130, 260)):
        ys, xs = np.mgrid[:H, :W]
        cb = ((xs + ys) % 2 == 0).astype(np.uint8)
        got = run_gpu(cb, conn)
        if conn == 4:
            np.testing.assert_array_equal(got, np.where(cb == 1, ys * W + xs + 1, 0))
        else:
            np.testing.assert_array_equal(got, cb.astype(np.int32))
        np.testing.assert_array_equal(run_gpu(np.ones((H, W), np.uint8), conn), 1)
        np.testing.assert_array_equal(run_gpu(np.zeros((H, W), np.uint8), conn), 0)


def test_config_512_bernoulli():
    img = synth.bernoulli(512, 512, 0.5, 0)
    assert_parity(img, 8, "512 bernoulli 0.5 seed 0")
    assert_parity(img, 4, "512 bernoulli 0.5 seed 0")


@pytest.mark.parametrize("conn", CONNS)
def test_config_4096_set(conn):
    # every density and granularity of the 4096x4096 set at seed 0, plus
    # seeds 1 and 2 at density 0.5
    for name, img in synth.noise_4096_set(seeds=(0,)):
        assert_parity(img, conn, name)
    for s in (1, 2):
        assert_parity(synth.bernoulli(4096, 4096, 0.5, s), conn, f"bernoulli 0.5 seed {s}")


def test_config_8192_stress():
    for name, img in synth.stress_8192_set():
        assert_parity(img, 8, name)


def test_stress_closed_forms_8192():
    torch = _torch()
    lab = torch.from_numpy(run_gpu(synth.spiral(8192), 8))
    assert int(lab.max()) == 1
    lab = run_gpu(synth.rings(8192), 8)
    assert len(np.unique(lab[lab > 0])) == synth.ring_count(8192)
    lab = run_gpu(synth.comb(8192, 8192), 8)
    assert lab.max() == 1


@pytest.mark.parametrize("conn", CONNS)
def test_large_image_ragged(conn):
    """An image of at least 1024 blocks (single 8-connected images of that
    size run on lane tiles of 8 rows), with ragged tails in both directions."""
    for p, seed in ((0.5, 1), (0.3, 2)):
        assert_parity(synth.bernoulli(4100, 8200, p, seed), conn, f"large ragged p={p}")


def test_pitch_alignment_and_nonzero_bytes():
    torch = _torch()
    g = np.random.default_rng(7)
    base = (g.random((300, 517)) < 0.5).astype(np.uint8)
    vals = base * g.integers(1, 256, size=base.shape).astype(np.uint8)
    for pad_w, off in ((517, 0), (528, 0), (600, 3), (640, 16), (530, 1)):
        buf = np.full((300, pad_w + off), 255, np.uint8)
        buf[:, off:off + 517] = vals
        dev = torch.from_numpy(buf).cuda()[:, off:off + 517]
        assert dev.stride(0) == pad_w + off
        for conn in CONNS:
            got = ccl.ccl_label(dev, conn).cpu().numpy()
            np.testing.assert_array_equal(got, oracle.label(base, conn), err_msg=f"pad={pad_w} off={off}")


def test_workspace_variant_and_streams():
    torch = _torch()
    img = synth.bernoulli(1000, 777, 0.45, 3)
    want = oracle.label(img, 8)
    dev = torch.from_numpy(img).cuda()
    ws = torch.empty(ccl.ccl_workspace_size(1000, 777, 8), dtype=torch.uint8, device="cuda")
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        lab = ccl.ccl_label_ws(dev, ws, 8)
        lab2 = ccl.ccl_label(dev, 8)
    s.synchronize()
    np.testing.assert_array_equal(lab.cpu().numpy(), want)
    np.testing.assert_array_equal(lab2.cpu().numpy(), want)


def test_host_entry_point():
    img = synth.smoothed(999, 1234, 4.0, 0.4, 5)
    for conn in CONNS:
        np.testing.assert_array_equal(ccl.ccl_label_host(img, conn), oracle.label(img, conn))
    # a host view with a row pitch
    wide = np.zeros((999, 1300), np.uint8)
    wide[:, :1234] = img
    np.testing.assert_array_equal(ccl.ccl_label_host(wide[:, :1234], 8), oracle.label(img, 8))
    # page-locked label buffers: the write-out stores into them directly
    import torch

    for conn in CONNS:
        for shape in ((999, 1234), (640, 1024)):
            im = img[: shape[0], : shape[1]].copy()
            pinned = torch.full(shape, -7, dtype=torch.int32).pin_memory().numpy()
            out = ccl.ccl_label_host(im, conn, labels=pinned)
            assert out is pinned
            np.testing.assert_array_equal(pinned, oracle.label(im, conn))


def test_empty_images():
    torch = _torch()
    for shape in ((0, 5), (5, 0), (0, 0)):
        out = ccl.ccl_label(torch.zeros(shape, dtype=torch.uint8, device="cuda"), 8)
        assert tuple(out.shape) == shape


def test_maximum_size_closed_form():
    """H*W = 2^31 - 2^16 pixels, close to the int32 limit: a comb (one
    component, label 1) checked on the device against its closed form."""
    torch = _torch()
    H, W = 32767, 65536
    img = torch.zeros((H, W), dtype=torch.uint8, device="cuda")
    img[:, 0::2] = 1
    gaps = torch.arange(1, W - 1, 2, device="cuda")
    img[0, gaps[(gaps // 2) % 2 == 0]] = 1
    img[H - 1, gaps[(gaps // 2) % 2 == 1]] = 1
    lab = ccl.ccl_label(img, 8)
    assert ccl.ccl_get_device_status() == ccl.CCL_OK
    assert bool(((lab == 1) == (img == 1)).all()) and bool((lab[img == 0] == 0).all())
    # 4-connectivity on isolated dots of the same extent: 1 + own position
    del lab
    img.zero_()
    img[::1024, ::1024] = 1
    lab = ccl.ccl_label(img, 4)
    ys = torch.arange(0, H, 1024, device="cuda", dtype=torch.int64)[:, None]
    xs = torch.arange(0, W, 1024, device="cuda", dtype=torch.int64)[None, :]
    assert bool((lab[::1024, ::1024].long() == ys * W + xs + 1).all())
    assert int((lab != 0).sum()) == ys.numel() * xs.numel()
    del lab, img
    torch.cuda.empty_cache()


def test_iteration_cap_reports_timeout_without_hanging():
    """Failure detection: a cap of one iteration makes the union-find loops
    give up on a long spiral; the device error word reports it and the next
    call with the default cap is correct again."""
    torch = _torch()
    img = synth.spiral(1024)
    dev = torch.from_numpy(img).cuda()
    assert ccl.ccl_get_device_status() == ccl.CCL_OK
    ccl.ccl_debug_set_iteration_cap(1)
    try:
        ccl.ccl_label(dev, 8)
        assert ccl.ccl_get_device_status() == ccl.CCL_ERR_DEVICE_TIMEOUT
    finally:
        ccl.ccl_debug_set_iteration_cap(0)
    assert ccl.ccl_get_device_status() == ccl.CCL_OK
    np.testing.assert_array_equal(ccl.ccl_label(dev, 8).cpu().numpy(), oracle.label(img, 8))


@pytest.mark.gpu
@pytest.mark.parametrize("conn", (4, 8))
def test_blocks_with_a_piece_per_column(conn):
    """Under 4-connectivity a band whose columns meet only diagonally holds a
    piece per column (32 per band, the most a lane tile can hold).
    Checkerboard patches in a noise image put such blocks beside ordinary ones
    into one call (twice in a row) and into one batch."""
    import torch

    g = np.random.default_rng(77)
    img = (g.random((300, 2100)) < 0.5).astype(np.uint8)
    y, x = np.mgrid[0:300, 0:2100]
    cb = ((x + y) % 2 == 0).astype(np.uint8)
    for y0, x0 in ((0, 0), (64, 600), (130, 1536), (250, 1900)):
        img[y0:y0 + 70, x0:x0 + 300] = cb[y0:y0 + 70, x0:x0 + 300]
    want = oracle.label(img, conn)
    d = torch.from_numpy(img).cuda()
    for _ in range(2):
        got = ccl.ccl_label(d, conn).cpu().numpy()
        assert ccl.ccl_get_device_status() == ccl.CCL_OK
        np.testing.assert_array_equal(got, want)
    pairs = [(d, torch.empty(img.shape, dtype=torch.int32, device="cuda")),
             (torch.from_numpy(cb[:100, :700].copy()).cuda(), torch.empty((100, 700), dtype=torch.int32, device="cuda"))]
    ccl.ccl_label_batched(pairs, conn, tile=0)
    np.testing.assert_array_equal(pairs[0][1].cpu().numpy(), want)
    np.testing.assert_array_equal(pairs[1][1].cpu().numpy(), oracle.label(cb[:100, :700], conn))
