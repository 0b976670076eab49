"""GPU parity of the 3D labelling (``ccl_label_3d``) against the CPU oracle.

Labels are integers, so the bar is bit-exact equality.  Shapes span several
32 x 16 x 16 blocks with ragged tails in every axis and degenerate extents of
one; densities 0.1..0.9; structured volumes whose components cross every
block face (shells, a comb through all slices, smoothed blobs); padded row
pitches; the full-size 512^3 volumes; the closed forms at the int32 size
limit; and the failure-detection hook.
"""
import numpy as np
import pytest

import oracle
from paper_1712_09789_gb300 import ccl, synth

pytestmark = pytest.mark.gpu
CONNS3 = (6, 26)


def _torch():
    import torch

    return torch


def run_gpu(vol: np.ndarray, conn: int) -> np.ndarray:
    torch = _torch()
    d = torch.from_numpy(np.ascontiguousarray(vol)).cuda()
    lab = ccl.ccl_label_3d(d, conn)
    assert ccl.ccl_get_device_status() == ccl.CCL_OK
    return lab.cpu().numpy()


def assert_parity(vol, conn, tag=""):
    got = run_gpu(vol, conn)
    want = oracle.label3d(vol, conn)
    if not np.array_equal(got, want):
        bad = np.argwhere(got != want)
        z, y, x = bad[0]
        raise AssertionError(f"{tag} conn={conn} shape={vol.shape}: {len(bad)} mismatches, first at "
                             f"(x={x}, y={y}, z={z}): got {got[z, y, x]}, want {want[z, y, x]}")


@pytest.mark.parametrize("conn", CONNS3)
@pytest.mark.parametrize("shape", [(37, 45, 101), (16, 16, 32), (17, 33, 65), (1, 40, 70), (40, 1, 70),
                                   (40, 35, 1), (1, 1, 1), (3, 2, 200), (50, 17, 31)])
def test_random_ragged(conn, shape):
    for i, p in enumerate((0.1, 0.3, 0.5, 0.7, 0.9)):
        assert_parity(synth.bernoulli3d(*shape, p, 11 * i + shape[2]), conn, f"p={p}")


@pytest.mark.parametrize("conn", CONNS3)
def test_structured(conn):
    assert_parity(synth.shells(61), conn, "shells")
    assert_parity(synth.comb3d(35, 40, 100), conn, "comb3d")
    for sigma, dens in ((2.0, 0.3), (3.0, 0.5), (1.5, 0.7)):
        assert_parity(synth.smoothed3d(48, 64, 96, sigma, dens, 5), conn, f"smoothed {sigma} {dens}")


@pytest.mark.parametrize("conn", CONNS3)
def test_closed_forms(conn):
    shape = (33, 35, 70)
    assert not run_gpu(np.zeros(shape, np.uint8), conn).any()
    assert (run_gpu(np.ones(shape, np.uint8), conn) == 1).all()
    z, y, x = np.indices(shape)
    cb = ((x + y + z) % 2 == 0).astype(np.uint8)
    want = np.where(cb == 1, x + y * 70 + z * 70 * 35 + 1, 0) if conn == 6 else cb.astype(np.int32)
    np.testing.assert_array_equal(run_gpu(cb, conn), want)
    # a diagonal chain through block corners
    vol = np.zeros((40, 40, 40), np.uint8)
    for i in range(40):
        vol[i, i, i] = 1
    got = run_gpu(vol, conn)
    assert len(np.unique(got[got > 0])) == (1 if conn == 26 else 40)


def test_pitch_and_nonzero_bytes():
    torch = _torch()
    g = np.random.default_rng(2)
    base = (g.random((20, 18, 45)) < 0.45).astype(np.uint8)
    for pitch in (45, 48, 61, 64):
        padded = np.full((20, 18, pitch), 9, np.uint8)
        padded[:, :, :45] = base * np.uint8(200)
        dev = torch.from_numpy(padded).cuda()[:, :, :45]
        for conn in CONNS3:
            got = ccl.ccl_label_3d(dev, conn).cpu().numpy()
            np.testing.assert_array_equal(got, oracle.label3d(base, conn))


def test_empty_volumes_and_streams():
    torch = _torch()
    for shape in ((0, 5, 5), (5, 0, 5), (5, 5, 0)):
        out = ccl.ccl_label_3d(torch.zeros(shape, dtype=torch.uint8, device="cuda"), 6)
        assert tuple(out.shape) == shape
    vol = synth.bernoulli3d(30, 40, 90, 0.4, 3)
    dev = torch.from_numpy(vol).cuda()
    want = oracle.label3d(vol, 26)
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        lab = ccl.ccl_label_3d(dev, 26, stream=s)
    s.synchronize()
    np.testing.assert_array_equal(lab.cpu().numpy(), want)
    # a preallocated output is fully overwritten
    out = torch.full(vol.shape, 12345, dtype=torch.int32, device="cuda")
    ccl.ccl_label_3d(dev, 26, labels=out)
    np.testing.assert_array_equal(out.cpu().numpy(), want)


@pytest.mark.parametrize("conn,p", [(6, 0.3), (26, 0.5), (6, 0.5), (26, 0.1)])
def test_full_size_512(conn, p):
    """The benchmark volumes (512^3 Bernoulli), every voxel against the oracle."""
    vol = synth.bernoulli3d(512, 512, 512, p, 0)
    assert_parity(vol, conn, "512^3")


def test_maximum_size_closed_forms():
    """D*H*W = 2^31 - 2^20 voxels, close to the int32 limit: isolated dots
    (label = 1 + own position) and a full volume (label 1)."""
    torch = _torch()
    D, H, W = 1023, 1024, 2049
    assert D * H * W <= 2 ** 31 - 2
    vol = torch.zeros((D, H, W), dtype=torch.uint8, device="cuda")
    vol[::256, ::256, ::256] = 1
    lab = ccl.ccl_label_3d(vol, 6)
    assert ccl.ccl_get_device_status() == ccl.CCL_OK
    zs = torch.arange(0, D, 256, device="cuda", dtype=torch.int64)[:, None, None]
    ys = torch.arange(0, H, 256, device="cuda", dtype=torch.int64)[None, :, None]
    xs = torch.arange(0, W, 256, device="cuda", dtype=torch.int64)[None, None, :]
    assert bool((lab[::256, ::256, ::256].long() == xs + W * (ys + H * zs) + 1).all())
    assert int((lab != 0).sum()) == zs.numel() * ys.numel() * xs.numel()
    vol.fill_(1)
    ccl.ccl_label_3d(vol, 26, labels=lab)
    assert ccl.ccl_get_device_status() == ccl.CCL_OK
    assert bool((lab == 1).all())
    del lab, vol
    torch.cuda.empty_cache()


def test_iteration_cap_reports_timeout_without_hanging():
    """Failure detection: a cap of one iteration makes the union-find loops
    give up on a comb through every slice; the device error word reports it
    and the next call with the default cap is correct again."""
    torch = _torch()
    vol = synth.comb3d(64, 64, 256)
    dev = torch.from_numpy(vol).cuda()
    assert ccl.ccl_get_device_status() == ccl.CCL_OK
    ccl.ccl_debug_set_iteration_cap(1)
    try:
        ccl.ccl_label_3d(dev, 6)
        assert ccl.ccl_get_device_status() == ccl.CCL_ERR_DEVICE_TIMEOUT
    finally:
        ccl.ccl_debug_set_iteration_cap(0)
    assert ccl.ccl_get_device_status() == ccl.CCL_OK
    np.testing.assert_array_equal(ccl.ccl_label_3d(dev, 6).cpu().numpy(), oracle.label3d(vol, 6))
