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


def _row_mask(vol, y, z):
    """Bits x = 0..31 of row (y, z) of the first block."""
    return sum(1 << x for x in range(32) if vol[z, y, x])


def _runs(m):
    """(first, last) column of every run of the bit mask m, in order."""
    out, x = [], 0
    while x < 32:
        if (m >> x) & 1:
            s = x
            while x < 32 and (m >> x) & 1:
                x += 1
            out.append((s, x - 1))
        else:
            x += 1
    return out


def _pairs6(vol):
    """Refinement pairs of the first 32x16x16 block under 6-connectivity:
    every (run, run) contact with the row above or the row of the slice
    before, less one per run that has any (its parent link)."""
    n = 0
    for z in range(16):
        for y in range(16):
            m = _row_mask(vol, y, z)
            nbs = [_row_mask(vol, y - 1, z) if y else 0, _row_mask(vol, y, z - 1) if z else 0]
            for s, e in _runs(m):
                run = ((2 << e) - 1) ^ ((1 << s) - 1)
                ev = sum(len(_runs(run & mn)) for mn in nbs)
                n += max(ev - 1, 0)
    return n


def _pairs26(vol):
    """Refinement pairs of the first block under 26-connectivity: contacts of
    every piece of a 2x2 row bundle with the pieces of its four earlier
    bundles (one per pair of pieces)."""
    def rows(Y, Z):
        return [_row_mask(vol, 2 * Y + dy, 2 * Z + dz) for dz in (0, 1) for dy in (0, 1)]  # r0, r0+1, r0+16, r0+17

    n = 0
    for Z in range(8):
        for Y in range(8):
            b = rows(Y, Z)
            ob = b[0] | b[1] | b[2] | b[3]
            for k, (dY, dZ, own, nbf) in enumerate(((-1, 0, (0, 2), (1, 3)), (0, -1, (0, 1), (2, 3)),
                                                     (-1, -1, (0,), (3,)), (1, -1, (1,), (2,)))):
                if not (0 <= Y + dY < 8 and 0 <= Z + dZ < 8):
                    continue
                nb = rows(Y + dY, Z + dZ)
                on = nb[0] | nb[1] | nb[2] | nb[3]
                fo = 0
                for i in own:
                    fo |= b[i]
                fn = 0
                for i in nbf:
                    fn |= nb[i]
                for s, e in _runs(ob):
                    run = ((2 << e) - 1) ^ ((1 << s) - 1)
                    t = fo & run
                    c = (t | (t << 1) | (t >> 1)) & fn & 0xFFFFFFFF
                    n += sum(1 for ps, pe in _runs(on) if c & (((2 << pe) - 1) ^ ((1 << ps) - 1)))
    return n


@pytest.mark.parametrize("conn", CONNS3)
def test_refinement_list_overflow(conn):
    """Blocks with more refinement pairs than the shared candidate list holds
    (2048 per 32x16x16 block): the surplus is joined directly (6-connectivity)
    or by a second pass over the contacts (26-connectivity)."""
    D, H, W = 40, 40, 70
    z, y, x = np.indices((D, H, W))
    if conn == 6:
        # full rows beside rows of every other voxel, alternating in y and z:
        # a full row meets 16 runs above it and 16 in the slice before
        vol = np.where((y + z) % 2 == 0, 1, x % 2 == 0).astype(np.uint8)
        assert _pairs6(vol) > 2048
    else:
        # every other x: each bundle holds 16 one-voxel-wide pieces, each
        # touching the piece of its column in every earlier bundle
        vol = (x % 2 == 0).astype(np.uint8)
        assert _pairs26(vol) > 2048
    assert_parity(vol, conn, "list overflow")
