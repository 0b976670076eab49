"""GPU parity of strip sharding: an image cut into G strips, each labelled by
``ccl_strip_begin`` / ``ccl_strip_finish`` on its own workspace and joined by
``ccl_strip_resolve``, must give the oracle's labels of the whole image bit
for bit.  Cases: ragged widths and a ragged last strip, both connectivities,
components that cross every seam (comb, spiral), the 8192x8192 Bernoulli(0.5)
image in 4 strips, pitched input, argument errors, and the same path run by
two processes that exchange their edge rows through gloo."""
import os
import socket

import numpy as np
import pytest

import oracle
from paper_1712_09789_gb300 import ccl, strips, synth

pytestmark = pytest.mark.gpu


def _torch():
    import torch

    return torch


def run_strips(img: np.ndarray, G: int, conn: int) -> np.ndarray:
    torch = _torch()
    d = torch.from_numpy(np.ascontiguousarray(img)).cuda()
    lab = strips.label_strips_one_gpu(d, G, conn)
    assert ccl.ccl_get_device_status() == ccl.CCL_OK
    return lab.cpu().numpy()


def assert_strip_parity(img, G, conn, tag=""):
    got = run_strips(img, G, conn)
    want = oracle.label(img, conn)
    if not np.array_equal(got, want):
        bad = np.argwhere(got != want)
        y, x = bad[0]
        raise AssertionError(f"{tag} G={G} conn={conn} shape={img.shape}: {len(bad)} mismatches, "
                             f"first at (y={y}, x={x}) got {got[y, x]} want {want[y, x]}")


@pytest.mark.parametrize("conn", [4, 8])
@pytest.mark.parametrize("H,W,G", [(128, 1, 2), (300, 97, 2), (300, 97, 5), (1000, 1500, 3), (1000, 1500, 7),
                                   (640, 4100, 4)])
@pytest.mark.parametrize("p", [0.3, 0.5, 0.8])
def test_bernoulli_strips(conn, H, W, G, p):
    assert_strip_parity(synth.bernoulli(H, W, p, 7), G, conn, f"bernoulli p={p}")


@pytest.mark.parametrize("conn", [4, 8])
def test_components_crossing_every_seam(conn):
    assert_strip_parity(synth.comb(2048, 1031), 8, conn, "comb")
    assert_strip_parity(synth.spiral(1025), 4, conn, "spiral")
    assert_strip_parity(synth.smoothed(1536, 1536, 8.0, 0.5, 3), 6, conn, "smoothed")


def test_seam_only_contacts():
    img = np.zeros((192, 600), dtype=np.uint8)
    img[63, 5] = img[64, 6] = 1          # diagonal across the first seam
    img[127, 520] = img[128, 520] = 1    # vertical across the second, in the second block column
    img[63, 511] = img[64, 512] = 1      # diagonal across a seam and a block-column edge at once
    for conn in (4, 8):
        assert_strip_parity(img, 3, conn, "seam contacts")


def test_full_size_bernoulli_in_four_strips():
    img = synth.bernoulli(8192, 8192, 0.5, 0)
    assert_strip_parity(img, 4, 8, "8192^2")


def test_pitched_input():
    torch = _torch()
    base = synth.bernoulli(384, 208, 0.5, 5)
    wide = torch.zeros((384, 256), dtype=torch.uint8, device="cuda")
    wide[:, :208] = torch.from_numpy(base).cuda()
    lab = strips.label_strips_one_gpu(wide[:, :208], 3, 8)
    np.testing.assert_array_equal(lab.cpu().numpy(), oracle.label(base, 8))


def test_argument_errors():
    torch = _torch()
    img = torch.zeros((256, 64), dtype=torch.uint8, device="cuda")
    ws = torch.empty(ccl.ccl_workspace_size(256, 64, 8), dtype=torch.uint8, device="cuda")
    for y0, h, H_total in ((32, 64, 256),    # off the 64-row grid
                           (0, 100, 256),    # a strip before the last with a ragged height
                           (192, 128, 256)):  # past the end of the image
        with pytest.raises(ccl.CclError) as e:
            ccl.ccl_strip_begin(img[:h], y0, H_total, ws, 8)
        assert e.value.status == ccl.CCL_ERR_INVALID_ARG
    small = torch.empty(256, dtype=torch.uint8, device="cuda")
    with pytest.raises(ccl.CclError):
        ccl.ccl_strip_begin(img[:128], 0, 256, small, 8)


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    import torch
    import torch.distributed as dist

    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        img = synth.bernoulli(700, 900, 0.5, 11)
        y0, h = strips.strip_bounds(700, world)[rank]
        d = torch.from_numpy(np.ascontiguousarray(img[y0:y0 + h])).cuda()
        lab = strips.label_strip(d, y0, 700, 8)
        status = ccl.ccl_get_device_status()
        out[rank] = (status, lab.cpu().numpy())
        dist.barrier()
    finally:
        dist.destroy_process_group()


def test_two_processes_exchange_edges_through_gloo():
    # both processes label their strip on the same GPU; nothing on the device
    # waits for the other process: the exchange is a host-side all-gather
    import torch.multiprocessing as mp

    with mp.Manager() as m:
        out = m.dict()
        mp.spawn(_rank, args=(2, _free_port(), out), nprocs=2, join=True)
        res = dict(out)
    assert res[0][0] == ccl.CCL_OK and res[1][0] == ccl.CCL_OK
    got = np.concatenate([res[0][1], res[1][1]])
    np.testing.assert_array_equal(got, oracle.label(synth.bernoulli(700, 900, 0.5, 11), 8))
