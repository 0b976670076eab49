"""Host side of strip sharding (Sec. 3.2's boundary analysis at strip seams),
on the CPU: every strip is labelled alone by the oracle, its edge rows are
gathered, the library's seam union (``ccl_strip_resolve``, host code) joins
them, and the joined labels must equal the oracle's labels of the whole image.
The exchange itself runs as two gloo ranks through ``strips.gather_edges``,
the function the GPU path uses."""
import os
import socket

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

import oracle
from paper_1712_09789_gb300 import ccl, strips, synth

BG = np.uint32(0xFFFFFFFF)


def strip_keys(img, y0, h, conn):
    """Oracle labels of rows [y0, y0 + h) labelled alone, as raster positions
    of the whole image (the smallest position of each component within the
    strip); BG for background."""
    W = img.shape[1]
    lab = oracle.label(np.ascontiguousarray(img[y0:y0 + h]), conn).astype(np.int64)
    return np.where(lab > 0, lab - 1 + y0 * W, 0xFFFFFFFF).astype(np.uint32)


def edge_rows(keys):
    return np.stack([keys[0], keys[-1]])


def apply_map(keys, pairs):
    """Labels of a strip from its keys and the resolved (key, smallest key) pairs."""
    out = keys.astype(np.int64)
    fg = keys != BG
    if len(pairs):
        idx = np.searchsorted(pairs[:, 0], keys)
        idx = np.minimum(idx, len(pairs) - 1)
        hit = fg & (pairs[idx, 0] == keys)
        out = np.where(hit, pairs[idx, 1].astype(np.int64), out)
    return np.where(fg, out + 1, 0).astype(np.int32)


def join_on_host(img, G, conn):
    bounds = strips.strip_bounds(img.shape[0], G)
    keys = [strip_keys(img, y0, h, conn) for y0, h in bounds]
    pairs = ccl.ccl_strip_resolve(np.stack([edge_rows(k) for k in keys]), conn)
    return np.concatenate([apply_map(k, pairs) for k in keys]), pairs


def _images():
    seam = np.zeros((192, 40), dtype=np.uint8)
    seam[63, 5] = seam[64, 6] = 1          # diagonal contact across the first seam
    seam[127, 20] = seam[128, 20] = 1      # vertical contact across the second
    u = np.zeros((192, 48), dtype=np.uint8)
    u[:70, 3] = u[:70, 40] = 1             # two bars of strip 0 ...
    u[69, 3:41] = 1                        # ... joined only inside strip 1
    return {
        "bernoulli_300x97": synth.bernoulli(300, 97, 0.5, 1),
        "bernoulli_256x130_p07": synth.bernoulli(256, 130, 0.7, 2),
        "comb_320x61": synth.comb(320, 61),
        "spiral_257": synth.spiral(257),
        "seam_contacts": seam,
        "u_through_lower_strip": u,
        "empty_192x50": np.zeros((192, 50), dtype=np.uint8),
        "full_200x33": np.ones((200, 33), dtype=np.uint8),
    }


IMAGES = _images()


@pytest.mark.parametrize("name", sorted(IMAGES))
@pytest.mark.parametrize("conn", [4, 8])
@pytest.mark.parametrize("G", [2, 3])
def test_seam_union_matches_oracle(name, conn, G):
    img = IMAGES[name]
    got, pairs = join_on_host(img, G, conn)
    np.testing.assert_array_equal(got, oracle.label(img, conn))
    if len(pairs):
        assert np.all(np.diff(pairs[:, 0].astype(np.int64)) > 0)   # sorted, distinct keys
        assert np.all(pairs[:, 1] < pairs[:, 0])                    # always to a smaller key


def test_diagonal_seam_contact_needs_8_connectivity():
    img = IMAGES["seam_contacts"]
    _, p4 = join_on_host(img, 3, 4)
    _, p8 = join_on_host(img, 3, 8)
    W = img.shape[1]
    assert (64 * W + 6, 63 * W + 5) in {tuple(map(int, r)) for r in p8}
    assert (64 * W + 6, 63 * W + 5) not in {tuple(map(int, r)) for r in p4}
    assert (128 * W + 20, 127 * W + 20) in {tuple(map(int, r)) for r in p4}


def test_comb_joins_through_every_strip():
    # the comb is one component that crosses each seam many times; its parts
    # in the middle strips join only through the first and last strips
    img = IMAGES["comb_320x61"]
    got, pairs = join_on_host(img, 5, 8)
    assert len(np.unique(got[got > 0])) == 1 and got.max() == 1
    assert np.all(pairs[:, 1] == 0)


def test_strip_bounds_follow_the_block_grid():
    assert strips.strip_bounds(8192, 4) == [(0, 2048), (2048, 2048), (4096, 2048), (6144, 2048)]
    assert strips.strip_bounds(300, 3) == [(0, 128), (128, 128), (256, 44)]
    assert strips.strip_bounds(64, 1) == [(0, 64)]
    with pytest.raises(ValueError):
        strips.strip_bounds(100, 3)     # two block rows cannot make three strips


def test_resolve_sizes_its_output_and_rejects_bad_arguments():
    import ctypes

    edges = np.stack([edge_rows(strip_keys(IMAGES["full_200x33"], y0, h, 8))
                      for y0, h in strips.strip_bounds(200, 3)])
    lib = ccl.load()
    n = ctypes.c_size_t(0)
    assert lib.ccl_strip_resolve(edges.ctypes.data, 3, 33, 8, None, 0, ctypes.byref(n)) == ccl.CCL_ERR_INVALID_ARG
    assert n.value == 2          # strips 1 and 2 each join strip 0's one component
    assert lib.ccl_strip_resolve(edges.ctypes.data, 3, 33, 6, None, 0, ctypes.byref(n)) == ccl.CCL_ERR_INVALID_ARG
    assert lib.ccl_strip_resolve(edges.ctypes.data, 1, 33, 8, None, 0, ctypes.byref(n)) == ccl.CCL_OK
    assert n.value == 0          # one strip has no seam


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, name, conn, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        img = IMAGES[name]
        y0, h = strips.strip_bounds(img.shape[0], world)[rank]
        keys = strip_keys(img, y0, h, conn)
        mine = torch.from_numpy(edge_rows(keys).view(np.int32).copy())
        gathered = strips.gather_edges(mine)
        pairs = ccl.ccl_strip_resolve(gathered, conn)
        out[rank] = (y0, apply_map(keys, pairs), pairs)
        dist.barrier()
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("name,conn", [("bernoulli_300x97", 8), ("comb_320x61", 4), ("u_through_lower_strip", 8)])
def test_two_gloo_ranks_exchange_edges_and_agree(name, conn):
    with mp.Manager() as m:
        out = m.dict()
        mp.spawn(_rank, args=(2, _free_port(), name, conn, out), nprocs=2, join=True)
        res = dict(out)
    # both ranks resolved the same map from the same gathered rows
    np.testing.assert_array_equal(res[0][2], res[1][2])
    got = np.concatenate([res[0][1], res[1][1]])
    np.testing.assert_array_equal(got, oracle.label(IMAGES[name], conn))


@pytest.mark.parametrize("conn", [4, 8])
def test_seam_union_fuzz(conn):
    # many small random images: runs that meet at one column, runs that touch
    # two runs across the seam, strips whose edge rows are empty or full
    rng = np.random.default_rng(1234 + conn)
    for trial in range(60):
        H = int(rng.integers(65, 400))
        W = int(rng.integers(1, 90))
        p = float(rng.choice([0.05, 0.3, 0.5, 0.7, 0.95]))
        img = (rng.random((H, W)) < p).astype(np.uint8)
        G = int(rng.integers(2, (H + 63) // 64 + 1))
        got, _ = join_on_host(img, G, conn)
        np.testing.assert_array_equal(got, oracle.label(img, conn), err_msg=f"trial {trial} {H}x{W} p={p} G={G}")
