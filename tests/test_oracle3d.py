"""Pins of the 3D oracle (6- and 26-connectivity, raster position
x + y*W + z*W*H), each against something other than the oracle itself:
exhaustive enumeration against pure-Python min-propagation and the flood
fill, a library routine (scipy.ndimage.label) for the partition, the 2D
oracle on volumes that are really images, closed forms and invariants."""
import numpy as np
import pytest

import oracle
from paper_1712_09789_gb300 import synth

CONNS3 = (6, 26)
TO_2D = {6: 4, 26: 8}


def all_volumes(D, H, W):
    n = D * H * W
    bits = ((np.arange(2 ** n)[:, None] >> np.arange(n)[None, :]) & 1).astype(np.uint8)
    return bits.reshape(-1, D, H, W)


def canonical_from_partition(lab):
    """Relabel any partition (0 = background) into 1 + min raster index."""
    flat = lab.ravel()
    out = np.zeros(flat.shape, dtype=np.int32)
    if not (flat > 0).any():
        return out.reshape(lab.shape)
    order = np.argsort(flat, kind="stable")
    f = flat[order]
    start = np.searchsorted(f, f, side="left")
    first = order[start]  # smallest raster index of each value (stable sort)
    out[order] = np.where(f > 0, first + 1, 0)
    return out.reshape(lab.shape)


def n_components(lab):
    return len(np.unique(lab[lab > 0]))


# --- exhaustive ---------------------------------------------------------------

@pytest.mark.parametrize("conn", CONNS3)
@pytest.mark.parametrize("shape", [(2, 2, 2), (1, 3, 3), (2, 2, 3), (3, 2, 2), (2, 3, 2)])
def test_exhaustive_vs_closure_and_bfs(conn, shape):
    for vol in all_volumes(*shape):
        want = oracle.label3d_closure(vol, conn)
        np.testing.assert_array_equal(oracle.label3d_two_pass(vol, conn), want)
        np.testing.assert_array_equal(oracle.label3d_bfs(vol, conn), want)


# --- library routine ------------------------------------------------------------

@pytest.mark.parametrize("conn", CONNS3)
def test_scipy_partition_random(conn):
    ndi = pytest.importorskip("scipy.ndimage")
    structure = ndi.generate_binary_structure(3, 1 if conn == 6 else 3)
    for k in range(1, 10):
        for seed in range(0, 30, 7):
            vol = synth.bernoulli3d(11, 13, 37, k / 10, seed)
            lab_sp, _ = ndi.label(vol, structure=structure)
            np.testing.assert_array_equal(oracle.label3d(vol, conn), canonical_from_partition(lab_sp))
    vol = synth.smoothed3d(24, 20, 40, 2.0, 0.4, 1)
    lab_sp, _ = ndi.label(vol, structure=structure)
    np.testing.assert_array_equal(oracle.label3d(vol, conn), canonical_from_partition(lab_sp))


def test_canonical_helper_on_known_partition():
    lab = np.array([[[0, 5, 5], [7, 0, 5]]])
    np.testing.assert_array_equal(canonical_from_partition(lab), [[[0, 2, 2], [4, 0, 2]]])


# --- reductions to 2D -------------------------------------------------------------

@pytest.mark.parametrize("conn", CONNS3)
def test_volume_of_one_slice_row_or_column_is_an_image(conn):
    for seed in range(6):
        img = synth.bernoulli(19, 23, 0.3 + 0.08 * seed, seed)
        want = oracle.label(img, TO_2D[conn])
        # one slice: positions x + y*W
        np.testing.assert_array_equal(oracle.label3d(img[None], conn)[0], want)
        # one row per slice: positions x + z*W
        np.testing.assert_array_equal(oracle.label3d(img[:, None, :], conn)[:, 0, :], want)
        # one column per slice: positions y + z*H
        np.testing.assert_array_equal(oracle.label3d(img[:, :, None], conn)[:, :, 0], want)


@pytest.mark.parametrize("conn", CONNS3)
def test_stacked_identical_slices(conn):
    """Every slice equal to one image: the components are the image's (4- or
    8-connected) components extruded, and their minimum lies in slice 0."""
    img = synth.bernoulli(17, 29, 0.45, 3)
    vol = np.repeat(img[None], 5, axis=0)
    want = oracle.label(img, TO_2D[conn])
    lab = oracle.label3d(vol, conn)
    for z in range(5):
        np.testing.assert_array_equal(lab[z], want)


# --- closed forms --------------------------------------------------------------------

@pytest.mark.parametrize("conn", CONNS3)
@pytest.mark.parametrize("shape", [(1, 1, 1), (3, 4, 5), (7, 1, 9), (4, 6, 1)])
def test_empty_and_full(conn, shape):
    assert not oracle.label3d(np.zeros(shape, np.uint8), conn).any()
    assert (oracle.label3d(np.ones(shape, np.uint8), conn) == 1).all()


@pytest.mark.parametrize("shape", [(2, 2, 2), (3, 5, 4), (6, 7, 9)])
def test_checkerboard(shape):
    D, H, W = shape
    z, y, x = np.indices(shape)
    vol = ((x + y + z) % 2 == 0).astype(np.uint8)
    idx = x + y * W + z * W * H
    # 6-connectivity: no two foreground voxels are face neighbours
    np.testing.assert_array_equal(oracle.label3d(vol, 6), np.where(vol == 1, idx + 1, 0))
    # 26-connectivity: edge diagonals join every foreground voxel to voxel 0
    np.testing.assert_array_equal(oracle.label3d(vol, 26), vol.astype(np.int32))


@pytest.mark.parametrize("conn", CONNS3)
def test_isolated_voxels(conn):
    shape = (7, 8, 9)
    z, y, x = np.indices(shape)
    vol = ((x % 2 == 0) & (y % 2 == 0) & (z % 2 == 0)).astype(np.uint8)
    idx = x + y * 9 + z * 72
    np.testing.assert_array_equal(oracle.label3d(vol, conn), np.where(vol == 1, idx + 1, 0))


@pytest.mark.parametrize("conn", CONNS3)
@pytest.mark.parametrize("N", [1, 4, 7, 16, 23])
def test_shells_count(conn, N):
    lab = oracle.label3d(synth.shells(N), conn)
    assert n_components(lab) == synth.ring_count(N)


@pytest.mark.parametrize("conn", CONNS3)
def test_comb3d_is_one_component(conn):
    lab = oracle.label3d(synth.comb3d(5, 9, 14), conn)
    assert n_components(lab) == 1 and lab[0, 0, 0] == 1


def test_diagonal_chain_needs_26():
    """Voxels (i, i, i): corner neighbours only."""
    vol = np.zeros((4, 4, 4), np.uint8)
    for i in range(4):
        vol[i, i, i] = 1
    assert n_components(oracle.label3d(vol, 26)) == 1
    assert n_components(oracle.label3d(vol, 6)) == 4


def test_u_shape_through_slices_takes_the_late_minimum():
    """Two towers joined only in the last slice: the label of both is the
    smaller of their first voxels, which the raster scan meets in slice 0."""
    vol = np.zeros((4, 3, 5), np.uint8)
    vol[:, 1, 1] = 1
    vol[:, 1, 3] = 1
    vol[3, 1, 1:4] = 1
    for conn in CONNS3:
        lab = oracle.label3d(vol, conn)
        assert set(np.unique(lab)) == {0, 1 + 5 * 1 + 1}


# --- invariants --------------------------------------------------------------------------

@pytest.mark.parametrize("conn", CONNS3)
def test_invariants(conn):
    for seed in range(4):
        vol = synth.bernoulli3d(9, 10, 12, 0.25 + 0.1 * seed, seed)
        lab = oracle.label3d(vol, conn)
        n = n_components(lab)
        # the root voxel carries its own label
        flat = lab.ravel()
        v = flat[flat > 0]
        assert (flat[v - 1] == v).all()
        # flips and axis permutations keep the component count
        for ax in range(3):
            assert n_components(oracle.label3d(np.ascontiguousarray(np.flip(vol, ax)), conn)) == n
        for perm in ((0, 2, 1), (1, 0, 2), (2, 1, 0), (1, 2, 0)):
            assert n_components(oracle.label3d(np.ascontiguousarray(vol.transpose(perm)), conn)) == n
        # idempotence
        np.testing.assert_array_equal(oracle.label3d((lab > 0).astype(np.uint8), conn), lab)
    # the 6-connected partition refines the 26-connected one
    vol = synth.bernoulli3d(10, 11, 12, 0.3, 7)
    l6, l26 = oracle.label3d(vol, 6), oracle.label3d(vol, 26)
    for v in np.unique(l6[l6 > 0]):
        assert len(np.unique(l26[l6 == v])) == 1


def test_pitch_and_nonzero_bytes():
    g = np.random.default_rng(5)
    base = (g.random((5, 6, 21)) < 0.5).astype(np.uint8)
    padded = np.full((5, 6, 32), 7, np.uint8)
    padded[:, :, :21] = base * g.integers(1, 256, base.shape, dtype=np.uint8).clip(1)
    for conn in CONNS3:
        want = oracle.label3d_closure(base, conn)
        np.testing.assert_array_equal(oracle.label3d_two_pass(padded[:, :, :21], conn), want)
        np.testing.assert_array_equal(oracle.label3d_bfs(padded[:, :, :21], conn), want)


def test_rejects_bad_arguments():
    vol = np.zeros((2, 2, 2), np.uint8)
    for conn in (4, 8, 18, 0):
        with pytest.raises(ValueError):
            oracle.label3d(vol, conn)
    with pytest.raises(ValueError):
        oracle.label3d(np.zeros((2, 2), np.uint8), 6)
    assert oracle.label3d(np.zeros((0, 3, 3), np.uint8), 6).shape == (0, 3, 3)
