"""Pins for the CPU oracle (no GPU).

The oracle computes canonical labels: background 0, every pixel of a component
1 + the component's smallest raster position (pixel model of Sec. 3, root rule
of Sec. 3.1.1).  Its answer is pinned here against things other than itself:

* exhaustive enumeration of every image up to 4x4 against the independent
  flood fill, and up to 3x4 against pure-Python min-propagation;
* hand-drawn worked examples with hand-computed labels (``tests/golden``);
* closed forms (empty, full, checkerboards, isolated pixels, single rows and
  columns, spiral, rings, comb);
* scipy.ndimage.label partitions on random images (a library routine);
* invariants (flip/transpose component counts, idempotence, root property,
  4-connected partition refining the 8-connected one).
"""
import itertools

import numpy as np
import pytest

import oracle
from paper_1712_09789_gb300 import synth
from tests.golden import fixtures

CONNS = (4, 8)


def all_images(H, W):
    n = H * W
    bits = ((np.arange(2 ** n)[:, None] >> np.arange(n)[None, :]) & 1).astype(np.uint8)
    return bits.reshape(-1, H, W)


def canonical_from_partition(lab):
    """Relabel any partition (0 = background) into canonical min-index form."""
    H, W = lab.shape
    flat = lab.ravel()
    out = np.zeros(flat.shape, dtype=np.int32)
    ids = np.unique(flat[flat > 0])
    idx = np.arange(flat.size)
    for v in ids:
        m = flat == v
        out[m] = idx[m].min() + 1
    return out.reshape(H, W)


def n_components(lab):
    return len(np.unique(lab[lab > 0]))


# --- exhaustive -------------------------------------------------------------

@pytest.mark.parametrize("conn", CONNS)
def test_exhaustive_two_pass_vs_bfs_up_to_4x4(conn):
    for H in range(1, 5):
        for W in range(1, 5):
            for img in all_images(H, W):
                a = oracle.label_two_pass(img, conn)
                b = oracle.label_bfs(img, conn)
                if not np.array_equal(a, b):
                    raise AssertionError(f"{H}x{W} conn={conn}\n{img}\n{a}\n{b}")


@pytest.mark.parametrize("conn", CONNS)
def test_exhaustive_vs_python_closure_up_to_3x4(conn):
    for H, W in [(1, 1), (1, 4), (4, 1), (2, 2), (2, 3), (3, 2), (3, 3), (3, 4), (4, 3)]:
        for img in all_images(H, W):
            a = oracle.label_two_pass(img, conn)
            c = oracle.label_closure(img, conn)
            if not np.array_equal(a, c):
                raise AssertionError(f"{H}x{W} conn={conn}\n{img}\n{a}\n{c}")


# --- hand-drawn worked examples ---------------------------------------------

@pytest.mark.parametrize("path", fixtures.all_fixtures(), ids=lambda p: p.rsplit("/", 1)[-1])
def test_golden_fixtures(path):
    img, expected = fixtures.load(path)
    assert expected, "fixture holds no labels"
    for conn, want in expected.items():
        assert want.shape == img.shape
        for fn in (oracle.label_two_pass, oracle.label_bfs, oracle.label_closure):
            got = fn(img, conn)
            np.testing.assert_array_equal(got, want, err_msg=f"{fn.__name__} conn={conn}")


# --- closed forms -------------------------------------------------------------

@pytest.mark.parametrize("conn", CONNS)
@pytest.mark.parametrize("H,W", [(1, 1), (1, 37), (37, 1), (5, 7), (64, 64), (33, 100)])
def test_empty_and_full(conn, H, W):
    z = np.zeros((H, W), np.uint8)
    np.testing.assert_array_equal(oracle.label(z, conn), 0)
    o = np.ones((H, W), np.uint8)
    np.testing.assert_array_equal(oracle.label(o, conn), 1)
    # any nonzero byte is foreground
    o7 = np.full((H, W), 7, np.uint8)
    np.testing.assert_array_equal(oracle.label(o7, conn), 1)


@pytest.mark.parametrize("H,W", [(1, 1), (2, 2), (9, 13), (64, 64), (31, 33)])
def test_checkerboard(H, W):
    ys, xs = np.mgrid[:H, :W]
    img = ((xs + ys) % 2 == 0).astype(np.uint8)
    idx = (ys * W + xs).astype(np.int32)
    # 4-connectivity: every foreground pixel is alone -> 1 + own position
    np.testing.assert_array_equal(oracle.label(img, 4), np.where(img == 1, idx + 1, 0))
    # 8-connectivity: all foreground pixels touch at corners -> one component;
    # its smallest position is (0,0)
    np.testing.assert_array_equal(oracle.label(img, 8), np.where(img == 1, 1, 0))
    # the other colour: 8-connected as well, smallest position is (1,0) = 1
    inv = 1 - img
    if inv.any():
        want = 2 if W > 1 else W + 1
        np.testing.assert_array_equal(oracle.label(inv, 8), np.where(inv == 1, want, 0))


@pytest.mark.parametrize("conn", CONNS)
def test_isolated_pixels(conn):
    H, W = 40, 50
    img = np.zeros((H, W), np.uint8)
    img[::3, ::3] = 1
    ys, xs = np.mgrid[:H, :W]
    want = np.where(img == 1, ys * W + xs + 1, 0)
    np.testing.assert_array_equal(oracle.label(img, conn), want)


@pytest.mark.parametrize("conn", CONNS)
def test_single_row_and_column_runs(conn):
    g = np.random.default_rng(5)
    for W in (1, 2, 3, 31, 32, 33, 200):
        row = (g.random((1, W)) < 0.5).astype(np.uint8)
        want = np.zeros((1, W), np.int32)
        start = None
        for x in range(W):
            if row[0, x]:
                if start is None:
                    start = x
                want[0, x] = start + 1
            else:
                start = None
        np.testing.assert_array_equal(oracle.label(row, conn), want)
        # a single column: runs along y, positions are y (W = 1)
        np.testing.assert_array_equal(oracle.label(row.T.copy(), conn), want.T)


@pytest.mark.parametrize("conn", CONNS)
@pytest.mark.parametrize("N", [1, 2, 3, 4, 5, 6, 7, 9, 16, 33, 64, 101, 256])
def test_spiral_is_one_component(conn, N):
    img = synth.spiral(N)
    lab = oracle.label(img, conn)
    assert n_components(lab) == 1
    assert lab[0, 0] == 1
    # the spiral leaves gaps: not a filled square once N > 2
    if N > 2:
        assert img.sum() < N * N


@pytest.mark.parametrize("conn", CONNS)
@pytest.mark.parametrize("N", [1, 2, 3, 7, 8, 20, 64, 99])
def test_rings_count(conn, N):
    img = synth.rings(N)
    lab = oracle.label(img, conn)
    assert n_components(lab) == synth.ring_count(N)


@pytest.mark.parametrize("conn", CONNS)
@pytest.mark.parametrize("H,W", [(3, 3), (4, 9), (50, 64), (64, 129)])
def test_comb_is_one_component(conn, H, W):
    lab = oracle.label(synth.comb(H, W), conn)
    assert n_components(lab) == 1 and lab[0, 0] == 1


# --- library routine ------------------------------------------------------------

@pytest.mark.parametrize("conn", CONNS)
def test_scipy_partition_random_64(conn):
    ndi = pytest.importorskip("scipy.ndimage")
    structure = np.ones((3, 3), int) if conn == 8 else ndi.generate_binary_structure(2, 1)
    for k in range(1, 10):
        for seed in range(0, 100, 9):
            img = synth.bernoulli(64, 64, k / 10, seed)
            lab_sp, _ = ndi.label(img, structure=structure)
            want = canonical_from_partition(lab_sp)
            np.testing.assert_array_equal(oracle.label(img, conn), want)


@pytest.mark.parametrize("conn", CONNS)
def test_random_64_two_pass_vs_bfs(conn):
    for k in range(1, 10):
        for seed in range(100):
            img = synth.bernoulli(64, 64, k / 10, seed)
            np.testing.assert_array_equal(oracle.label_two_pass(img, conn),
                                          oracle.label_bfs(img, conn))


# --- invariants -------------------------------------------------------------------

@pytest.mark.parametrize("conn", CONNS)
def test_invariants(conn):
    g = np.random.default_rng(11)
    for trial in range(30):
        H, W = int(g.integers(1, 80)), int(g.integers(1, 80))
        img = (g.random((H, W)) < g.uniform(0.2, 0.8)).astype(np.uint8)
        lab = oracle.label(img, conn)
        n = n_components(lab)
        # component count is invariant under flips and transpose
        for t in (img[::-1], img[:, ::-1], img.T):
            assert n_components(oracle.label(np.ascontiguousarray(t), conn)) == n
        # idempotence: labelling the foreground of the output gives the output
        np.testing.assert_array_equal(oracle.label((lab > 0).astype(np.uint8), conn), lab)
        # root property: the pixel at position v-1 carries label v
        flat = lab.ravel()
        vals = np.unique(flat[flat > 0])
        np.testing.assert_array_equal(flat[vals - 1], vals)
        # every pixel's label is <= 1 + its own position
        pos = np.arange(flat.size) + 1
        assert np.all(flat[flat > 0] <= pos[flat > 0])
    # the 4-connected partition refines the 8-connected one
    for trial in range(30):
        img = (g.random((40, 40)) < 0.5).astype(np.uint8)
        l4, l8 = oracle.label(img, 4), oracle.label(img, 8)
        for v in np.unique(l4[l4 > 0]):
            assert len(np.unique(l8[l4 == v])) == 1


def test_pitch_and_nonzero_bytes():
    g = np.random.default_rng(3)
    base = (g.random((30, 41)) < 0.5).astype(np.uint8)
    padded = np.zeros((30, 64), np.uint8)
    padded[:, :41] = base * g.integers(1, 256, size=base.shape).astype(np.uint8)
    padded[:, 41:] = 1  # bytes beyond W must be ignored
    view = padded[:, :41]
    assert view.strides[0] == 64
    for conn in CONNS:
        np.testing.assert_array_equal(oracle.label(view, conn), oracle.label(base, conn))


def test_rejects_bad_arguments():
    with pytest.raises(ValueError):
        oracle.label(np.zeros((3, 3), np.uint8), 6)
    with pytest.raises(ValueError):
        oracle.label(np.zeros((3, 3), np.int32), 4)
    # empty images label to empty outputs
    assert oracle.label(np.zeros((0, 5), np.uint8), 4).shape == (0, 5)


# -- component statistics (oracle.component_stats), pinned by closed forms and
# by a per-component brute force
def test_component_stats_closed_forms():
    # one filled rectangle: area, box and coordinate sums in closed form
    img = np.zeros((9, 13), np.uint8)
    img[2:7, 3:11] = 1
    st = oracle.component_stats(oracle.label(img, 8))
    assert st.shape == (1, 8)
    xs, ys = np.arange(3, 11), np.arange(2, 7)
    assert st[0].tolist() == [1 + 2 * 13 + 3, 40, 3, 2, 10, 6, ys.size * xs.sum(), xs.size * ys.sum()]
    # 4-connected checkerboard: every pixel its own component, label 1 + index
    y, x = np.mgrid[0:5, 0:7]
    cb = ((x + y) % 2 == 0).astype(np.uint8)
    st = oracle.component_stats(oracle.label(cb, 4))
    py, px = np.nonzero(cb)
    assert st[:, 0].tolist() == (1 + px + py * 7).tolist()
    assert (st[:, 1] == 1).all()
    assert st[:, 2].tolist() == px.tolist() and st[:, 4].tolist() == px.tolist()
    assert st[:, 3].tolist() == py.tolist() and st[:, 5].tolist() == py.tolist()
    assert st[:, 6].tolist() == px.tolist() and st[:, 7].tolist() == py.tolist()
    # empty image: no rows
    assert oracle.component_stats(np.zeros((3, 3), np.int32)).shape == (0, 8)


@pytest.mark.parametrize("conn", (4, 8))
def test_component_stats_brute_force(conn):
    g = np.random.default_rng(31)
    img = (g.random((40, 57)) < 0.45).astype(np.uint8)
    lab = oracle.label(img, conn)
    st = oracle.component_stats(lab)
    assert st[:, 1].sum() == int(img.astype(bool).sum())
    for row in st:
        yy, xx = np.nonzero(lab == row[0])
        assert row[1] == yy.size
        assert (row[2], row[3], row[4], row[5]) == (xx.min(), yy.min(), xx.max(), yy.max())
        assert (row[6], row[7]) == (xx.sum(), yy.sum())
        # the label is the component's smallest raster position plus one
        assert row[0] == 1 + (yy * img.shape[1] + xx).min()
