"""The oracle's pins must catch plausible mistakes in it.

Each case copies ``oracle/ccl_oracle.c`` to a temporary folder, plants one
mistake by text substitution, compiles the copy with gcc and runs a small
battery of the pins from ``test_oracle.py`` on it (exhaustive 3x3 and 2x4
images against pure-Python min-propagation, the hand-drawn worked examples, a
padded-pitch image).  Every planted mistake must fail the battery, and the
unmodified source must pass it.  Nothing here touches the oracle in place.
"""
import ctypes
import os
import subprocess

import numpy as np
import pytest

import oracle
from tests.golden import fixtures

SRC = os.path.join(os.path.dirname(oracle.__file__), "ccl_oracle.c")

MUTATIONS = {
    "no_mutation": [],
    "drop_up_right_neighbour": [
        ("uf_union(parent, p, (int32_t)(p - W + 1));", ";")],
    "drop_up_neighbour": [
        ("uf_union(parent, p, (int32_t)(p - W));", ";")],
    "drop_left_neighbour": [
        ("uf_union(parent, p, p - 1);", ";")],
    "link_smaller_under_larger": [
        ("if (ra < rb) parent[rb] = ra;\n    else parent[ra] = rb;",
         "if (ra < rb) parent[ra] = rb;\n    else parent[rb] = ra;")],
    "label_without_plus_one": [
        ("uf_find(parent, (int32_t)p) + 1;", "uf_find(parent, (int32_t)p);")],
    "row_stride_w_instead_of_pitch": [
        ("is_fg(img, pitch,", "is_fg(img, W,", -1)],
    "up_left_index_off_by_one": [
        ("uf_union(parent, p, (int32_t)(p - W - 1));", "uf_union(parent, p, (int32_t)(p - W));")],
    "first_row_skips_left_link": [
        ("if (x > 0 && is_fg(img, pitch, x - 1, y))", "if (x > 0 && y > 0 && is_fg(img, pitch, x - 1, y))")],
}


def _build_variant(tmp_path, name, subs, symbol="ccl_oracle_two_pass"):
    text = open(SRC).read()
    for sub in subs:
        old, new = sub[0], sub[1]
        count = sub[2] if len(sub) > 2 else 1
        assert old in text, f"mutation {name}: pattern not found"
        text = text.replace(old, new, count)
    c = tmp_path / f"{name}.c"
    so = tmp_path / f"{name}.so"
    c.write_text(text)
    subprocess.check_call(["gcc", "-O1", "-std=c11", "-shared", "-fPIC", str(c), "-o", str(so)])
    lib = ctypes.CDLL(str(so))
    fn = getattr(lib, symbol)
    fn.restype = ctypes.c_int
    nsizes = 4 if symbol.startswith("ccl_oracle3d") else 3
    fn.argtypes = [ctypes.c_void_p] + [ctypes.c_int64] * nsizes + [ctypes.c_int, ctypes.c_void_p]
    return fn


def _run(fn, img, conn):
    H, W = img.shape
    pitch = img.strides[0] if H > 1 else W
    out = np.empty((H, W), np.int32)
    assert fn(img.ctypes.data, H, W, pitch, conn, out.ctypes.data) == 0
    return out


def _battery_passes(fn):
    for conn in (4, 8):
        for H, W in ((3, 3), (2, 4)):
            n = H * W
            for code in range(2 ** n):
                img = np.array([(code >> i) & 1 for i in range(n)], np.uint8).reshape(H, W)
                if not np.array_equal(_run(fn, img, conn), oracle.label_closure(img, conn)):
                    return False
    for path in fixtures.all_fixtures():
        img, want = fixtures.load(path)
        for conn, lab in want.items():
            if not np.array_equal(_run(fn, img, conn), lab):
                return False
    g = np.random.default_rng(3)
    base = (g.random((12, 41)) < 0.5).astype(np.uint8)
    padded = np.ones((12, 64), np.uint8)
    padded[:, :41] = base
    for conn in (4, 8):
        if not np.array_equal(_run(fn, padded[:, :41], conn), oracle.label_closure(base, conn)):
            return False
    return True


@pytest.mark.parametrize("name", sorted(MUTATIONS))
def test_planted_mistake_is_caught(tmp_path, name):
    fn = _build_variant(tmp_path, name, MUTATIONS[name])
    ok = _battery_passes(fn)
    if name == "no_mutation":
        assert ok, "the unmodified oracle must pass its own battery"
    else:
        assert not ok, f"planted mistake '{name}' went unnoticed"


# --- the volume routine -------------------------------------------------------------

MUTATIONS3 = {
    # every planted mistake keeps the routine inside its buffers: it drops or
    # misplaces links and reads, it never follows an unset parent
    "no_mutation": [],
    "previous_slice_skips_the_next_row": [
        ("int earlier = dz < 0 || (dy < 0) || (dy == 0 && dx < 0);",
         "int earlier = (dz < 0 && dy <= 0) || (dy < 0) || (dy == 0 && dx < 0);")],
    "left_link_only_across_slices": [
        ("int earlier = dz < 0 || (dy < 0) || (dy == 0 && dx < 0);",
         "int earlier = dz < 0 || (dy < 0) || (dy == 0 && dx < 0 && dz < 0);")],
    "eighteen_for_twenty_six": [
        ("return conn == 26 || a == 1;", "return (conn == 26 && a <= 2) || a == 1;")],
    "six_without_slice_links": [
        ("return conn == 26 || a == 1;", "return conn == 26 || (a == 1 && dz == 0);")],
    "slice_stride_not_scaled_by_pitch": [
        ("return img[(z * H + y) * pitch + x] != 0;", "return img[z * H + y * pitch + x] != 0;")],
    "label_without_plus_one": [
        ("labels[p] = parent[p] < 0 ? 0 : 1 + uf_find(parent, (int32_t)p);",
         "labels[p] = parent[p] < 0 ? 0 : uf_find(parent, (int32_t)p);")],
}


def _run3(fn, vol, conn):
    D, H, W = vol.shape
    pitch = vol.strides[1]
    assert vol.strides[0] == pitch * H
    out = np.empty((D, H, W), np.int32)
    assert fn(vol.ctypes.data, D, H, W, pitch, conn, out.ctypes.data) == 0
    return out


def _battery3_passes(fn):
    for conn in (6, 26):
        for shape in ((2, 2, 2), (2, 2, 3), (2, 3, 2)):
            n = shape[0] * shape[1] * shape[2]
            for code in range(2 ** n):
                vol = np.array([(code >> i) & 1 for i in range(n)], np.uint8).reshape(shape)
                if not np.array_equal(_run3(fn, vol, conn), oracle.label3d_closure(vol, conn)):
                    return False
    g = np.random.default_rng(4)
    base = (g.random((4, 5, 13)) < 0.45).astype(np.uint8)
    padded = np.ones((4, 5, 16), np.uint8)
    padded[:, :, :13] = base
    for conn in (6, 26):
        if not np.array_equal(_run3(fn, padded[:, :, :13], conn), oracle.label3d_closure(base, conn)):
            return False
    return True


@pytest.mark.parametrize("name", sorted(MUTATIONS3))
def test_planted_mistake_in_volume_routine_is_caught(tmp_path, name):
    fn = _build_variant(tmp_path, "v3_" + name, MUTATIONS3[name], symbol="ccl_oracle3d_two_pass")
    ok = _battery3_passes(fn)
    if name == "no_mutation":
        assert ok, "the unmodified volume routine must pass its own battery"
    else:
        assert not ok, f"planted mistake '{name}' went unnoticed"
