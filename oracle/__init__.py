"""CPU oracle for canonical connected-components labels.

TEST INFRASTRUCTURE ONLY: the tests, ``__graft_entry__.smoke()`` and the CPU
baseline of ``bench.py`` may import this package; the library path must not.
It shares no code with the CUDA implementation.

Canonical labels (the definition every implementation is checked against):
background pixels get 0; every pixel of a connected component gets
1 + the smallest raster position ``x + y*W`` found in that component
(pixel model of Sec. 3; root = element whose label equals its own address,
Sec. 3.1.1; links always point from the larger to the smaller label,
Sec. 3.1.3).  Any nonzero input byte is foreground.

Three independent routes to that result:

* ``label_two_pass`` -- raster two-pass union-find, plain C (``ccl_oracle.c``).
* ``label_bfs``      -- breadth-first flood fill in raster order, plain C.
* ``label_closure``  -- pure Python: repeated min-propagation over the
  adjacency until nothing changes.  Slow; for images of a few hundred pixels.

3D volumes (the 2D/3D problem statement of Sec. 1) follow the same rule one
dimension up: voxel (x, y, z) of a ``(D, H, W)`` array has raster position
``x + y*W + z*W*H``; 6- or 26-connectivity.  ``label3d_two_pass`` and
``label3d_bfs`` (C) and ``label3d_closure`` (pure Python) mirror the 2D
routines.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "ccl_oracle.c")
_LIB = os.path.join(_HERE, "libccl_oracle.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile ``ccl_oracle.c`` into ``libccl_oracle.so`` beside it with gcc."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-shared", "-fPIC", _SRC, "-o", tmp])
        os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    with _lock:
        if _lib is None:
            build()
            lib = ctypes.CDLL(_LIB)
            for name in ("ccl_oracle_two_pass", "ccl_oracle_bfs"):
                fn = getattr(lib, name)
                fn.restype = ctypes.c_int
                fn.argtypes = [ctypes.c_void_p, ctypes.c_int64, ctypes.c_int64,
                               ctypes.c_int64, ctypes.c_int, ctypes.c_void_p]
            for name in ("ccl_oracle3d_two_pass", "ccl_oracle3d_bfs"):
                fn = getattr(lib, name)
                fn.restype = ctypes.c_int
                fn.argtypes = [ctypes.c_void_p, ctypes.c_int64, ctypes.c_int64, ctypes.c_int64,
                               ctypes.c_int64, ctypes.c_int, ctypes.c_void_p]
            _lib = lib
    return _lib


def _call(name: str, img: np.ndarray, conn: int) -> np.ndarray:
    img = np.asarray(img)
    if img.ndim != 2 or img.dtype != np.uint8:
        raise ValueError("image must be a 2D uint8 array")
    if conn not in (4, 8):
        raise ValueError("connectivity must be 4 or 8")
    H, W = img.shape
    if img.strides[1] != 1 or (H > 1 and img.strides[0] < W):
        img = np.ascontiguousarray(img)
    # numpy may report any stride for a dimension of extent 1
    pitch = img.strides[0] if H > 1 else W
    out = np.empty((H, W), dtype=np.int32)
    if H == 0 or W == 0:
        return out
    rc = getattr(_load(), name)(img.ctypes.data, H, W, pitch, conn, out.ctypes.data)
    if rc != 0:
        raise RuntimeError(f"{name} failed with status {rc}")
    return out


def label_two_pass(img: np.ndarray, conn: int) -> np.ndarray:
    """Canonical labels by raster two-pass union-find (C)."""
    return _call("ccl_oracle_two_pass", img, conn)


def label_bfs(img: np.ndarray, conn: int) -> np.ndarray:
    """Canonical labels by raster-order breadth-first flood fill (C)."""
    return _call("ccl_oracle_bfs", img, conn)


def label(img: np.ndarray, conn: int) -> np.ndarray:
    """The oracle's answer: the two-pass union-find labels."""
    return label_two_pass(img, conn)


def label_closure(img: np.ndarray, conn: int) -> np.ndarray:
    """Canonical labels by min-propagation to a fixed point (pure Python).

    Every foreground pixel starts with 1 + its own raster position; each sweep
    replaces a pixel's value by the minimum over itself and its foreground
    neighbours.  At the fixed point every pixel holds the minimum of its
    component.  Quadratic in the worst case: small images only.
    """
    img = np.asarray(img)
    H, W = img.shape
    fg = [[bool(img[y, x]) for x in range(W)] for y in range(H)]
    lab = [[(y * W + x + 1) if fg[y][x] else 0 for x in range(W)] for y in range(H)]
    if conn == 4:
        nbrs = [(-1, 0), (1, 0), (0, -1), (0, 1)]
    elif conn == 8:
        nbrs = [(dx, dy) for dy in (-1, 0, 1) for dx in (-1, 0, 1) if (dx, dy) != (0, 0)]
    else:
        raise ValueError("connectivity must be 4 or 8")
    changed = True
    while changed:
        changed = False
        for y in range(H):
            for x in range(W):
                if not fg[y][x]:
                    continue
                best = lab[y][x]
                for dx, dy in nbrs:
                    nx, ny = x + dx, y + dy
                    if 0 <= nx < W and 0 <= ny < H and fg[ny][nx] and lab[ny][nx] < best:
                        best = lab[ny][nx]
                if best != lab[y][x]:
                    lab[y][x] = best
                    changed = True
    return np.array(lab, dtype=np.int32).reshape(H, W)


def _call3d(name: str, vol: np.ndarray, conn: int) -> np.ndarray:
    vol = np.asarray(vol)
    if vol.ndim != 3 or vol.dtype != np.uint8:
        raise ValueError("volume must be a 3D uint8 array")
    if conn not in (6, 26):
        raise ValueError("connectivity must be 6 or 26")
    D, H, W = vol.shape

    # the C routines take a row pitch and a slice stride of H * pitch
    # (numpy may report any stride for a dimension of extent 1)
    def fits(v):
        s0, s1, s2 = v.strides
        if W > 1 and s2 != 1:
            return False
        if H > 1:
            return s1 >= W and (D == 1 or s0 == s1 * H)
        return D == 1 or s0 >= W

    if not fits(vol):
        vol = np.ascontiguousarray(vol)
    pitch = vol.strides[1] if H > 1 else (vol.strides[0] if D > 1 else W)
    out = np.empty((D, H, W), dtype=np.int32)
    if D == 0 or H == 0 or W == 0:
        return out
    rc = getattr(_load(), name)(vol.ctypes.data, D, H, W, pitch, conn, out.ctypes.data)
    if rc != 0:
        raise RuntimeError(f"{name} failed with status {rc}")
    return out


def label3d_two_pass(vol: np.ndarray, conn: int) -> np.ndarray:
    """Canonical labels of a volume by raster two-pass union-find (C)."""
    return _call3d("ccl_oracle3d_two_pass", vol, conn)


def label3d_bfs(vol: np.ndarray, conn: int) -> np.ndarray:
    """Canonical labels of a volume by raster-order breadth-first flood fill (C)."""
    return _call3d("ccl_oracle3d_bfs", vol, conn)


def label3d(vol: np.ndarray, conn: int) -> np.ndarray:
    """The oracle's answer for a volume: the two-pass union-find labels."""
    return label3d_two_pass(vol, conn)


def label3d_closure(vol: np.ndarray, conn: int) -> np.ndarray:
    """Canonical labels of a volume by min-propagation to a fixed point (pure
    Python; volumes of a few hundred voxels)."""
    vol = np.asarray(vol)
    D, H, W = vol.shape
    if conn not in (6, 26):
        raise ValueError("connectivity must be 6 or 26")
    nbrs = [(dx, dy, dz) for dz in (-1, 0, 1) for dy in (-1, 0, 1) for dx in (-1, 0, 1)
            if (dx, dy, dz) != (0, 0, 0) and (conn == 26 or abs(dx) + abs(dy) + abs(dz) == 1)]
    fg = vol != 0
    lab = {}
    for z in range(D):
        for y in range(H):
            for x in range(W):
                if fg[z, y, x]:
                    lab[(x, y, z)] = x + y * W + z * W * H + 1
    changed = True
    while changed:
        changed = False
        for (x, y, z), v in list(lab.items()):
            best = v
            for dx, dy, dz in nbrs:
                w = lab.get((x + dx, y + dy, z + dz))
                if w is not None and w < best:
                    best = w
            if best != v:
                lab[(x, y, z)] = best
                changed = True
    out = np.zeros((D, H, W), dtype=np.int32)
    for (x, y, z), v in lab.items():
        out[z, y, x] = v
    return out


def component_stats(labels: np.ndarray) -> np.ndarray:
    """Statistics of every component of a canonical label image, in increasing
    label order (the use the paper motivates in Sec. 1: size and location of
    each region).  One row per component:
    ``label, area, x0, y0, x1, y1, sum_x, sum_y`` -- area is the pixel count,
    (x0, y0)-(x1, y1) the inclusive bounding box, sum_x and sum_y the sums of
    the pixel coordinates (centroid = sum / area).  Plain numpy on the
    definition: every pixel with label l > 0 belongs to component l."""
    labels = np.asarray(labels)
    H, W = labels.shape
    ys, xs = np.nonzero(labels)
    lab = labels[ys, xs].astype(np.int64)
    order = np.argsort(lab, kind="stable")
    lab, ys, xs = lab[order], ys[order].astype(np.int64), xs[order].astype(np.int64)
    if lab.size == 0:
        return np.zeros((0, 8), dtype=np.int64)
    uniq, first, area = np.unique(lab, return_index=True, return_counts=True)
    out = np.zeros((uniq.size, 8), dtype=np.int64)
    out[:, 0] = uniq
    out[:, 1] = area
    out[:, 2] = np.minimum.reduceat(xs, first)
    out[:, 3] = np.minimum.reduceat(ys, first)
    out[:, 4] = np.maximum.reduceat(xs, first)
    out[:, 5] = np.maximum.reduceat(ys, first)
    out[:, 6] = np.add.reduceat(xs, first)
    out[:, 7] = np.add.reduceat(ys, first)
    return out
