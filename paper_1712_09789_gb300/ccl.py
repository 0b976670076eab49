"""Thin Python binding of the C ABI in ``include/ccl.h``.

Argument marshalling only: every function hands tensors' device pointers,
sizes and the current CUDA stream to ``libccl.so`` and raises ``CclError``
on a non-OK status.  The library must have been built (``build()`` in
``__graft_entry__`` or ``python -m paper_1712_09789_gb300.build``); there is
no fallback, and importing a missing library fails loudly.

Tensors: images are 2D ``uint8`` CUDA tensors whose rows are contiguous
(``stride(1) == 1``; the row stride ``stride(0)`` is passed as the pitch);
labels are 2D ``int32`` CUDA tensors, contiguous.
"""
from __future__ import annotations

import ctypes
import os
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libccl.so")
_lock = threading.Lock()
_lib = None

CCL_OK = 0
CCL_ERR_INVALID_ARG = 1
CCL_ERR_UNSUPPORTED = 2
CCL_ERR_OUT_OF_MEMORY = 3
CCL_ERR_CUDA = 4
CCL_ERR_DEVICE_TIMEOUT = 5
CCL_ERR_BUSY = 6
CCL_ERR_NOT_FOUND = 7


class CclError(RuntimeError):
    def __init__(self, status: int, where: str):
        self.status = status
        super().__init__(f"{where}: {ccl_status_string(status)} ({status})")


_c = ctypes


class CclImage(ctypes.Structure):
    """``ccl_image``: one entry of a batch."""
    _fields_ = [("img", ctypes.c_void_p), ("labels", ctypes.c_void_p), ("H", ctypes.c_int),
                ("W", ctypes.c_int), ("pitch", ctypes.c_size_t)]


class CclServerConfig(ctypes.Structure):
    """``ccl_server_config``."""
    _fields_ = [("max_slots", ctypes.c_int), ("n_streams", ctypes.c_int), ("max_batch", ctypes.c_int),
                ("device", ctypes.c_int), ("hbm_budget_bytes", ctypes.c_size_t)]


class CclServerStats(ctypes.Structure):
    """``ccl_server_stats_t``."""
    _fields_ = [("submitted", ctypes.c_uint64), ("completed", ctypes.c_uint64), ("rejected", ctypes.c_uint64),
                ("in_flight", ctypes.c_int), ("queued", ctypes.c_int), ("pixels", ctypes.c_uint64),
                ("arena_bytes", ctypes.c_size_t), ("arena_used_bytes", ctypes.c_size_t),
                ("p50_ms", ctypes.c_double), ("p99_ms", ctypes.c_double), ("max_ms", ctypes.c_double),
                ("mean_ms", ctypes.c_double), ("gpixel_s", ctypes.c_double),
                ("queue_p50_ms", ctypes.c_double), ("queue_p99_ms", ctypes.c_double),
                ("h2d_p50_ms", ctypes.c_double), ("h2d_p99_ms", ctypes.c_double),
                ("label_p50_ms", ctypes.c_double), ("label_p99_ms", ctypes.c_double),
                ("d2h_p50_ms", ctypes.c_double), ("d2h_p99_ms", ctypes.c_double),
                ("batches", ctypes.c_uint64), ("multi_request_batches", ctypes.c_uint64),
                ("overlapped_batches", ctypes.c_uint64), ("max_batch_requests", ctypes.c_int),
                ("max_batches_in_flight", ctypes.c_int)]


_SIGS = {
    "ccl_status_string": (_c.c_char_p, [_c.c_int]),
    "ccl_version": (_c.c_int, []),
    "ccl_label": (_c.c_int, [_c.c_void_p, _c.c_int, _c.c_int, _c.c_size_t, _c.c_int, _c.c_void_p,
                             _c.c_void_p]),
    "ccl_workspace_size": (_c.c_int, [_c.c_int, _c.c_int, _c.c_int, _c.POINTER(_c.c_size_t)]),
    "ccl_label_ws": (_c.c_int, [_c.c_void_p, _c.c_int, _c.c_int, _c.c_size_t, _c.c_int, _c.c_void_p,
                                _c.c_void_p, _c.c_size_t, _c.c_void_p]),
    "ccl_label_host": (_c.c_int, [_c.c_void_p, _c.c_int, _c.c_int, _c.c_size_t, _c.c_int,
                                  _c.c_void_p, _c.c_void_p]),
    "ccl_label_host_async": (_c.c_int, [_c.c_void_p, _c.c_int, _c.c_int, _c.c_size_t, _c.c_int,
                                        _c.c_void_p, _c.c_void_p]),
    "ccl_get_device_status": (_c.c_int, [_c.c_void_p]),
    "ccl_release_stream": (_c.c_int, [_c.c_void_p]),
    "ccl_label_noalloc": (_c.c_int, [_c.c_void_p, _c.c_int, _c.c_int, _c.c_size_t, _c.c_int, _c.c_void_p,
                                     _c.c_void_p]),
    "ccl_noalloc_max_workspace_bytes": (_c.c_size_t, []),
    "ccl_component_stats": (_c.c_int, [_c.c_void_p, _c.c_int, _c.c_int, _c.c_void_p, _c.c_int,
                                       _c.POINTER(_c.c_int), _c.c_void_p]),
    "ccl_label_variant": (_c.c_int, [_c.c_void_p, _c.c_int, _c.c_int, _c.c_size_t, _c.c_int, _c.c_int, _c.c_void_p,
                                     _c.POINTER(_c.c_ulonglong), _c.c_void_p]),
    "ccl_label_3d": (_c.c_int, [_c.c_void_p, _c.c_int, _c.c_int, _c.c_int, _c.c_size_t, _c.c_int, _c.c_void_p,
                                _c.c_void_p]),
    "ccl_label_batched": (_c.c_int, [_c.POINTER(CclImage), _c.c_int, _c.c_int, _c.c_void_p]),
    "ccl_label_batched_tile": (_c.c_int, [_c.POINTER(CclImage), _c.c_int, _c.c_int, _c.c_int, _c.c_void_p]),
    "ccl_autotune_batched": (_c.c_int, [_c.POINTER(CclImage), _c.c_int, _c.c_int, _c.c_void_p,
                                        _c.POINTER(_c.c_int)]),
    "ccl_batched_tile": (_c.c_int, [_c.POINTER(CclImage), _c.c_int, _c.c_int, _c.POINTER(_c.c_int)]),
    "ccl_tile_count": (_c.c_int, []),
    "ccl_server_create": (_c.c_int, [_c.POINTER(CclServerConfig), _c.POINTER(_c.c_void_p)]),
    "ccl_server_frame_bytes": (_c.c_int, [_c.c_int, _c.c_int, _c.POINTER(_c.c_size_t)]),
    "ccl_server_submit": (_c.c_int, [_c.c_void_p, _c.c_void_p, _c.c_int, _c.c_int, _c.c_size_t, _c.c_int,
                                     _c.c_void_p, _c.POINTER(_c.c_uint64)]),
    "ccl_server_wait": (_c.c_int, [_c.c_void_p, _c.c_uint64, _c.c_int]),
    "ccl_server_poll": (_c.c_int, [_c.c_void_p, _c.c_uint64]),
    "ccl_server_stats": (_c.c_int, [_c.c_void_p, _c.POINTER(CclServerStats)]),
    "ccl_server_reset_stats": (_c.c_int, [_c.c_void_p]),
    "ccl_server_destroy": (None, [_c.c_void_p]),
    "ccl_tile_name": (_c.c_char_p, [_c.c_int]),
    "ccl_strip_begin": (_c.c_int, [_c.c_void_p, _c.c_int, _c.c_int, _c.c_size_t, _c.c_int, _c.c_int, _c.c_int,
                                   _c.c_void_p, _c.c_size_t, _c.c_void_p, _c.c_void_p]),
    "ccl_strip_resolve": (_c.c_int, [_c.c_void_p, _c.c_int, _c.c_int, _c.c_int, _c.c_void_p, _c.c_size_t,
                                     _c.POINTER(_c.c_size_t)]),
    "ccl_strip_finish": (_c.c_int, [_c.c_int, _c.c_int, _c.c_int, _c.c_int, _c.c_int, _c.c_void_p, _c.c_size_t,
                                    _c.c_void_p, _c.c_void_p, _c.c_size_t, _c.c_void_p]),
    "ccl_debug_set_iteration_cap": (None, [_c.c_int]),
    "ccl_debug_kernel_timing": (None, [_c.c_int]),
    "ccl_debug_kernel_times": (_c.c_int, [_c.POINTER(_c.c_double), _c.POINTER(_c.c_longlong), _c.c_int]),
    "ccl_debug_kernel_name": (_c.c_char_p, [_c.c_int]),
}


def load() -> ctypes.CDLL:
    """Load ``libccl.so`` and declare its signatures (once)."""
    global _lib
    with _lock:
        if _lib is None:
            if not os.path.exists(LIB_PATH):
                raise ImportError(
                    f"{LIB_PATH} is missing: build the CUDA library first "
                    "(python -m paper_1712_09789_gb300.build)")
            lib = ctypes.CDLL(LIB_PATH)
            for name, (res, args) in _SIGS.items():
                fn = getattr(lib, name, None)
                if fn is None:
                    continue
                fn.restype = res
                fn.argtypes = args
            _lib = lib
    return _lib


def _check(st: int, where: str):
    if st != CCL_OK:
        raise CclError(st, where)


def _device_guard(device):
    """Context that makes `device` the current CUDA device.  The library takes
    its per-device scratch (and the no-allocation array's address) from the
    current device, so every call runs with the tensors' device current."""
    import torch

    return torch.cuda.device(device)


def _call(name: str, device, *args):
    """Calls C-ABI function `name` with `device` current (see _device_guard)."""
    with _device_guard(device):
        return getattr(load(), name)(*args)


def ccl_status_string(status: int) -> str:
    return load().ccl_status_string(status).decode()


def ccl_version() -> int:
    return load().ccl_version()


def _stream_ptr(stream, device) -> int:
    import torch

    if stream is None:
        stream = torch.cuda.current_stream(device)
    return int(stream.cuda_stream) if hasattr(stream, "cuda_stream") else int(stream)


def _image_args(img):
    import torch

    if not isinstance(img, torch.Tensor) or img.dtype != torch.uint8 or img.dim() != 2:
        raise ValueError("image must be a 2D torch.uint8 tensor")
    if not img.is_cuda:
        raise ValueError("image must be a CUDA tensor")
    H, W = img.shape
    if W > 0 and H > 1 and img.stride(1) != 1:
        raise ValueError("image rows must be contiguous (stride(1) == 1)")
    pitch = img.stride(0) if H > 1 else W
    return H, W, pitch


def _labels_for(img, labels):
    import torch

    H, W = img.shape
    if labels is None:
        return torch.empty((H, W), dtype=torch.int32, device=img.device)
    if labels.dtype != torch.int32 or tuple(labels.shape) != (H, W) or not labels.is_contiguous():
        raise ValueError("labels must be a contiguous int32 tensor of the image's shape")
    if labels.device != img.device:
        raise ValueError("labels must be on the image's device")
    return labels


def ccl_label(img, connectivity: int = 8, labels=None, stream=None):
    """Canonical labels of a device image (``ccl_label``).  Returns ``labels``."""
    H, W, pitch = _image_args(img)
    labels = _labels_for(img, labels)
    st = _call("ccl_label", img.device, img.data_ptr(), H, W, pitch, connectivity, labels.data_ptr(),
                          _stream_ptr(stream, img.device))
    _check(st, "ccl_label")
    return labels


def ccl_label_noalloc(img, connectivity: int = 8, labels=None, stream=None):
    """``ccl_label`` without any device allocation (``ccl_label_noalloc``):
    the scratch is the library's fixed per-device array, so this suits callers
    that may not allocate while running.  ``labels`` should be preallocated by
    such callers; overlapping calls race on the shared scratch."""
    H, W, pitch = _image_args(img)
    labels = _labels_for(img, labels)
    st = _call("ccl_label_noalloc", img.device, img.data_ptr(), H, W, pitch, connectivity, labels.data_ptr(),
                                  _stream_ptr(stream, img.device))
    _check(st, "ccl_label_noalloc")
    return labels


def ccl_label_3d(vol, connectivity: int = 26, labels=None, stream=None):
    """Canonical labels of a device volume (``ccl_label_3d``): ``vol`` is a 3D
    ``torch.uint8`` CUDA tensor ``[D][H][W]`` with contiguous rows and a slice
    stride of H row strides; ``labels`` a contiguous int32 ``[D][H][W]``
    tensor (allocated when None).  Returns ``labels``."""
    import torch

    if not isinstance(vol, torch.Tensor) or vol.dtype != torch.uint8 or vol.dim() != 3:
        raise ValueError("volume must be a 3D torch.uint8 tensor")
    if not vol.is_cuda:
        raise ValueError("volume must be a CUDA tensor")
    D, H, W = vol.shape
    # numpy-style strides of extent-1 dimensions carry no meaning
    if W > 1 and vol.stride(2) != 1:
        raise ValueError("volume rows must be contiguous (stride(2) == 1)")
    if H > 1:
        pitch = vol.stride(1)
        if D > 1 and vol.stride(0) != pitch * H:
            raise ValueError("the slice stride must be H times the row stride")
    else:
        pitch = vol.stride(0) if D > 1 else W
    if labels is None:
        labels = torch.empty((D, H, W), dtype=torch.int32, device=vol.device)
    elif (labels.dtype != torch.int32 or tuple(labels.shape) != (D, H, W) or not labels.is_contiguous()
          or labels.device != vol.device):
        raise ValueError("labels must be a contiguous int32 tensor of the volume's shape and device")
    st = _call("ccl_label_3d", vol.device, vol.data_ptr(), D, H, W, pitch, connectivity, labels.data_ptr(),
                             _stream_ptr(stream, vol.device))
    _check(st, "ccl_label_3d")
    return labels


VARIANTS = ("C2FL", "RC2FL", "CC2FL", "NC2FL")


def ccl_label_variant(img, connectivity: int = 8, variant: int = 0, labels=None, stream=None,
                      counters: bool = False):
    """One of the coarse-labelling variants of Sec. 4.2 (``ccl_label_variant``):
    0 C2FL (the method), 1 RC2FL, 2 CC2FL, 3 NC2FL; all give the same labels.
    With ``counters`` the call is synchronous and also returns the counts of
    step 1: {"merges", "find_steps", "atomics"}."""
    H, W, pitch = _image_args(img)
    labels = _labels_for(img, labels)
    cnt = (ctypes.c_ulonglong * 3)()
    st = _call("ccl_label_variant", img.device, img.data_ptr(), H, W, pitch, connectivity, variant, labels.data_ptr(),
                                  cnt if counters else None, _stream_ptr(stream, img.device))
    _check(st, "ccl_label_variant")
    if counters:
        return labels, {"merges": cnt[0], "find_steps": cnt[1], "atomics": cnt[2]}
    return labels


# numpy layout of ``ccl_component`` (40 bytes)
COMPONENT_DTYPE = [("label", "<i4"), ("area", "<i4"), ("x0", "<i4"), ("y0", "<i4"), ("x1", "<i4"), ("y1", "<i4"),
                   ("sum_x", "<i8"), ("sum_y", "<i8")]


def ccl_component_stats(labels, stream=None, capacity=None):
    """Size and location of every component of a canonical label image on the
    device (``ccl_component_stats``): a numpy structured array in label order
    with fields label, area, x0, y0, x1, y1, sum_x, sum_y.  Without
    ``capacity`` a first call counts the components."""
    import numpy as np
    import torch

    if labels.dtype != torch.int32 or labels.dim() != 2 or not labels.is_cuda or not labels.is_contiguous():
        raise ValueError("labels must be a contiguous 2D int32 CUDA tensor")
    H, W = labels.shape
    sp = _stream_ptr(stream, labels.device)
    n = ctypes.c_int(0)
    if capacity is None:
        _check(_call("ccl_component_stats", labels.device, labels.data_ptr(), H, W, None, 0, ctypes.byref(n), sp),
               "ccl_component_stats")
        capacity = n.value
    buf = torch.empty(max(1, capacity) * 40, dtype=torch.uint8, device=labels.device)
    _check(_call("ccl_component_stats", labels.device, labels.data_ptr(), H, W, buf.data_ptr(), capacity,
                 ctypes.byref(n), sp),
           "ccl_component_stats")
    k = min(n.value, capacity)
    return np.frombuffer(buf[: k * 40].cpu().numpy().tobytes(), dtype=np.dtype(COMPONENT_DTYPE))


def ccl_noalloc_max_workspace_bytes() -> int:
    return load().ccl_noalloc_max_workspace_bytes()


def ccl_workspace_size(H: int, W: int, connectivity: int = 8) -> int:
    out = ctypes.c_size_t(0)
    _check(load().ccl_workspace_size(H, W, connectivity, ctypes.byref(out)), "ccl_workspace_size")
    return out.value


def ccl_label_ws(img, workspace, connectivity: int = 8, labels=None, stream=None):
    """``ccl_label`` with a caller-owned scratch tensor (``ccl_label_ws``)."""
    H, W, pitch = _image_args(img)
    labels = _labels_for(img, labels)
    nbytes = workspace.numel() * workspace.element_size()
    st = _call("ccl_label_ws", img.device, img.data_ptr(), H, W, pitch, connectivity, labels.data_ptr(),
                             workspace.data_ptr(), nbytes, _stream_ptr(stream, img.device))
    _check(st, "ccl_label_ws")
    return labels


def ccl_strip_begin(img, y0: int, H_total: int, workspace, connectivity: int = 8, edges=None, stream=None):
    """First half of a strip's labelling (``ccl_strip_begin``): `img` is rows
    [y0, y0 + H) of an H_total-row image.  Returns the strip's edge rows, an
    int32 device tensor [2, W] holding the uint32 keys (0xFFFFFFFF, i.e. -1,
    for background)."""
    import torch

    H, W, pitch = _image_args(img)
    if edges is None:
        edges = torch.empty((2, W), dtype=torch.int32, device=img.device)
    elif edges.dtype != torch.int32 or tuple(edges.shape) != (2, W) or not edges.is_contiguous():
        raise ValueError("edges must be a contiguous int32 tensor [2, W]")
    nbytes = workspace.numel() * workspace.element_size()
    st = _call("ccl_strip_begin", img.device, img.data_ptr(), H, W, pitch, connectivity, y0, H_total,
               workspace.data_ptr(), nbytes, edges.data_ptr(), _stream_ptr(stream, img.device))
    _check(st, "ccl_strip_begin")
    return edges


def ccl_strip_resolve(edges_all: np.ndarray, connectivity: int = 8) -> np.ndarray:
    """Seam equivalences of gathered edge rows (``ccl_strip_resolve``, host
    only): `edges_all` is uint32 (or int32 bits) [strips, 2, W] in strip order.
    Returns a uint32 array [n, 2] of (key, smallest key) sorted by key."""
    e = np.ascontiguousarray(edges_all).view(np.uint32)
    if e.ndim != 3 or e.shape[1] != 2:
        raise ValueError("edges_all must have shape [strips, 2, W]")
    G, _, W = e.shape
    n = ctypes.c_size_t(0)
    # at most one pair per pixel of the seam rows
    out = np.empty((max(2 * (G - 1) * W, 1), 2), dtype=np.uint32)
    st = load().ccl_strip_resolve(e.ctypes.data, G, W, connectivity, out.ctypes.data, out.shape[0],
                                  ctypes.byref(n))
    _check(st, "ccl_strip_resolve")
    return out[:n.value]


def ccl_strip_finish(H: int, W: int, y0: int, H_total: int, seam_map, workspace, connectivity: int = 8,
                     labels=None, stream=None):
    """Second half of a strip's labelling (``ccl_strip_finish``): `seam_map`
    is the device copy (int32 bits, [n, 2]) of ``ccl_strip_resolve``'s pairs.
    Writes and returns the strip's labels (labels of the whole image)."""
    import torch

    dev = workspace.device
    if labels is None:
        labels = torch.empty((H, W), dtype=torch.int32, device=dev)
    elif labels.dtype != torch.int32 or tuple(labels.shape) != (H, W) or not labels.is_contiguous():
        raise ValueError("labels must be a contiguous int32 tensor [H, W]")
    n = 0 if seam_map is None else int(seam_map.shape[0])
    if n and (seam_map.dtype != torch.int32 or not seam_map.is_contiguous() or seam_map.device != dev):
        raise ValueError("seam_map must be a contiguous int32 tensor on the workspace's device")
    nbytes = workspace.numel() * workspace.element_size()
    st = _call("ccl_strip_finish", dev, H, W, connectivity, y0, H_total, seam_map.data_ptr() if n else None, n,
               labels.data_ptr(), workspace.data_ptr(), nbytes, _stream_ptr(stream, dev))
    _check(st, "ccl_strip_finish")
    return labels


def ccl_label_host(img: np.ndarray, connectivity: int = 8, labels: np.ndarray | None = None,
                   stream=None) -> np.ndarray:
    """Labels of a host image; copies in, labels, copies out and waits
    (``ccl_label_host``).  ``img`` is a 2D uint8 array with contiguous rows."""
    if not isinstance(img, np.ndarray) or img.dtype != np.uint8 or img.ndim != 2:
        raise ValueError("image must be a 2D numpy uint8 array")
    H, W = img.shape
    if W > 0 and H > 1 and img.strides[1] != 1:
        raise ValueError("image rows must be contiguous")
    pitch = img.strides[0] if H > 1 else W
    if labels is None:
        labels = np.empty((H, W), np.int32)
    elif labels.dtype != np.int32 or labels.shape != (H, W) or not labels.flags.c_contiguous:
        raise ValueError("labels must be a contiguous int32 array of the image's shape")
    import torch

    dev = torch.device("cuda", torch.cuda.current_device())
    st = _call("ccl_label_host", dev, img.ctypes.data, H, W, pitch, connectivity, labels.ctypes.data,
               _stream_ptr(stream, dev))
    _check(st, "ccl_label_host")
    return labels


def ccl_label_host_async(img: np.ndarray, labels: np.ndarray, connectivity: int = 8, stream=None) -> None:
    """Enqueues copy in, labelling and copy out of a host image on ``stream``
    (``ccl_label_host_async``); ``labels`` holds the result once the stream
    has reached that point.  Both arrays should be page-locked (e.g. numpy
    views of pinned torch tensors) and must stay alive until then."""
    if not isinstance(img, np.ndarray) or img.dtype != np.uint8 or img.ndim != 2:
        raise ValueError("image must be a 2D numpy uint8 array")
    H, W = img.shape
    if W > 0 and H > 1 and img.strides[1] != 1:
        raise ValueError("image rows must be contiguous")
    if labels.dtype != np.int32 or labels.shape != (H, W) or not labels.flags.c_contiguous:
        raise ValueError("labels must be a contiguous int32 array of the image's shape")
    pitch = img.strides[0] if H > 1 else W
    import torch

    dev = torch.device("cuda", torch.cuda.current_device())
    st = _call("ccl_label_host_async", dev, img.ctypes.data, H, W, pitch, connectivity, labels.ctypes.data,
               _stream_ptr(stream, dev))
    _check(st, "ccl_label_host_async")


def ccl_get_device_status(stream=None) -> int:
    """Waits for the stream and returns (and clears) the device status code."""
    import torch

    dev = torch.device("cuda", torch.cuda.current_device())
    return _call("ccl_get_device_status", dev, _stream_ptr(stream, dev))


def ccl_release_stream(stream=None) -> None:
    """Frees the library's scratch, staging and batched graphs held for
    ``stream`` (``ccl_release_stream``); call before the stream goes away."""
    import torch

    dev = torch.device("cuda", torch.cuda.current_device())
    _check(_call("ccl_release_stream", dev, _stream_ptr(stream, dev)), "ccl_release_stream")


def ccl_debug_set_iteration_cap(cap: int) -> None:
    load().ccl_debug_set_iteration_cap(cap)


def ccl_debug_kernel_timing(enable: bool) -> None:
    load().ccl_debug_kernel_timing(1 if enable else 0)


def ccl_debug_kernel_times() -> dict:
    """Per-kernel ``{name: (total_ms, launches)}`` since timing was enabled."""
    lib = load()
    n = lib.ccl_debug_kernel_times(None, None, 0)
    ms = (ctypes.c_double * n)()
    cnt = (ctypes.c_longlong * n)()
    lib.ccl_debug_kernel_times(ms, cnt, n)
    return {lib.ccl_debug_kernel_name(k).decode(): (ms[k], cnt[k]) for k in range(n)}


def _batch_array(pairs):
    """ctypes array of CclImage from (image, labels) tensor pairs."""
    arr = (CclImage * max(1, len(pairs)))()
    for i, (img, lab) in enumerate(pairs):
        H, W, pitch = _image_args(img)
        _labels_for(img, lab)
        arr[i] = CclImage(img.data_ptr(), lab.data_ptr(), H, W, pitch)
    return arr


def ccl_label_batched(pairs, connectivity: int = 8, stream=None, tile: int | None = None):
    """Label a batch of ``(image, labels)`` CUDA tensor pairs in one launch
    sequence (``ccl_label_batched``; ``ccl_label_batched_tile`` when ``tile``
    is given).  Returns the labels tensors."""
    import torch

    dev = pairs[0][0].device if pairs else torch.device("cuda", torch.cuda.current_device())
    arr = _batch_array(pairs)
    sp = _stream_ptr(stream, dev)
    if tile is None:
        st = _call("ccl_label_batched", dev, arr, len(pairs), connectivity, sp)
    else:
        st = _call("ccl_label_batched_tile", dev, arr, len(pairs), connectivity, tile, sp)
    _check(st, "ccl_label_batched")
    return [lab for _, lab in pairs]


def ccl_autotune_batched(pairs, connectivity: int = 8, stream=None) -> int:
    """Time every block shape on the batch, remember and return the fastest."""
    arr = _batch_array(pairs)
    out = ctypes.c_int(-1)
    dev = pairs[0][0].device
    _check(_call("ccl_autotune_batched", dev, arr, len(pairs), connectivity, _stream_ptr(stream, dev),
                 ctypes.byref(out)), "ccl_autotune_batched")
    return out.value


def ccl_batched_tile(pairs, connectivity: int = 8) -> int:
    arr = _batch_array(pairs)
    out = ctypes.c_int(-1)
    _check(_call("ccl_batched_tile", pairs[0][0].device, arr, len(pairs), connectivity, ctypes.byref(out)),
           "ccl_batched_tile")
    return out.value


def ccl_tile_names() -> list:
    lib = load()
    return [lib.ccl_tile_name(i).decode() for i in range(lib.ccl_tile_count())]


def ccl_server_frame_bytes(H: int, W: int) -> int:
    """Arena bytes one H x W frame needs when served alone (``ccl_server_frame_bytes``)."""
    out = ctypes.c_size_t(0)
    _check(load().ccl_server_frame_bytes(H, W, ctypes.byref(out)), "ccl_server_frame_bytes")
    return out.value


class CclServer:
    """Binding of the ``ccl_server_*`` entry points.  Host frames are numpy
    arrays (uint8 image, int32 labels of the same shape); the server keeps a
    reference to both until the request is collected with ``wait``."""

    def __init__(self, max_slots=64, n_streams=4, max_batch=32, hbm_budget_bytes=4 << 30, device=0):
        cfg = CclServerConfig(max_slots, n_streams, max_batch, device, hbm_budget_bytes)
        handle = ctypes.c_void_p()
        _check(load().ccl_server_create(ctypes.byref(cfg), ctypes.byref(handle)), "ccl_server_create")
        self._h = handle
        self._keep = {}

    def submit(self, img: np.ndarray, labels: np.ndarray, connectivity: int = 8) -> int:
        if img.dtype != np.uint8 or img.ndim != 2 or (img.shape[0] > 1 and img.strides[1] != 1):
            raise ValueError("image must be a 2D uint8 array with contiguous rows")
        if labels.dtype != np.int32 or labels.shape != img.shape or not labels.flags.c_contiguous:
            raise ValueError("labels must be a contiguous int32 array of the image's shape")
        H, W = img.shape
        pitch = img.strides[0] if H > 1 else W
        t = ctypes.c_uint64(0)
        _check(load().ccl_server_submit(self._h, img.ctypes.data, H, W, pitch, connectivity, labels.ctypes.data,
                                        ctypes.byref(t)), "ccl_server_submit")
        self._keep[t.value] = (img, labels)
        return t.value

    def wait(self, ticket: int, timeout_ms: int = -1) -> int:
        st = load().ccl_server_wait(self._h, ticket, timeout_ms)
        if st != CCL_ERR_BUSY:
            self._keep.pop(ticket, None)
        return st

    def poll(self, ticket: int) -> int:
        return load().ccl_server_poll(self._h, ticket)

    def stats(self) -> dict:
        st = CclServerStats()
        _check(load().ccl_server_stats(self._h, ctypes.byref(st)), "ccl_server_stats")
        return {name: getattr(st, name) for name, _ in CclServerStats._fields_}

    def reset_stats(self) -> None:
        _check(load().ccl_server_reset_stats(self._h), "ccl_server_reset_stats")

    def close(self) -> None:
        if self._h:
            load().ccl_server_destroy(self._h)
            self._h = None
            self._keep.clear()

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()
