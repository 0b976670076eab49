"""Serving path (ccl_server_*): continuous batching of host frames.

The central check: every frame's labels are the same whether the frame is
served alone or in a mix of concurrent requests of different sizes, and equal
to the CPU oracle (labels are integers: bit-exact)."""
import threading

import numpy as np
import pytest

import oracle
from paper_1712_09789_gb300 import build as ccl_build
from paper_1712_09789_gb300 import ccl, synth

SIZES = synth.SERVING_SIZES


def pinned_frames(n, seed, sizes=SIZES):
    import torch

    g = np.random.default_rng(seed)
    frames = []
    for i in range(n):
        H, W = sizes[int(g.integers(0, len(sizes)))]
        img = synth.smoothed(H, W, 6.0, float(g.uniform(0.3, 0.6)), seed * 100 + i)
        t = torch.from_numpy(img).pin_memory()
        frames.append(t.numpy())
    return frames


def settled_stats(srv, timeout_s=5.0):
    """Server statistics once every batch has been retired: a request is
    complete when its labels are in host memory, and its batch's scratch is
    returned to the arena just after the batch's last copy."""
    import time

    t0 = time.monotonic()
    while True:
        st = srv.stats()
        if (st["arena_used_bytes"] == 0 and st["in_flight"] == 0) or time.monotonic() - t0 > timeout_s:
            return st
        time.sleep(0.01)


def pinned_labels(shape):
    import torch

    return torch.empty(shape, dtype=torch.int32).pin_memory().numpy()


def test_server_argument_checks_without_gpu():
    ccl_build.build()
    lib = ccl.load()
    cfg = ccl.CclServerConfig(0, 1, 1, 0, 1 << 30)  # max_slots = 0
    h = ccl.ctypes.c_void_p()
    assert lib.ccl_server_create(ccl.ctypes.byref(cfg), ccl.ctypes.byref(h)) == ccl.CCL_ERR_INVALID_ARG
    cfg = ccl.CclServerConfig(4, 0, 1, 0, 1 << 30)  # no streams
    assert lib.ccl_server_create(ccl.ctypes.byref(cfg), ccl.ctypes.byref(h)) == ccl.CCL_ERR_INVALID_ARG
    cfg = ccl.CclServerConfig(4, 2, 8, 0, 1024)  # arena below 1 MiB
    assert lib.ccl_server_create(ccl.ctypes.byref(cfg), ccl.ctypes.byref(h)) == ccl.CCL_ERR_INVALID_ARG


def test_frame_bytes_counts_scratch_without_gpu():
    ccl_build.build()
    b = ccl.ccl_server_frame_bytes(1080, 1920)
    assert b > 1080 * 1920 * 5 and b % 256 == 0
    assert ccl.ccl_server_frame_bytes(2160, 3840) > 3.9 * b
    with pytest.raises(ccl.CclError):
        ccl.ccl_server_frame_bytes(0, 5)


@pytest.mark.gpu
def test_alone_equals_in_mix_equals_oracle():
    frames = pinned_frames(18, seed=1)
    conns = [8 if i % 3 else 4 for i in range(len(frames))]
    with ccl.CclServer(max_slots=8, n_streams=3, max_batch=4, hbm_budget_bytes=1 << 30) as srv:
        alone = []
        for f, c in zip(frames, conns):
            out = pinned_labels(f.shape)
            t = srv.submit(f, out, c)
            assert srv.wait(t) == ccl.CCL_OK
            alone.append(out.copy())
        # the mix: all at once from two submitting threads
        srv.reset_stats()
        outs = [pinned_labels(f.shape) for f in frames]
        tickets = [None] * len(frames)

        def submitter(idx):
            for i in idx:
                tickets[i] = srv.submit(frames[i], outs[i], conns[i])

        th = [threading.Thread(target=submitter, args=(range(k, len(frames), 2),)) for k in (0, 1)]
        for x in th:
            x.start()
        for x in th:
            x.join()
        for t in tickets:
            assert srv.wait(t) == ccl.CCL_OK
        st = settled_stats(srv)
        assert st["completed"] == len(frames) and st["rejected"] == 0
        assert 0 < st["p50_ms"] <= st["p99_ms"] <= st["max_ms"]
        # continuous batching, shown by the server's own records: some batch
        # held several requests, several batches were on the device at once,
        # and some batch's device span (copy-in to copy-out, CUDA events)
        # overlapped another's
        assert st["multi_request_batches"] >= 1 and st["max_batch_requests"] >= 2
        assert st["max_batches_in_flight"] >= 2
        assert st["overlapped_batches"] >= 1
        assert 0 < st["label_p50_ms"] <= st["label_p99_ms"]
        assert 0 <= st["queue_p50_ms"] <= st["queue_p99_ms"]
        assert st["arena_used_bytes"] == 0
    for i, f in enumerate(frames):
        want = oracle.label(f, conns[i])
        np.testing.assert_array_equal(alone[i], want, err_msg=f"alone {i}")
        np.testing.assert_array_equal(outs[i], want, err_msg=f"mix {i}")


@pytest.mark.gpu
def test_admission_by_arena_memory():
    # the arena holds only two 1920x1080 frames (image, labels, their
    # labelling scratch and job table) at a time, so requests are admitted as
    # earlier ones release their memory
    frames = pinned_frames(10, seed=2, sizes=((1080, 1920),))
    per_frame = ccl.ccl_server_frame_bytes(1080, 1920)
    assert per_frame > 1080 * 1920 * 5  # the scratch is counted too
    with ccl.CclServer(max_slots=16, n_streams=4, max_batch=8, hbm_budget_bytes=2 * per_frame + 4096) as srv:
        outs = [pinned_labels(f.shape) for f in frames]
        tickets = [srv.submit(f, o, 8) for f, o in zip(frames, outs)]
        for t in tickets:
            assert srv.wait(t, 60000) == ccl.CCL_OK
        st = settled_stats(srv)
        assert st["completed"] == len(frames) and st["arena_used_bytes"] == 0
        assert st["max_batches_in_flight"] <= 2 and st["max_batch_requests"] <= 2
        # a frame larger than the whole arena is refused outright
        big = np.zeros((2160, 3840), np.uint8)
        with pytest.raises(ccl.CclError) as e:
            srv.submit(big, np.empty(big.shape, np.int32), 8)
        assert e.value.status == ccl.CCL_ERR_UNSUPPORTED
    for f, o in zip(frames, outs):
        np.testing.assert_array_equal(o, oracle.label(f, 8))


@pytest.mark.gpu
def test_ticket_semantics_and_bad_requests():
    f = pinned_frames(1, seed=3, sizes=((480, 640),))[0]
    with ccl.CclServer(max_slots=2, n_streams=1, max_batch=2, hbm_budget_bytes=64 << 20) as srv:
        out = pinned_labels(f.shape)
        t = srv.submit(f, out, 8)
        assert srv.wait(t) == ccl.CCL_OK
        assert srv.wait(t) == ccl.CCL_ERR_NOT_FOUND  # collected already
        assert srv.poll(123456789) == ccl.CCL_ERR_NOT_FOUND
        lib = ccl.load()
        tk = ccl.ctypes.c_uint64()
        # pitch < W and a bad connectivity are refused at submit
        assert lib.ccl_server_submit(srv._h, f.ctypes.data, 480, 640, 320, 8, out.ctypes.data,
                                     ccl.ctypes.byref(tk)) == ccl.CCL_ERR_INVALID_ARG
        assert lib.ccl_server_submit(srv._h, f.ctypes.data, 480, 640, 640, 5, out.ctypes.data,
                                     ccl.ctypes.byref(tk)) == ccl.CCL_ERR_INVALID_ARG
    np.testing.assert_array_equal(out, oracle.label(f, 8))


@pytest.mark.gpu
def test_destroy_with_queued_requests_cancels_them():
    """Host-side cancellation: many requests behind a single slot, then the
    server is destroyed; it finishes what is on the device, fails the rest
    and returns without hanging."""
    frames = pinned_frames(6, seed=4, sizes=((1080, 1920),))
    srv = ccl.CclServer(max_slots=1, n_streams=1, max_batch=1, hbm_budget_bytes=64 << 20)
    outs = [pinned_labels(f.shape) for f in frames]
    for f, o in zip(frames, outs):
        srv.submit(f, o, 8)
    srv.close()  # must return
