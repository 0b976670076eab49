"""Two host threads label images of growing size on the same stream through
``ccl_label``.  Each call that needs a larger library scratch buffer frees
the old one; the library holds its lock until a call's kernels are on the
stream, so no call can launch on a buffer another thread has just freed.
Every result must equal the CPU oracle."""
import threading

import numpy as np
import pytest

import oracle
from paper_1712_09789_gb300 import ccl, synth


@pytest.mark.gpu
def test_two_threads_growing_sizes_on_one_stream():
    import torch

    ccl.load()
    sizes = [(64 + 97 * k, 80 + 131 * k) for k in range(12)]
    imgs = {t: [synth.bernoulli(h, w, 0.45 + 0.05 * t, 100 * t + k) for k, (h, w) in enumerate(sizes)]
            for t in (0, 1)}
    dev = {t: [torch.from_numpy(im).cuda() for im in imgs[t]] for t in (0, 1)}
    outs = {t: [torch.empty(im.shape, dtype=torch.int32, device="cuda") for im in imgs[t]] for t in (0, 1)}
    stream = torch.cuda.current_stream()
    torch.cuda.synchronize()
    errors = []
    start = threading.Barrier(2)

    def worker(t):
        try:
            torch.cuda.set_device(0)
            start.wait()
            for k in range(len(sizes)):
                ccl.ccl_label(dev[t][k], 8 if (k + t) % 2 else 4, labels=outs[t][k], stream=stream)
        except Exception as exc:  # reported below
            errors.append(exc)

    th = [threading.Thread(target=worker, args=(t,)) for t in (0, 1)]
    for x in th:
        x.start()
    for x in th:
        x.join()
    assert not errors, errors
    assert ccl.ccl_get_device_status(stream) == ccl.CCL_OK
    for t in (0, 1):
        for k in range(len(sizes)):
            want = oracle.label(imgs[t][k], 8 if (k + t) % 2 else 4)
            np.testing.assert_array_equal(outs[t][k].cpu().numpy(), want, err_msg=f"thread {t} image {k}")


@pytest.mark.gpu
def test_release_stream_then_reuse():
    import torch

    s = torch.cuda.Stream()
    img_np = synth.bernoulli(700, 900, 0.5, 5)
    img = torch.from_numpy(img_np).cuda()
    with torch.cuda.stream(s):
        a = ccl.ccl_label(img, 8, stream=s)
        ccl.ccl_release_stream(s)
        b = ccl.ccl_label(img, 8, stream=s)  # allocates afresh
    s.synchronize()
    want = oracle.label(img_np, 8)
    np.testing.assert_array_equal(a.cpu().numpy(), want)
    np.testing.assert_array_equal(b.cpu().numpy(), want)


@pytest.mark.gpu
def test_host_async_on_three_streams():
    """ccl_label_host_async: images enqueued round-robin on three streams from
    page-locked host buffers; each result equals the oracle."""
    import torch

    imgs = [synth.bernoulli(300 + 111 * k, 517 + 77 * k, 0.3 + 0.1 * (k % 5), k) for k in range(9)]
    pin_in = [torch.from_numpy(im).pin_memory().numpy() for im in imgs]
    pin_out = [torch.empty(im.shape, dtype=torch.int32).pin_memory().numpy() for im in imgs]
    streams = [torch.cuda.Stream() for _ in range(3)]
    for k in range(len(imgs)):
        ccl.ccl_label_host_async(pin_in[k], pin_out[k], 8 if k % 2 else 4, stream=streams[k % 3])
    for s in streams:
        s.synchronize()
    assert ccl.ccl_get_device_status() == ccl.CCL_OK
    for k, im in enumerate(imgs):
        np.testing.assert_array_equal(pin_out[k], oracle.label(im, 8 if k % 2 else 4), err_msg=f"image {k}")
    for s in streams:
        ccl.ccl_release_stream(s)
