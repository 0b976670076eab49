"""Back-to-back ``ccl_label`` calls on one stream.  Under 8-connectivity a
call's step 1 may start while the previous call's write-out still runs
(programmatic dependent launch), on the other half of the library scratch.
Every result must equal the CPU oracle: calls of growing, shrinking and equal
sizes, 4- and 8-connected calls mixed, and an image that is the previous
call's label buffer read as bytes (the chained start must be refused there)."""
import numpy as np
import pytest

import oracle
from paper_1712_09789_gb300 import ccl, synth

pytestmark = pytest.mark.gpu


def test_back_to_back_calls_of_mixed_sizes():
    import torch

    s = torch.cuda.Stream()
    shapes = [(2048, 2048), (4096, 4096), (512, 700), (4096, 4096), (3000, 1000), (8192, 8192), (64, 64),
              (8192, 8192), (1000, 3000), (2048, 2048)]
    conns = [8, 8, 8, 4, 8, 8, 8, 8, 4, 8]
    imgs = [synth.bernoulli(h, w, 0.5, 40 + i) for i, (h, w) in enumerate(shapes)]
    dev = [torch.from_numpy(im).cuda() for im in imgs]
    outs = [torch.empty(im.shape, dtype=torch.int32, device="cuda") for im in imgs]
    torch.cuda.synchronize()
    with torch.cuda.stream(s):
        for _ in range(2):
            for i in range(len(imgs)):
                ccl.ccl_label(dev[i], conns[i], labels=outs[i], stream=s)
    s.synchronize()
    assert ccl.ccl_get_device_status(s) == ccl.CCL_OK
    for i in range(len(imgs)):
        np.testing.assert_array_equal(outs[i].cpu().numpy(), oracle.label(imgs[i], conns[i]), err_msg=f"call {i}")


def test_image_that_is_the_previous_calls_labels():
    import torch

    img_np = synth.bernoulli(1024, 1024, 0.5, 3)
    img = torch.from_numpy(img_np).cuda()
    lab = ccl.ccl_label(img, 8)
    # the labels' bytes as a 1024 x 4096 image (nonzero bytes are foreground)
    as_bytes = lab.view(torch.uint8)
    again = ccl.ccl_label(as_bytes, 8)
    torch.cuda.synchronize()
    assert ccl.ccl_get_device_status() == ccl.CCL_OK
    want_lab = oracle.label(img_np, 8)
    np.testing.assert_array_equal(lab.cpu().numpy(), want_lab)
    np.testing.assert_array_equal(again.cpu().numpy(), oracle.label(want_lab.view(np.uint8), 8))
