"""ccl_label_noalloc: the labelling entry point for callers that may not
allocate device memory while they run (for example a program whose memory
pool owns the whole GPU, or a loop that must not let cudaMalloc/cudaFree block
the device).  Its scratch is the library's fixed per-device array.

The GPU test calls it through the C ABI three times in a row -- a large image,
a small one, then the large one again -- so that every call runs over what
the previous call left in the shared array.  Each call's labels must equal
those of ``ccl_label`` and of the CPU oracle bit for bit (labels are integers,
so the tolerance is zero).  The file sorts last so that a run stopping at the
first failure has already run every other test; it passes alone in a fresh
process as well.
"""
import pytest

from paper_1712_09789_gb300 import build as ccl_build
from paper_1712_09789_gb300 import ccl, synth


def test_noalloc_declared_and_exported_without_gpu():
    ccl_build.build()
    lib = ccl.load()
    assert hasattr(lib, "ccl_label_noalloc")
    assert ccl.ccl_noalloc_max_workspace_bytes() == 64 << 20
    # arguments are checked before any device work
    assert lib.ccl_label_noalloc(0x1000, 4, 4, 4, 6, 0x900000, None) == ccl.CCL_ERR_INVALID_ARG
    # too large for the fixed scratch: rejected, nothing enqueued
    assert ccl.ccl_workspace_size(8192, 8192) > ccl.ccl_noalloc_max_workspace_bytes()
    assert lib.ccl_label_noalloc(0x1000, 8192, 8192, 8192, 8, 0x90000000, None) == ccl.CCL_ERR_UNSUPPORTED


@pytest.mark.gpu
def test_noalloc_matches_ccl_label_and_oracle_on_calls_in_a_row():
    import numpy as np
    import torch

    import oracle

    ccl_build.build()
    large = (synth.smoothed(4096, 4096, 8.0, 0.5, 12), 4)
    small = (synth.bernoulli(1000, 1537, 0.5, 11), 8)
    cases = [large, small, large]
    # the 4096 x 4096 image needs about a third of the 64 MiB scratch
    assert ccl.ccl_workspace_size(4096, 4096) <= ccl.ccl_noalloc_max_workspace_bytes()
    imgs = [torch.from_numpy(img).cuda() for img, _ in cases]
    outs = [torch.full(img.shape, -7, dtype=torch.int32, device="cuda") for img in imgs]
    torch.cuda.synchronize()
    for (img_np, conn), img, out in zip(cases, imgs, outs):
        ccl.ccl_label_noalloc(img, conn, labels=out)
    assert ccl.ccl_get_device_status() == ccl.CCL_OK
    for k, ((img_np, conn), img, out) in enumerate(zip(cases, imgs, outs)):
        want = ccl.ccl_label(img, conn)
        assert ccl.ccl_get_device_status() == ccl.CCL_OK
        assert torch.equal(out, want), f"call {k}: {tuple(img.shape)} conn={conn}"
        np.testing.assert_array_equal(out.cpu().numpy(), oracle.label(img_np, conn), err_msg=f"call {k}")
    # an image beyond the scratch limit is refused with a clear status
    big = torch.zeros((8192, 8192), dtype=torch.uint8, device="cuda")
    with pytest.raises(ccl.CclError) as e:
        ccl.ccl_label_noalloc(big, 8)
    assert e.value.status == ccl.CCL_ERR_UNSUPPORTED
