"""The Python binding makes the tensors' device current around every C-ABI
call that uses per-device library state (scratch buffers, the no-allocation
array's address, batched runners).  Checked on the host: a fake library
records which device was current when it was called."""
import contextlib
import re

from paper_1712_09789_gb300 import ccl

# entry points whose C side looks up state of the current device
DEVICE_CALLS = (
    "ccl_label", "ccl_label_ws", "ccl_label_host", "ccl_label_host_async", "ccl_label_noalloc",
    "ccl_label_3d", "ccl_label_variant", "ccl_component_stats", "ccl_label_batched",
    "ccl_label_batched_tile", "ccl_autotune_batched", "ccl_batched_tile", "ccl_get_device_status",
    "ccl_release_stream",
)


class _FakeLib:
    def __init__(self, state):
        self.state = state

    def __getattr__(self, name):
        def fn(*args):
            self.state["calls"].append((name, self.state["current"], args))
            return 0
        return fn


def test_call_runs_with_the_given_device_current(monkeypatch):
    state = {"current": "cuda:0", "calls": []}

    @contextlib.contextmanager
    def guard(device):
        prev = state["current"]
        state["current"] = str(device)
        try:
            yield
        finally:
            state["current"] = prev

    monkeypatch.setattr(ccl, "_device_guard", guard)
    monkeypatch.setattr(ccl, "load", lambda: _FakeLib(state))
    assert ccl._call("ccl_label", "cuda:1", 11, 22) == 0
    assert state["calls"] == [("ccl_label", "cuda:1", (11, 22))]
    assert state["current"] == "cuda:0"  # restored afterwards


def test_every_device_call_goes_through_the_guard():
    src = open(ccl.__file__).read()
    for name in DEVICE_CALLS:
        # never called straight on the library object
        assert not re.search(r"(load\(\)|lib)\." + name + r"\(", src), name
    for name in DEVICE_CALLS:
        if name in ("ccl_label_host_async",) or f'"{name}"' in src:
            assert f'_call("{name}"' in src, name
