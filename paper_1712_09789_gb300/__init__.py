"""GB300-native block-based connected-components labelling.

The product is the C-ABI library ``libccl.so`` (declared in ``include/ccl.h``,
sources under ``csrc/``); ``ccl`` is its thin Python binding and ``synth``
draws the seeded synthetic inputs.
"""
from . import ccl  # noqa: F401  (the binding loads libccl.so on first use)

__all__ = ["ccl"]
