"""A small, fixed labelling workload for profiler captures.

``python -m paper_1712_09789_gb300.profile_case --size 8192 --reps 3 --conn 8``
labels one seeded Bernoulli(p) image ``reps`` times through ``ccl_label`` on
cuda:0 and checks the device status.  With --size 8192 the input (67 MB) and
labels (268 MB) exceed L2 while the device holds well under 1 GB, so profiler
DRAM counters of one launch describe a full-size launch.
"""
from __future__ import annotations

import argparse
import sys


def main(argv=None) -> int:
    ap = argparse.ArgumentParser()
    ap.add_argument("--size", type=int, default=8192)
    ap.add_argument("--p", type=float, default=0.5)
    ap.add_argument("--seed", type=int, default=0)
    ap.add_argument("--conn", type=int, default=8, choices=(4, 8))
    ap.add_argument("--reps", type=int, default=3)
    args = ap.parse_args(argv)

    import torch

    from . import ccl, synth

    img = torch.from_numpy(synth.bernoulli(args.size, args.size, args.p, args.seed)).cuda()
    out = torch.empty((args.size, args.size), dtype=torch.int32, device="cuda")
    for _ in range(args.reps):
        ccl.ccl_label(img, args.conn, labels=out)
    status = ccl.ccl_get_device_status()
    if status != ccl.CCL_OK:
        print(f"device status {ccl.ccl_status_string(status)}", file=sys.stderr)
        return 1
    print(f"labelled {args.size}x{args.size} p={args.p} conn={args.conn} x{args.reps}: "
          f"{int(out.max().item())} max label")
    return 0


if __name__ == "__main__":
    sys.exit(main())
