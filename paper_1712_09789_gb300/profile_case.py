"""Small, fixed workloads for profiler captures.

``python -m paper_1712_09789_gb300.profile_case --size 8192 --reps 3 --conn 8``
labels one seeded Bernoulli(p) image ``reps`` times through ``ccl_label`` on
cuda:0 and checks the device status.  With --size 8192 the input (67 MB) and
labels (268 MB) exceed L2 while the device holds well under 1 GB, so profiler
DRAM counters of one launch describe a full-size launch.

``--stats`` then runs ``ccl_component_stats`` on the labels: once with
capacity 0 (count only), then ``reps`` times with room for every record.

``--volume D`` labels a D x D x D Bernoulli(p) volume with ``ccl_label_3d``
instead, ``reps`` times with 6-connectivity at p = --p (default 0.3 there)
and then ``reps`` times with 26-connectivity at p = 0.5.
"""
from __future__ import annotations

import argparse
import sys


def main(argv=None) -> int:
    ap = argparse.ArgumentParser()
    ap.add_argument("--size", type=int, default=8192)
    ap.add_argument("--p", type=float, default=None)
    ap.add_argument("--seed", type=int, default=0)
    ap.add_argument("--conn", type=int, default=8, choices=(4, 8))
    ap.add_argument("--reps", type=int, default=3)
    ap.add_argument("--stats", action="store_true", help="component statistics of the labels as well")
    ap.add_argument("--volume", type=int, default=0, help="label a D^3 volume instead (6- then 26-connectivity)")
    args = ap.parse_args(argv)

    import torch

    from . import ccl, synth

    if args.volume:
        D = args.volume
        for p, conn in ((0.3 if args.p is None else args.p, 6), (0.5, 26)):
            vol = torch.from_numpy(synth.bernoulli3d(D, D, D, p, args.seed)).cuda()
            out = torch.empty((D, D, D), dtype=torch.int32, device="cuda")
            for _ in range(args.reps):
                ccl.ccl_label_3d(vol, conn, labels=out)
            status = ccl.ccl_get_device_status()
            if status != ccl.CCL_OK:
                print(f"device status {ccl.ccl_status_string(status)}", file=sys.stderr)
                return 1
            print(f"labelled {D}^3 p={p} conn={conn} x{args.reps}")
            del vol, out
        return 0

    p = 0.5 if args.p is None else args.p
    img = torch.from_numpy(synth.bernoulli(args.size, args.size, p, args.seed)).cuda()
    out = torch.empty((args.size, args.size), dtype=torch.int32, device="cuda")
    for _ in range(args.reps):
        ccl.ccl_label(img, args.conn, labels=out)
    status = ccl.ccl_get_device_status()
    if status != ccl.CCL_OK:
        print(f"device status {ccl.ccl_status_string(status)}", file=sys.stderr)
        return 1
    print(f"labelled {args.size}x{args.size} p={p} conn={args.conn} x{args.reps}: "
          f"{int(out.max().item())} max label")
    if args.stats:
        n = len(ccl.ccl_component_stats(out))
        for _ in range(args.reps):
            ccl.ccl_component_stats(out, capacity=n)
        print(f"statistics of {n} components x{args.reps + 1}")
    return 0


if __name__ == "__main__":
    sys.exit(main())
