"""Loader for the hand-drawn worked examples in this folder.

Each ``*.txt`` file holds comment lines (``#``), a ``conn`` line listing the
connectivities it covers, an ``image`` block of 0/1 rows and one
``labels <conn>`` block per connectivity with the hand-computed canonical
labels.
"""
import glob
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))


def load(path):
    img_rows, labels, conns = [], {}, []
    cur = None
    with open(path) as f:
        for raw in f:
            line = raw.strip()
            if not line or line.startswith("#"):
                continue
            if line.startswith("conn"):
                conns = [int(v) for v in line.split()[1:]]
            elif line == "image":
                cur = img_rows
            elif line.startswith("labels"):
                cur = labels.setdefault(int(line.split()[1]), [])
            else:
                cur.append([int(v) for v in line.split()])
    img = np.array(img_rows, dtype=np.uint8)
    return img, {c: np.array(labels[c], dtype=np.int32) for c in conns}


def all_fixtures():
    return sorted(glob.glob(os.path.join(HERE, "*.txt")))
