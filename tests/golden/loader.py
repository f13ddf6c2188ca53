"""Parse the plain-text golden fixtures in this folder.

A record is a header line ``name d0 [d1]`` followed by rows of numbers.
Lines starting with '#' are comments.
"""
from __future__ import annotations

import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))


def load(name: str) -> dict:
    out = {}
    with open(os.path.join(HERE, name)) as fh:
        lines = [ln.strip() for ln in fh if ln.strip() and not ln.lstrip().startswith("#")]
    k = 0
    while k < len(lines):
        head = lines[k].split()
        key, dims = head[0], [int(x) for x in head[1:]]
        nrows = dims[0] if len(dims) == 2 else 1
        rows = [[float(x) for x in lines[k + 1 + r].split()] for r in range(nrows)]
        arr = np.array(rows)
        out[key] = arr if len(dims) == 2 else arr.ravel()
        k += 1 + nrows
    return out
