"""Loaders for the text fixtures in this folder."""
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))


def load_blocks(name):
    """Parse a key/value block file (``#`` comments, blank-line separated)."""
    blocks, cur = [], {}
    with open(os.path.join(HERE, name)) as f:
        for raw in f:
            line = raw.split("#", 1)[0].strip()
            if not line:
                if cur:
                    blocks.append(cur)
                    cur = {}
                continue
            key, _, val = line.partition(" ")
            cur[key] = val.strip()
    if cur:
        blocks.append(cur)
    return blocks


def hand_steps():
    out = []
    for b in load_blocks("hand_steps.txt"):
        sizes = tuple(int(v) for v in b["sizes"].split())
        periodic = bool(int(b["periodic"]))
        shape = sizes if periodic else tuple(n + 2 for n in sizes)
        out.append(dict(
            name=b["name"], dims=int(b["dims"]), sizes=sizes, periodic=periodic,
            coeffs=np.array([float(v) for v in b["coeffs"].split()]),
            T=int(b["T"]),
            init=np.array([float(v) for v in b["init"].split()]).reshape(shape),
            expected=np.array([float(v) for v in b["expected"].split()]).reshape(shape)))
    return out


def pcot_orders():
    out = []
    for b in load_blocks("pcot_order.txt"):
        sizes = tuple(int(v) for v in b["sizes"].split())
        vals = np.array([int(v) for v in b["order"].split()], dtype=np.int64)
        out.append(dict(name=b["name"], sizes=sizes, T=int(b["T"]),
                        leaf=tuple(int(v) for v in b["leaf"].split()),
                        order=vals.reshape(-1, len(sizes) + 1)))
    return out
