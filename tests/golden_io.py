"""Reader for the hand-worked example fixtures under tests/golden/."""
import os

import numpy as np

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def hand_examples():
    out, cur = [], None
    with open(os.path.join(GOLDEN, "hand_examples.txt")) as f:
        for line in f:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            key, _, rest = line.partition(" ")
            if key == "example":
                cur = dict(name=rest, rows=[], L=[], trace=[])
            elif key == "params":
                cur["n"], cur["m"], cur["minsup"], cur["M"] = map(int, rest.split())
            elif key == "row":
                cur["rows"].append(sorted(int(x) for x in rest.split()))
            elif key == "L":
                its, _, s = rest.partition(":")
                cur["L"].append((tuple(int(x) for x in its.split()), int(s)))
            elif key == "trace":
                cur["trace"].append([int(x) for x in rest.split()])
            elif key == "tests":
                cur["tests"] = int(rest)
            elif key == "end":
                assert len(cur["rows"]) == cur["n"]
                out.append(cur)
    return out


def to_csr(rows):
    rows = [sorted(set(int(x) for x in r)) for r in rows]
    row_ptr = np.zeros(len(rows) + 1, dtype=np.uint64)
    row_ptr[1:] = np.cumsum([len(r) for r in rows]) if rows else []
    items = np.array([x for r in rows for x in r] or [], dtype=np.uint32)
    return row_ptr, items
