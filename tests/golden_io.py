"""Reader for the hand-derived fixtures in tests/golden (text; '#' lines are the
derivation and citation)."""
import os

import numpy as np

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def read(name: str) -> dict:
    out = {}
    with open(os.path.join(GOLDEN, name)) as f:
        lines = [ln.strip() for ln in f if ln.strip() and not ln.lstrip().startswith("#")]
    i = 0
    while i < len(lines):
        tok = lines[i].split()
        key = tok[0]
        if key in ("image", "filter", "expected", "window"):
            h, w = int(tok[1]), int(tok[2])
            rows = [[float(v) for v in lines[i + 1 + r].split()] for r in range(h)]
            out[key] = np.array(rows, dtype=np.float64).reshape(h, w)
            i += 1 + h
        elif key == "border":
            out["border"] = tok[1]
            out["border_value"] = float(tok[2])
            i += 1
        else:
            out[key] = float(tok[1])
            i += 1
    return out


def names(prefix: str = ""):
    return sorted(n for n in os.listdir(GOLDEN) if n.endswith(".txt") and n.startswith(prefix))
