"""Reader of the Philox4x32-10 known-answer vectors in tests/golden."""
import os

import numpy as np

KAT_PATH = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "philox4x32_10_kat.txt")


def philox_kat():
    """[(counter uint32[4], key uint32[2], expected uint32[4])] from the golden file."""
    rows = []
    for line in open(KAT_PATH):
        line = line.strip()
        if not line or line.startswith("#"):
            continue
        ctr, key, out = (np.array([int(w, 16) for w in part.split()], dtype=np.uint32)
                         for part in line.split(";"))
        assert ctr.size == 4 and key.size == 2 and out.size == 4
        rows.append((ctr, key, out))
    return rows
