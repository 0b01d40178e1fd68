"""Reader for the stored oracle counts (plain text, no oracle import)."""
import numpy as np


def read_counts(path):
    """(header dict, int64 counts) of a file written by write_counts."""
    hdr = {}
    rows = []
    with open(path) as f:
        for line in f:
            if line.startswith("# "):
                key, _, val = line[2:].strip().partition(" ")
                hdr[key] = val
            elif line.strip():
                c, v = line.split()
                rows.append((int(c), int(v)))
    counts = np.zeros(int(hdr["classes"]), dtype=np.int64)
    for c, v in rows:
        counts[c] = v
    assert int(counts.sum()) == int(hdr["total"])
    return hdr, counts
