"""Write the stored expectations for the full-size workloads.

Calls only the CPU oracle (``oracle/``) and the seeded generators
(``synth/``); nothing here touches the CUDA path.  Each output file records
the workload, the SHA-256 of the generated arc list (so a test can tell that
it regenerated the same graph), N_k and every nonzero class count.

    python tests/golden/make_golden.py [--threads T] [--only NAME ...] [--batch] [--serving] [--million]
"""
import argparse
import hashlib
import os
import sys
import time

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

import oracle  # noqa: E402
import synth  # noqa: E402
from tests.golden.golden_io import read_counts  # noqa: E402,F401

WORKLOADS = {
    "er_n1000_m5000_k3": (synth.er_k3, 3),
    "chung_lu_n20000_m100000_k4": (synth.chung_lu_k4, 4),
    "regulatory_n5000_m15000_k5": (synth.regulatory_k5, 5),
}


def write_counts(path, name, g, k, counts, seconds, threads):
    with open(path, "w") as f:
        f.write(f"# workload {name}\n")
        f.write(f"# graph {g.name} n={g.n} m={g.m} sha256={synth.graph_digest(g)}\n")
        f.write(f"# k {k}\n")
        f.write(f"# classes {len(counts)}\n")
        f.write(f"# total {int(counts.sum())}\n")
        f.write(f"# oracle ESU, {threads} threads, {seconds:.1f} s\n")
        for c, v in enumerate(counts):
            if v:
                f.write(f"{c} {int(v)}\n")


def counts_digest(counts):
    """SHA-256 of an int64 count block (little-endian, row-major)."""
    return hashlib.sha256(np.ascontiguousarray(counts, dtype="<i8").tobytes()).hexdigest()


def graphs_digest(graphs):
    h = hashlib.sha256()
    for g in graphs:
        h.update(synth.graph_digest(g).encode())
    return h.hexdigest()


def oracle_randomisation(base, b, i):
    """Copy i of batch base b by the oracle's double-edge swaps: 3m attempts
    on the base's out-CSR positions, seed 10^6 (b+1) + i."""
    rowptr, col = base.csr()
    src = np.repeat(np.arange(base.n, dtype=np.int32), np.diff(rowptr))
    dst, _ = oracle.swap_randomise(base.n, rowptr, col, 3 * base.m, 1_000_000 * (b + 1) + i)
    return synth.Graph(base.n, src, dst, f"batch_base{b}_rand{i}")


def make_batch_golden(path, threads, n_rand=synth.BATCH_RANDOMISATIONS):
    """Batched k=4 workload: per base graph, the digest of its 1 + n_rand
    graphs, the digest and total of their int64 counts [1 + n_rand, 199] and
    the Z-scores of the base against its randomisations (hex doubles)."""
    with open(path, "w") as f:
        f.write("# workload batch_k4: 8 directed Chung-Lu bases (exponent 2.3, m = 4n) x "
                f"(1 + {n_rand} degree-preserving randomisations, 3m swap attempts "
                "on out-CSR positions, copy i of base b seeded 10^6 (b+1) + i)\n")
        f.write(f"# oracle ESU, {threads} threads; one line per base:\n")
        f.write("# base n m graphs_sha256 counts_sha256 total z_hex[199]\n")
        for b in range(synth.BATCH_BASES):
            base = synth.batch_base(b)
            graphs = [base] + [oracle_randomisation(base, b, i) for i in range(n_rand)]
            t = time.time()
            counts = np.stack([oracle.count(g.n, g.src, g.dst, 4, threads=threads) for g in graphs])
            z = oracle.zscores(counts[0], counts[1:])
            f.write(f"{b} {base.n} {base.m} {graphs_digest(graphs)} {counts_digest(counts)} "
                    f"{int(counts.sum())} {' '.join(float(x).hex() for x in z)}\n")
            f.flush()
            print(f"batch base {b}: n={base.n} total={int(counts.sum())} in {time.time() - t:.1f} s", flush=True)


def make_serving_pool_golden(path, threads):
    """Serving tests' graph pool: per graph and k = 3, 4, 5, the graph's
    digest, N_k and the digest of its int64 counts."""
    from tests.graph_helpers import serving_test_pool
    with open(path, "w") as f:
        f.write("# serving test pool: directed Chung-Lu graphs (exponent 2.2, cap 120, 10% reciprocal)\n")
        f.write(f"# oracle ESU, {threads} threads; one line per graph and k:\n")
        f.write("# graph k n m graph_sha256 total counts_sha256\n")
        for gi, g in enumerate(serving_test_pool()):
            for k in (3, 4, 5):
                t = time.time()
                counts = oracle.count(g.n, g.src, g.dst, k, threads=threads)
                f.write(f"{gi} {k} {g.n} {g.m} {synth.graph_digest(g)} {int(counts.sum())} "
                        f"{counts_digest(counts)}\n")
                f.flush()
                print(f"serving graph {gi} k={k}: N_k = {int(counts.sum())} in {time.time() - t:.1f} s", flush=True)


def million_vertex_graph():
    """Sparse directed Chung-Lu graph above the dense block's size limit:
    10^6 vertices, 3 * 10^6 arcs, exponent 2.3, degree cap 100, 10%
    reciprocal, seed 3600."""
    return synth.chung_lu(1_000_000, 3_000_000, 2.3, 100, 10, 3600)


def make_million_golden(path, threads):
    """The million-vertex graph at k = 3 and 4: graph digest, N_k and the
    digest of its int64 counts."""
    g = million_vertex_graph()
    with open(path, "w") as f:
        f.write("# sparse directed Chung-Lu graph, n = 10^6, m = 3 10^6 (exponent 2.3, cap 100, 10% reciprocal,"
                " seed 3600)\n")
        f.write(f"# oracle ESU, {threads} threads; one line per k:\n")
        f.write("# k n m graph_sha256 total counts_sha256\n")
        for k in (3, 4):
            t = time.time()
            counts = oracle.count(g.n, g.src, g.dst, k, threads=threads)
            f.write(f"{k} {g.n} {g.m} {synth.graph_digest(g)} {int(counts.sum())} {counts_digest(counts)}\n")
            f.flush()
            print(f"million-vertex graph k={k}: N_k = {int(counts.sum())} in {time.time() - t:.1f} s", flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--threads", type=int, default=oracle.max_threads())
    ap.add_argument("--only", nargs="*")
    ap.add_argument("--batch", action="store_true", help="also write the batched k=4 expectations")
    ap.add_argument("--serving", action="store_true", help="also write the serving test pool's expectations")
    ap.add_argument("--million", action="store_true", help="also write the million-vertex graph's expectations")
    args = ap.parse_args()
    if args.million:
        make_million_golden(os.path.join(HERE, "million_vertices.txt"), args.threads)
    if args.batch:
        make_batch_golden(os.path.join(HERE, "batch_k4.txt"), args.threads)
    if args.serving:
        make_serving_pool_golden(os.path.join(HERE, "serving_pool.txt"), args.threads)
    if args.only is not None and not args.only:
        return
    for name, (make, k) in WORKLOADS.items():
        if args.only and name not in args.only:
            continue
        g = make()
        t = time.time()
        counts = oracle.count(g.n, g.src, g.dst, k, threads=args.threads)
        dt = time.time() - t
        write_counts(os.path.join(HERE, f"{name}.txt"), name, g, k, counts, dt, args.threads)
        print(f"{name}: N_{k} = {int(counts.sum())} in {dt:.1f} s", flush=True)


if __name__ == "__main__":
    main()
