"""Seeded random GPU parity sweep: single counts in every mode (repeated, so
the launch-graph replay is exercised), batches, randomised copies in both
modes and on both plain kernels, and the host-buffer entry point, over mixed
graph families (random densities, power-law, hub stars, repeated arcs and
unsorted rows), each result compared element by element with the oracle."""
import numpy as np
import pytest

import oracle
import synth
from tests.gpu_helpers import csr_arrays
from tests.graph_helpers import random_digraph

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("seed,iterations", [(101, 60), (202, 60)])
def test_random_sweep(seed, iterations):
    import torch
    from paper_1203_3415_gb300 import build
    build.build()
    import paper_1203_3415_gb300 as acc
    rng = np.random.default_rng(seed)
    cnt = acc.Counter(0)
    checks = 0

    def make_graph():
        kind = rng.integers(0, 5)
        if kind == 0:
            n = int(rng.integers(0, 80))
            s, d = random_digraph(rng, n, p=float(rng.random()) ** 2, recip=float(rng.random()))
        elif kind == 1:
            n = int(rng.integers(200, 6000))
            m = int(n * rng.uniform(1.5, 5))
            g = synth.chung_lu(n, m, float(rng.uniform(2.0, 2.6)), int(rng.integers(20, 300)), int(rng.integers(0, 40)), int(rng.integers(1, 10**6)))
            s, d = g.src, g.dst
        elif kind == 2:
            n = int(rng.integers(50, 3000))
            m = int(n * rng.uniform(1, 4))
            g = synth.erdos_renyi(n, m, int(rng.integers(0, 50)), int(rng.integers(1, 10**6)))
            s, d = g.src, g.dst
        elif kind == 3:  # stars with a few hubs
            n = int(rng.integers(100, 2000))
            h = int(rng.integers(1, 5))
            src = []
            dst = []
            for hub in range(h):
                leaves = rng.choice(np.arange(h, n), size=int(rng.integers(10, min(400, n - h))), replace=False)
                for l in leaves:
                    if rng.random() < 0.5:
                        src.append(hub)
                        dst.append(int(l))
                    else:
                        src.append(int(l))
                        dst.append(hub)
            pairs = np.unique(np.array(list(zip(src, dst)), dtype=np.int64).reshape(-1, 2), axis=0)
            s, d = pairs[:, 0].astype(np.int32), pairs[:, 1].astype(np.int32)
        else:  # repeated arcs and unsorted rows
            n = int(rng.integers(2, 300))
            m = int(rng.integers(0, 3 * n))
            s = rng.integers(0, n, m).astype(np.int32)
            d = rng.integers(0, n, m).astype(np.int32)
            keep = s != d
            s, d = s[keep], d[keep]
        return n, np.asarray(s, np.int32), np.asarray(d, np.int32)

    def oracle_count(n, s, d, k):
        return oracle.count(n, s, d, k, threads=oracle.max_threads())

    for _ in range(iterations):
        test = rng.integers(0, 4)
        if test == 0:  # single counts, repeated (replay), modes
            n, s, d = make_graph()
            k = int(rng.choice([3, 4, 5], p=[0.4, 0.4, 0.2]))
            if k == 5 and len(s) > 12000: k = 4
            mode = int(rng.integers(0, 3))
            cnt.set_mode(mode)
            r, c = csr_arrays(n, s, d)
            if rng.random() < 0.5:  # shuffle within rows
                for v in range(min(n, 50)):
                    a, b = r[v], r[v + 1]
                    c[a:b] = rng.permutation(c[a:b])
            rt, ct = torch.from_numpy(r).cuda(), torch.from_numpy(c).cuda()
            want = oracle_count(n, s, d, k)
            out = torch.zeros(acc.NUM_CLASSES[k], dtype=torch.int64, device='cuda')
            for rep in range(int(rng.integers(1, 4))):
                cnt.count(rt, ct, n, k, counts=out)
                got = out.cpu().numpy()
                assert np.array_equal(got, want), ('single', n, len(s), k, mode, rep)
                checks += 1
        elif test == 1:  # batch
            k = int(rng.choice([3, 4]))
            cnt.set_mode(int(rng.integers(0, 3)))
            gs = [make_graph() for _ in range(int(rng.integers(1, 12)))]
            dev = []
            for n, s, d in gs:
                r, c = csr_arrays(n, s, d)
                dev.append((torch.from_numpy(r).cuda(), torch.from_numpy(c).cuda(), n))
            cnt.prepare_batch(dev, k)
            got = cnt.run_batch().cpu().numpy()
            for i, (n, s, d) in enumerate(gs):
                assert np.array_equal(got[i], oracle_count(n, s, d, k)), ('batch', i, k)
            checks += len(gs)
        elif test == 2:  # randomise
            gs = []
            for _ in range(int(rng.integers(1, 5))):
                n, s, d = make_graph()
                pairs = np.unique(np.stack([s.astype(np.int64), d.astype(np.int64)], 1).reshape(-1, 2), axis=0) if len(s) else np.zeros((0, 2), np.int64)
                gs.append((n, pairs[:, 0].astype(np.int32), pairs[:, 1].astype(np.int32)))
            mode = int(rng.integers(0, 2))
            cnt.set_randomise_memory(0 if rng.random() < 0.3 else 16 << 30)
            dev = []
            for n, s, d in gs:
                r, c = csr_arrays(n, s, d)
                dev.append((torch.from_numpy(r).cuda(), torch.from_numpy(c).cuda(), n))
            R = int(rng.integers(1, 4))
            q = int(rng.integers(0, 4))
            seeds = [int(rng.integers(0, 2**63)) for _ in gs]
            out, accd = cnt.randomise(dev, R, seeds, attempts_per_arc=q, mode=mode)
            out = out.cpu().numpy()
            accd = accd.cpu().numpy()
            off = 0
            for gi, ((n, s, d), (rt, ct, _)) in enumerate(zip(gs, dev)):
                rp, cl = rt.cpu().numpy(), ct.cpu().numpy()
                m = len(cl)
                for r_ in range(R):
                    want, wa = oracle.swap_randomise(n, rp, cl, q * m, seeds[gi] + r_, mode)
                    assert np.array_equal(out[off + r_ * m: off + (r_ + 1) * m], want) and accd[gi, r_] == wa, ('rand', gi, r_, mode)
                    checks += 1
                off += R * m
        else:  # host entry point
            n, s, d = make_graph()
            k = int(rng.choice([3, 4]))
            cnt.set_mode(int(rng.integers(0, 3)))
            r, c = csr_arrays(n, s, d)
            for _ in range(2):
                got = cnt.count_host(r, c, n, k)
                assert np.array_equal(got, oracle_count(n, s, d, k)), ('host', n, k)
                checks += 1
    cnt.close()
    assert checks >= iterations
