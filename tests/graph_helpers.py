"""Small structured and random digraphs for tests (arc lists only)."""
import numpy as np


def _arr(src, dst):
    return np.asarray(src, dtype=np.int32), np.asarray(dst, dtype=np.int32)


def random_digraph(rng, n, p, recip):
    """Each unordered pair is linked with probability p; a linked pair is
    bidirected with probability recip, else one arc with a random direction."""
    src, dst = [], []
    for a in range(n):
        for b in range(a + 1, n):
            if rng.random() < p:
                if rng.random() < recip:
                    src += [a, b]; dst += [b, a]
                elif rng.random() < 0.5:
                    src.append(a); dst.append(b)
                else:
                    src.append(b); dst.append(a)
    return _arr(src, dst)


def bidirected(edges):
    src, dst = [], []
    for a, b in edges:
        src += [a, b]; dst += [b, a]
    return _arr(src, dst)


def complete_bidirected(n):
    return bidirected([(a, b) for a in range(n) for b in range(a + 1, n)])


def directed_path(n):
    return _arr(list(range(n - 1)), list(range(1, n)))


def directed_cycle(n):
    return _arr(list(range(n)), [(i + 1) % n for i in range(n)])


def transitive_tournament(n):
    return _arr([i for i in range(n) for j in range(i + 1, n)],
                [j for i in range(n) for j in range(i + 1, n)])


def out_star(leaves):
    return _arr([0] * leaves, list(range(1, leaves + 1)))


def in_star(leaves):
    return _arr(list(range(1, leaves + 1)), [0] * leaves)


def relabel(perm, src, dst):
    perm = np.asarray(perm)
    return _arr(perm[src], perm[dst])


def esu_scanned_entries(n, src, dst, k):
    """Neighbour entries the last two ESU levels read when they are counted
    from the extension lists: for every prefix P of k-2 vertices (root v = its
    smallest) with extension list E(P), the sum over x in E(P) of the
    neighbours of x above v.  Lists follow ESU's order: N(v) above v; then
    N(v) above w1 followed by the neighbours of w1 above v not adjacent to v;
    then level 2's list after w2 followed by the neighbours of w2 above v
    adjacent to neither v nor w1.  Vertex ids as given (no renumbering)."""
    nb = [set() for _ in range(n)]
    for a, b in zip(src, dst):
        if a != b:
            nb[a].add(b)
            nb[b].add(a)
    adj = [sorted(x) for x in nb]

    def above(x, v):
        return sum(1 for u in adj[x] if u > v)

    total = 0
    for v in range(n):
        E1 = [x for x in adj[v] if x > v]
        if k == 3:
            total += sum(above(x, v) for x in E1)
            continue
        for w1 in E1:
            E2 = [x for x in adj[v] if x > w1] + [u for u in adj[w1] if u > v and u not in nb[v]]
            if k == 4:
                total += sum(above(x, v) for x in E2)
                continue
            for j2, w2 in enumerate(E2):
                E3 = E2[j2 + 1:] + [u for u in adj[w2] if u > v and u not in nb[v] and u not in nb[w1]]
                total += sum(above(x, v) for x in E3)
    return total


# Graph pool of the serving tests: (n, m, seed) of directed Chung-Lu graphs
# (exponent 2.2, degree cap 120, 10% reciprocal, seed 7000 + s).
SERVING_TEST_POOL = [(300, 1200, 1), (800, 3200, 2), (2500, 12000, 3), (6000, 30000, 4), (150, 600, 5),
                     (4000, 16000, 6), (1200, 9000, 7), (9000, 40000, 8)]


def serving_test_pool():
    import synth
    return [synth.chung_lu(n, m, 2.2, 120, 10, 7000 + s) for n, m, s in SERVING_TEST_POOL]
