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
