"""Lattice graphs and contraction trees (structure only, no arithmetic).

Graphs are lists of undirected edges ``(i, j)`` with ``i < j`` over sites
``0..n-1``; site order is the global order of the fermionic tensors
(Sec. IV.B: tensors are created in site order and arrows point from later to
earlier sites).  A contraction tree is a list of SSA pairs: the inputs are ids
``0..n-1`` and step ``s`` creates id ``n + s``.
"""
from __future__ import annotations

import itertools

import numpy as np

from .gen import rng

__all__ = [
    "square_lattice",
    "diamond_lattice",
    "random_regular_graph",
    "sequential_tree",
    "random_tree",
    "connected_random_tree",
    "all_trees_small",
]


def square_lattice(lx, ly):
    """Open lx-by-ly square lattice, sites row-major (site = x * ly + y)."""
    edges = []
    for x in range(lx):
        for y in range(ly):
            s = x * ly + y
            if y + 1 < ly:
                edges.append((s, s + 1))
            if x + 1 < lx:
                edges.append((s, s + ly))
    return lx * ly, sorted(edges)


def diamond_lattice(nx, ny, nz):
    """Diamond structure on nx*ny*nz conventional cubic cells, open boundaries.

    Atoms: the FCC points (0,0,0), (0,1/2,1/2), (1/2,0,1/2), (1/2,1/2,0) of each
    cell plus the same points shifted by (1/4,1/4,1/4); 8 sites per cell.
    Nearest neighbours are at distance sqrt(3)/4.  Sites are ordered
    lexicographically by (x, y, z).  Returns (n_sites, edges, coords).
    """
    fcc = [(0, 0, 0), (0, 2, 2), (2, 0, 2), (2, 2, 0)]  # in units of 1/4
    pts = []
    for cx in range(nx):
        for cy in range(ny):
            for cz in range(nz):
                for b in ((0, 0, 0), (1, 1, 1)):
                    for f in fcc:
                        pts.append((4 * cx + f[0] + b[0], 4 * cy + f[1] + b[1], 4 * cz + f[2] + b[2]))
    pts = sorted(set(pts))
    idx = {p: i for i, p in enumerate(pts)}
    edges = []
    for p in pts:
        for d in itertools.product((-1, 1), repeat=3):
            q = (p[0] + d[0], p[1] + d[1], p[2] + d[2])
            if q in idx and idx[p] < idx[q]:
                edges.append((idx[p], idx[q]))
    return len(pts), sorted(set(edges)), np.array(pts, dtype=float) / 4.0


def random_regular_graph(n, degree, seed, max_tries=1000):
    """Random simple degree-regular graph by the pairing model with rejection."""
    g = rng(seed)
    if (n * degree) % 2:
        raise ValueError("n * degree must be even")
    for _ in range(max_tries):
        stubs = np.repeat(np.arange(n), degree)
        g.shuffle(stubs)
        pairs = stubs.reshape(-1, 2)
        ok = True
        seen = set()
        for a, b in pairs:
            a, b = int(a), int(b)
            if a == b or (min(a, b), max(a, b)) in seen:
                ok = False
                break
            seen.add((min(a, b), max(a, b)))
        if ok:
            return n, sorted(seen)
    raise RuntimeError("pairing model did not produce a simple graph")


def sequential_tree(order):
    """Contract order[0] with order[1], the result with order[2], and so on."""
    n = len(order)
    pairs = []
    cur = order[0]
    for s, t in enumerate(order[1:]):
        pairs.append((cur, t))
        cur = n + s
    return pairs


def random_tree(n, seed):
    """Uniformly random sequence of pairwise merges, random operand order."""
    g = rng(seed)
    live = list(range(n))
    pairs = []
    nxt = n
    while len(live) > 1:
        i, j = g.choice(len(live), size=2, replace=False)
        a, b = live[i], live[j]
        pairs.append((int(a), int(b)))
        live = [x for x in live if x not in (a, b)] + [nxt]
        nxt += 1
    return pairs


def connected_random_tree(n, edges, seed):
    """Random merges restricted to pairs that share at least one edge."""
    g = rng(seed)
    members = {i: {i} for i in range(n)}
    adj = [(a, b) for a, b in edges]
    pairs = []
    nxt = n
    while len(members) > 1:
        keys = list(members)
        cand = []
        for x in range(len(keys)):
            for y in range(x + 1, len(keys)):
                A, B = members[keys[x]], members[keys[y]]
                if any((a in A and b in B) or (a in B and b in A) for a, b in adj):
                    cand.append((keys[x], keys[y]))
        if not cand:
            cand = [(keys[0], keys[1])]
        a, b = cand[int(g.integers(len(cand)))]
        if g.integers(2):
            a, b = b, a
        pairs.append((a, b))
        members[nxt] = members.pop(a) | members.pop(b)
        nxt += 1
    return pairs


def all_trees_small(n, limit=None):
    """Every merge sequence (with operand order) for a handful of tensors."""
    out = []

    def rec(live, nxt, acc):
        if limit is not None and len(out) >= limit:
            return
        if len(live) == 1:
            out.append(list(acc))
            return
        for i in range(len(live)):
            for j in range(len(live)):
                if i == j:
                    continue
                a, b = live[i], live[j]
                rest = [x for x in live if x not in (a, b)]
                acc.append((a, b))
                rec(rest + [nxt], nxt + 1, acc)
                acc.pop()

    rec(list(range(n)), n, [])
    return out
