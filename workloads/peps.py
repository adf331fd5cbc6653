"""PEPS structure on a graph: which leg of which site tensor meets which.

Structure only (no arithmetic).  Site tensors are created in site order with
the arrows of every bond pointing from the later site to the earlier one and
the +/- labels aligned with the arrows (Sec. IV.B): on bond (s, t) with
s < t, site s holds the incoming ('-', dual 1) leg and site t the outgoing
('+', dual 0) leg.  The physical leg is last and outgoing.
"""
from __future__ import annotations

from .gen import random_blocks

__all__ = ["peps_layout", "random_peps", "double_layer_tree", "site_sweep_tree", "boundary_mps_tree", "cluster_sites",
           "dangling_bonds",
           "bond_gauges", "cluster_ids", "cluster_tree"]


def peps_layout(n, edges, D, phys=(2, 2)):
    """Per-site leg lists and the ket-layer bonds.

    ``D`` is a pair (d_even, d_odd) for every virtual bond (or a dict edge ->
    pair).  Returns ``{"n", "legs": [[(d0, d1, dual), ...] per site],
    "nbrs": [[neighbour per virtual leg] per site], "bonds": [(s, ks, t, kt)],
    "edges"}``.
    """
    nbrs = [[] for _ in range(n)]
    for a, b in edges:
        nbrs[a].append(b)
        nbrs[b].append(a)
    for s in range(n):
        nbrs[s].sort()
    legs = []
    for s in range(n):
        ls = []
        for t in nbrs[s]:
            e = (min(s, t), max(s, t))
            d = D[e] if isinstance(D, dict) else D
            ls.append((int(d[0]), int(d[1]), 1 if s < t else 0))
        ls.append((int(phys[0]), int(phys[1]), 0))
        legs.append(ls)
    bonds = []
    for a, b in sorted(edges):
        bonds.append((a, nbrs[a].index(b), b, nbrs[b].index(a)))
    return {"n": n, "legs": legs, "nbrs": nbrs, "bonds": bonds, "edges": sorted(edges)}


def random_peps(layout, seed, scale=1.0):
    """Even-parity site tensors with i.i.d. N(0, scale^2) allowed entries, as
    lists of (bits, block) per site."""
    return [random_blocks(layout["legs"][s], 0, 7919 * seed + 31 * s + 5, scale) for s in range(layout["n"])]


def double_layer_tree(n, site_tree, op_sites=()):
    """SSA tree over a double-layer network with ids kets 0..n-1, bras n..2n-1
    and (when ``op_sites`` is not empty) the operator at 2n.

    First every site's ket and bra are merged (the operator is merged into the
    ket of its first site before that site's bra); the merged site tensors then
    follow ``site_tree``, an SSA tree over n site nodes.
    """
    pairs = []
    nt = 2 * n + (1 if op_sites else 0)
    nxt = nt
    site_id = {}
    for s in range(n):
        k = s
        if op_sites and s == op_sites[0]:
            pairs.append((2 * n, k))
            k = nxt
            nxt += 1
        pairs.append((k, n + s))
        site_id[s] = nxt
        nxt += 1
    remap = dict(site_id)
    for q, (a, b) in enumerate(site_tree):
        pairs.append((remap[a], remap[b]))
        remap[n + q] = nxt
        nxt += 1
    return pairs


def boundary_mps_tree(lx, ly):
    """Site-level SSA tree of the boundary-MPS row sweep on an lx-by-ly open
    square lattice (sites row-major, site = x * ly + y): column y's boundary
    tensor starts as site (0, y) and absorbs (1, y), (2, y), ... row by row
    (row x into every column before row x + 1), so the boundary stays a chain
    of one tensor per column whose horizontal bonds grow by the vertical bond
    dimension per row (the bonds a late compression caps at chi); after the
    last row the column tensors are merged left to right."""
    n = lx * ly
    pairs = []
    cur = list(range(ly))
    nxt = n
    for x in range(1, lx):
        for y in range(ly):
            pairs.append((cur[y], x * ly + y))
            cur[y] = nxt
            nxt += 1
    acc = cur[0]
    for y in range(1, ly):
        pairs.append((acc, cur[y]))
        acc = nxt
        nxt += 1
    return pairs


def site_sweep_tree(order):
    """Site-level sequential tree: merge order[0], order[1], ... one by one."""
    n = len(order)
    pairs = []
    cur = order[0]
    for s, t in enumerate(order[1:]):
        pairs.append((cur, t))
        cur = n + s
    return pairs


# ---- cluster approximation (structure and stand-in gauges) -------------------

def cluster_sites(layout, targets, r):
    """Sites within graph distance r of any target site, sorted."""
    dist = {t: 0 for t in targets}
    frontier = list(targets)
    for d in range(1, r + 1):
        nxt = []
        for s in frontier:
            for t in layout["nbrs"][s]:
                if t not in dist:
                    dist[t] = d
                    nxt.append(t)
        frontier = nxt
    return sorted(dist)


def dangling_bonds(layout, sites):
    """Bonds leaving the cluster: (s, leg of s, t) with s inside, t outside, in
    increasing (s, t)."""
    inside = set(sites)
    out = []
    for s in sites:
        for k, t in enumerate(layout["nbrs"][s]):
            if t not in inside:
                out.append((s, k, t))
    return out


def bond_gauges(layout, decay=0.5):
    """Stand-in for simple-update bond gauges: on every bond the diagonal
    weights decay**k for the k-th state of each sector.  Returns
    {edge (s, t), s < t: (even weights, odd weights)}."""
    out = {}
    for s, ks, t, kt in layout["bonds"]:
        d0, d1, _ = layout["legs"][s][ks]
        out[(s, t)] = ([decay**k for k in range(d0)], [decay**k for k in range(d1)])
    return out


def cluster_ids(layout, sites, with_op):
    """Tensor ids of a cluster network: kets 0..m-1 (cluster order), bras
    m..2m-1, the operator 2m (if any), then one gauge tensor per dangling bond
    in :func:`dangling_bonds` order.  Returns (local index of each cluster site,
    operator id or None, first gauge id)."""
    m = len(sites)
    loc = {s: i for i, s in enumerate(sites)}
    op = 2 * m if with_op else None
    return loc, op, 2 * m + (1 if with_op else 0)


def cluster_tree(layout, sites, targets, with_op):
    """SSA contraction tree of a cluster network (ids of :func:`cluster_ids`):
    every gauge tensor is merged into its site's ket, the operator into the
    ket of its first site, each ket into its bra, and the merged sites in
    breadth-first order from the targets."""
    m = len(sites)
    loc, op, g0 = cluster_ids(layout, sites, with_op)
    dang = dangling_bonds(layout, sites)
    nt = g0 + len(dang)
    nxt = nt
    cur = {i: i for i in range(m)}  # current node of each site's ket
    pairs = []
    for g, (s, _, _) in enumerate(dang):
        pairs.append((g0 + g, cur[loc[s]]))
        cur[loc[s]] = nxt
        nxt += 1
    site_node = {}
    for i in range(m):
        k = cur[i]
        if with_op and sites[i] == targets[0]:
            pairs.append((op, k))
            k = nxt
            nxt += 1
        pairs.append((k, m + i))
        site_node[i] = nxt
        nxt += 1
    order = []
    seen = set()
    frontier = list(targets)
    while frontier:
        for s in frontier:
            if s not in seen:
                seen.add(s)
                order.append(s)
        frontier = sorted({t for s in frontier for t in layout["nbrs"][s] if t in loc and t not in seen})
    acc = site_node[loc[order[0]]]
    for s in order[1:]:
        pairs.append((acc, site_node[loc[s]]))
        acc = nxt
        nxt += 1
    return pairs
