"""PEPS norm and energy networks assembled for libftn's contraction executor.

Marshalling only: this module builds bond lists, positions and term index
tables and calls the C ABI (ftn_tensor_dagger, ftn_hubbard_term, ftn_energy,
ftn_energy_reduce); every contraction, compression, ratio and sum runs in
libftn.

Networks follow the globally ordered picture of the norm (Sec. IV.B, Fig. 4a):
the bra layer -- the daggers of the ket tensors, in reversed site order --
comes first, then (for <Psi|h_t|Psi>) the operator, then the ket layer.  The
same bonds and arrows serve the locally ordered contraction (positions
omitted): arrows point from later to earlier tensors, so both formalisms give
the same value.
Tensor ids: ket s -> s, bra s -> n + s, operator -> 2n.
"""
from __future__ import annotations

import weakref

from . import ftn

# Structure of cluster networks (bonds, positions, tree as int32 arrays) by
# cluster function and (targets, with operator): it depends on the lattice
# alone, so repeated evaluations of one lattice build it once.
_CLUSTER_STRUCT: "weakref.WeakKeyDictionary" = weakref.WeakKeyDictionary()


def layers(ctx, layout, kets):
    """Bra tensors and the bonds of both layers (no physical bonds yet)."""
    n = layout["n"]
    bras = [ftn.dagger(ctx, k) for k in kets]
    bonds = []
    for s, ks, t, kt in layout["bonds"]:
        bonds.append((s, ks, t, kt))
        bonds.append((n + s, kets[s].rank - 1 - ks, n + t, kets[t].rank - 1 - kt))
    return bras, bonds


def norm_network(ctx, layout, kets, bras=None):
    n = layout["n"]
    if bras is None:
        bras, bonds = layers(ctx, layout, kets)
    else:
        bonds = layers_bonds(layout, kets)
    for s in range(n):
        bonds.append((n + s, 0, s, kets[s].rank - 1))
    pos = [n + s for s in range(n)] + [n - 1 - s for s in range(n)]
    return list(kets) + list(bras), bonds, pos


def layers_bonds(layout, kets):
    n = layout["n"]
    out = []
    for s, ks, t, kt in layout["bonds"]:
        out.append((s, ks, t, kt))
        out.append((n + s, kets[s].rank - 1 - ks, n + t, kets[t].rank - 1 - kt))
    return out


def term_network(layout, kets, bras, op, sites):
    """<Psi|h|Psi> with operator tensor ``op`` (bra-side legs first in site
    order, then ket-side legs in reverse site order) on ``sites``."""
    n = layout["n"]
    bonds = layers_bonds(layout, kets)
    sites = list(sites)
    for s in range(n):
        if s not in sites:
            bonds.append((n + s, 0, s, kets[s].rank - 1))
    k = len(sites)
    for q, s in enumerate(sites):
        bonds.append((n + s, 0, 2 * n, q))
        bonds.append((2 * n, 2 * k - 1 - q, s, kets[s].rank - 1))
    pos = [n + 1 + s for s in range(n)] + [n - 1 - s for s in range(n)] + [n]
    return list(kets) + list(bras) + [op], bonds, pos


def energy_networks(ctx, layout, kets, t, u, tree_fn, mode="local", policy="exact", chi=0, dtype=ftn.F64):
    """The norm network followed by one network per nearest-neighbour hopping
    term and per on-site term, each with the tree tree_fn(op_sites), and the
    term table of ftn_energy (term t = network t + 1 over network 0).
    Returns (networks, num, den, group_end, keep) -- ``keep`` holds tensors
    the networks borrow (bras, operators)."""
    n = layout["n"]
    bras = [ftn.dagger(ctx, k) for k in kets]
    glob = mode == "global"
    hop = ftn.hubbard_term(ctx, 0, t, 0.0, dtype)
    onsite = ftn.hubbard_term(ctx, 1, 0.0, u, dtype)
    jobs = []
    tens, bonds, pos = norm_network(ctx, layout, kets, bras)
    jobs.append((tens, bonds, pos, tree_fn(())))
    for a, b in layout["edges"]:
        tens, bonds, pos = term_network(layout, kets, bras, hop, (a, b))
        jobs.append((tens, bonds, pos, tree_fn((a, b))))
    for s in range(n):
        tens, bonds, pos = term_network(layout, kets, bras, onsite, (s,))
        jobs.append((tens, bonds, pos, tree_fn((s,))))
    nets = [{"tensors": tens, "bonds": bonds, "tree": tree, "positions": pos if glob else None, "policy": policy,
             "chi": chi} for tens, bonds, pos, tree in jobs]
    nt = len(nets) - 1
    return nets, list(range(1, nt + 1)), [0] * nt, [nt], (bras, hop, onsite)


def energy(ctx, layout, kets, t, u, tree_fn, mode="local", policy="exact", chi=0, prec="f64", batch=0):
    """sum_t <h_t>/<Psi|Psi> over all nearest-neighbour hopping and on-site
    terms; each term and the norm are contracted with tree_fn(op_sites)
    (ftn_energy).  Returns (energy, norm mantissa, norm log-scale).

    ``ctx`` may be a list of contexts (each on its own stream): the norm and
    the terms are independent contractions, which libftn's host threads, one
    per context, take from a shared counter and run concurrently on the GPU.
    The kets belong to the first context and are only read by the others.
    ``batch`` > 0 contracts runs of up to ``batch`` networks in lock step
    (ftn_contract_batch).  The value is the same bit for bit in every case."""
    ctxs = list(ctx) if isinstance(ctx, (list, tuple)) else [ctx]
    dt = ftn.F64 if prec == "f64" else ftn.F32
    nets, num, den, ge, keep = energy_networks(ctxs[0], layout, kets, t, u, tree_fn, mode, policy, chi, dt)
    en, _, vals = ftn.energy(ctxs, nets, num, den, ge, prec, batch)
    del keep
    return en[0], vals[0][0], vals[0][1]


# ---- cluster approximation (Sec. V) -------------------------------------------

def gauge_tensor(ctx, lam_even, lam_odd, dual_to_bra, dtype=ftn.F64):
    """Even rank-2 tensor diag(lambda^2) closing a dangling bond: leg 0 meets
    the bra's leg, leg 1 the ket's (``dual_to_bra`` = the ket leg's dual)."""
    import numpy as np

    d0, d1 = len(lam_even), len(lam_odd)
    legs = [(d0, d1, dual_to_bra), (d0, d1, 1 - dual_to_bra)]
    blocks = []
    if d0:
        blocks.append(((0, 0), np.diag(np.asarray(lam_even, float) ** 2)))
    if d1:
        blocks.append(((1, 1), np.diag(np.asarray(lam_odd, float) ** 2)))
    return ftn.Tensor.from_blocks(ctx, legs, 0, blocks, dtype)


def cluster_network(layout, kets, bras, sites, dangling, gauge_of, op=None, targets=()):
    """Globally ordered network of one cluster (Fig. 4b): bra cluster in
    reversed order, then the operator (if any) and one gauge tensor per
    dangling bond, then the ket cluster.  Ids: kets 0..m-1 (order of
    ``sites``), bras m..2m-1, operator 2m, then the gauges in ``dangling``
    order; ``gauge_of(s, leg)`` gives the library gauge tensor of a dangling
    ket leg.  Returns (tensors, bonds, positions)."""
    m = len(sites)
    loc = {s: i for i, s in enumerate(sites)}
    tensors = [kets[s] for s in sites] + [bras[s] for s in sites]
    rank = [kets[s].rank for s in sites]
    bonds = []
    for s, a, t, b in layout["bonds"]:
        if s in loc and t in loc:
            i, j = loc[s], loc[t]
            bonds.append((i, a, j, b))
            bonds.append((m + i, rank[i] - 1 - a, m + j, rank[j] - 1 - b))
    targets = list(targets)
    for s in sites:
        if op is None or s not in targets:
            i = loc[s]
            bonds.append((m + i, 0, i, rank[i] - 1))
    nmid = 0
    if op is not None:
        tensors.append(op)
        nmid = 1
        k = len(targets)
        for q, s in enumerate(targets):
            i = loc[s]
            bonds.append((m + i, 0, 2 * m, q))
            bonds.append((2 * m, 2 * k - 1 - q, i, rank[i] - 1))
    for s, a, _t in dangling:
        i = loc[s]
        gid = len(tensors)
        tensors.append(gauge_of(s, a))
        nmid += 1
        bonds.append((m + i, rank[i] - 1 - a, gid, 0))
        bonds.append((gid, 1, i, a))
    pos = [m + nmid + i for i in range(m)] + [m - 1 - i for i in range(m)] + [m + q for q in range(nmid)]
    return tensors, bonds, pos


def _cluster_structure(layout, kets, cluster_fn, targets):
    """Sites, dangling bonds and, with and without the operator, the bonds,
    positions and tree of a term's cluster network (int32 arrays)."""
    import numpy as np

    sites, dang, tree_op, tree_norm = cluster_fn(list(targets))
    st = {"sites": list(sites), "dang": list(dang)}
    for with_op, tree in ((True, tree_op), (False, tree_norm)):
        _t, bonds, pos = cluster_network(layout, kets, kets, sites, dang, lambda s, a: None,
                                         object() if with_op else None, targets)
        st[with_op] = (np.asarray(bonds, dtype=np.int32).reshape(-1, 4), np.asarray(pos, dtype=np.int32),
                       np.asarray(tree, dtype=np.int32).reshape(-1, 2))
    return st


def cluster_networks(ctx, instances, t, u, policy="exact", chi=0, dtype=ftn.F64, terms=None):
    """Cluster networks of every hopping and on-site term of every instance
    (layout, kets, cluster_fn, gauges) -- or of the target tuples ``terms``
    (pairs are hopping terms, single sites on-site terms): for each term the
    network with the operator, then the same network without it (its
    normalisation), and the term table of ftn_energy with one group per
    instance.  ``cluster_fn`` must depend on the targets alone: the
    networks' structure is kept per cluster function and reused by later
    calls.  Returns (networks, num, den, group_end, keep)."""
    hop = ftn.hubbard_term(ctx, 0, t, 0.0, dtype)
    onsite = ftn.hubbard_term(ctx, 1, 0.0, u, dtype)
    nets, group_end, keep = [], [], [hop, onsite]
    by_content = {}  # gauge tensors by (weights, duality): equal weights share one tensor
    keep.append(by_content)
    for layout, kets, cluster_fn, gauges in instances:
        bras = [ftn.dagger(ctx, k) for k in kets]
        cache = {}

        def gauge_of(s, a, layout=layout, kets=kets, gauges=gauges, cache=cache):
            if (s, a) not in cache:
                nb = layout["nbrs"][s][a]
                lam = gauges[(min(s, nb), max(s, nb))]
                key = (tuple(map(float, lam[0])), tuple(map(float, lam[1])), kets[s].legs[a][2])
                if key not in by_content:
                    by_content[key] = gauge_tensor(ctx, lam[0], lam[1], key[2], dtype)
                cache[(s, a)] = by_content[key]
            return cache[(s, a)]

        if terms is None:
            tl = [((a, b), hop) for a, b in layout["edges"]] + [((s,), onsite) for s in range(layout["n"])]
        else:
            tl = [(tuple(tg), hop if len(tg) == 2 else onsite) for tg in terms]
        memo = _CLUSTER_STRUCT.setdefault(cluster_fn, {})
        for targets, op in tl:
            st = memo.get(targets)
            if st is None:
                st = memo[targets] = _cluster_structure(layout, kets, cluster_fn, targets)
            sites, dang = st["sites"], st["dang"]
            base = [kets[s] for s in sites] + [bras[s] for s in sites]
            gauges = [gauge_of(s, a) for s, a, _t in dang]
            for with_op, o in ((True, op), (False, None)):
                bonds, pos, tree = st[with_op]
                tens = base + ([o] if with_op else []) + gauges
                nets.append({"tensors": tens, "bonds": bonds, "tree": tree, "positions": pos, "policy": policy,
                             "chi": chi})
        group_end.append(len(nets) // 2)
        keep.append((bras, cache))
    nt = len(nets) // 2
    return nets, [2 * q for q in range(nt)], [2 * q + 1 for q in range(nt)], group_end, keep


def cluster_energy(ctx, layout, kets, t, u, cluster_fn, gauges, policy="exact", chi=0, prec="f64", batch=0):
    """Cluster approximation of sum_t <h_t>: every hopping and on-site term
    is the ratio of its cluster network with the operator to the same network
    without it, both contracted in the globally ordered formalism.
    ``cluster_fn(targets)`` gives (sites, dangling bonds, tree with the
    operator, tree without it); ``gauges[(s, t)]`` = (even, odd) weights of
    the bond's stand-in gauge.  ``ctx`` may be a list of contexts (the
    contractions then run concurrently, as in :func:`energy`); ``batch`` as
    in :func:`energy`.  Returns (energy, per-term ratios)."""
    return cluster_energies(ctx, [(layout, kets, cluster_fn, gauges)], t, u, policy, chi, prec, batch)[0]


def cluster_energies(ctx, instances, t, u, policy="exact", chi=0, prec="f64", batch=0, terms=None):
    """:func:`cluster_energy` of several states at once: ``instances`` is a
    list of (layout, kets, cluster_fn, gauges); the networks of all terms of
    all instances are contracted by one ftn_energy call (in lock-step runs of
    up to ``batch`` networks when ``batch`` > 0); ``terms`` as in
    :func:`cluster_networks`.  Returns [(energy, ratios)] per instance."""
    ctxs = list(ctx) if isinstance(ctx, (list, tuple)) else [ctx]
    dt = ftn.F64 if prec == "f64" else ftn.F32
    nets, num, den, ge, keep = cluster_networks(ctxs[0], instances, t, u, policy, chi, dt, terms)
    en, ratios, _ = ftn.energy(ctxs, nets, num, den, ge, prec, batch)
    del keep
    out, t0 = [], 0
    for g, t1 in enumerate(ge):
        out.append((en[g], ratios[t0:t1]))
        t0 = t1
    return out
