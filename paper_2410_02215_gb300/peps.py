"""PEPS norm and energy networks assembled for libftn's contraction executor.

Marshalling only: this module builds bond lists and positions and calls the
C ABI (ftn_tensor_dagger, ftn_hubbard_term, ftn_contract, ftn_contract_batch);
every contraction, compression and reduction runs in libftn.

Networks follow the globally ordered picture of the norm (Sec. IV.B, Fig. 4a):
the bra layer -- the daggers of the ket tensors, in reversed site order --
comes first, then (for <Psi|h_t|Psi>) the operator, then the ket layer.  The
same bonds and arrows serve the locally ordered contraction (positions
omitted): arrows point from later to earlier tensors, so both formalisms give
the same value.
Tensor ids: ket s -> s, bra s -> n + s, operator -> 2n.
"""
from __future__ import annotations

import math

from . import ftn


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


def energy(ctx, layout, kets, t, u, tree_fn, mode="local", policy="exact", chi=0, prec="f64", batch=0):
    """sum_t <h_t>/<Psi|Psi> over all nearest-neighbour hopping and on-site
    terms; each term and the norm are contracted with tree_fn(op_sites).
    Returns (energy, norm mantissa, norm log-scale).

    ``ctx`` may be a list of contexts (each on its own stream): the norm and
    the terms are independent contractions, so host threads, one per
    context, take them from a shared counter and run them concurrently on
    the GPU.  The kets, bras and operator tensors belong to the first
    context and are only read by the others.  The sum runs in term order,
    so the result does not depend on the schedule.  ``batch`` as in
    :func:`contract_many` (bit-identical results either way)."""
    ctxs = list(ctx) if isinstance(ctx, (list, tuple)) else [ctx]
    c0 = ctxs[0]
    dt = ftn.F64 if prec == "f64" else ftn.F32
    n = layout["n"]
    bras = [ftn.dagger(c0, k) for k in kets]
    glob = mode == "global"
    hop = ftn.hubbard_term(c0, 0, t, 0.0, dt)
    onsite = ftn.hubbard_term(c0, 1, 0.0, u, dt)
    jobs = []
    tens, bonds, pos = norm_network(c0, layout, kets, bras)
    jobs.append((tens, bonds, pos, tree_fn(())))
    for a, b in layout["edges"]:
        tens, bonds, pos = term_network(layout, kets, bras, hop, (a, b))
        jobs.append((tens, bonds, pos, tree_fn((a, b))))
    for s in range(n):
        tens, bonds, pos = term_network(layout, kets, bras, onsite, (s,))
        jobs.append((tens, bonds, pos, tree_fn((s,))))

    nets = [{"tensors": tens, "bonds": bonds, "tree": tree, "positions": pos if glob else None, "policy": policy,
             "chi": chi} for tens, bonds, pos, tree in jobs]
    results = contract_many(ctxs, nets, prec, batch)
    nm, nl = results[0]
    total = 0.0
    for m, lg in results[1:]:
        total += m / nm * math.exp(lg - nl)
    return total, nm, nl


def contract_many(ctx, networks, prec="f64", batch=0):
    """(mantissa, log_scale) of every network (dicts as for
    :func:`ftn.contract_batch`), in order.  ``batch`` = 0: one ftn_contract
    per network; > 0: batches of up to ``batch`` networks per
    ftn_contract_batch call.  With several contexts, host threads (one per
    context) take networks or batches from a shared counter."""
    ctxs = list(ctx) if isinstance(ctx, (list, tuple)) else [ctx]
    nets = list(networks)
    if batch and batch > 0:
        chunks = [nets[i:i + batch] for i in range(0, len(nets), batch)]
        res = _run_jobs(ctxs, chunks, lambda c, ch: ftn.contract_batch(c, ch, prec=prec))
        return [r for part in res for r in part]

    def run(c, job):
        return ftn.contract(c, job["tensors"], job["bonds"], job["tree"], positions=job.get("positions"),
                            policy=job.get("policy", "exact"), chi=job.get("chi", 0), prec=prec)

    return _run_jobs(ctxs, nets, run)


def _run_jobs(ctxs, jobs, run):
    """run(ctx, job) for every job; with several contexts, host threads (one
    per context) take jobs from a shared counter.  Results in job order."""
    c0 = ctxs[0]
    if len(ctxs) == 1:
        return [run(c0, job) for job in jobs]
    import threading

    c0.synchronize()  # inputs ready before other streams read them
    results = [None] * len(jobs)
    errors = []
    lock = threading.Lock()
    nxt = [0]

    def worker(c):
        try:
            while True:
                with lock:
                    i = nxt[0]
                    nxt[0] += 1
                if i >= len(jobs) or errors:
                    return
                results[i] = run(c, jobs[i])
        except BaseException as e:  # re-raised on the calling thread
            errors.append(e)

    threads = [threading.Thread(target=worker, args=(c,)) for c in ctxs]
    for th in threads:
        th.start()
    for th in threads:
        th.join()
    if errors:
        raise errors[0]
    return results


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


def cluster_energy(ctx, layout, kets, t, u, cluster_fn, gauges, policy="exact", chi=0, prec="f64", batch=0):
    """Cluster approximation of sum_t <h_t>: every hopping and on-site term
    is the ratio of its cluster network with the operator to the same network
    without it, both contracted in the globally ordered formalism.
    ``cluster_fn(targets)`` gives (sites, dangling bonds, tree with the
    operator, tree without it); ``gauges[(s, t)]`` = (even, odd) weights of
    the bond's stand-in gauge.  ``ctx`` may be a list of contexts (the
    contractions then run concurrently, as in :func:`energy`); ``batch`` as
    in :func:`contract_many`.  Returns (energy, per-term ratios)."""
    return cluster_energies(ctx, [(layout, kets, cluster_fn, gauges)], t, u, policy, chi, prec, batch)[0]


def cluster_energies(ctx, instances, t, u, policy="exact", chi=0, prec="f64", batch=0):
    """:func:`cluster_energy` of several states at once: ``instances`` is a
    list of (layout, kets, cluster_fn, gauges); the networks of all terms of
    all instances are contracted together (in batches of up to ``batch``
    networks when ``batch`` > 0).  Returns [(energy, ratios)] per instance."""
    ctxs = list(ctx) if isinstance(ctx, (list, tuple)) else [ctx]
    c0 = ctxs[0]
    dt = ftn.F64 if prec == "f64" else ftn.F32
    hop = ftn.hubbard_term(c0, 0, t, 0.0, dt)
    onsite = ftn.hubbard_term(c0, 1, 0.0, u, dt)
    nets, nterms, keep = [], [], []
    for layout, kets, cluster_fn, gauges in instances:
        bras = [ftn.dagger(c0, k) for k in kets]
        cache = {}

        def gauge_of(s, a, layout=layout, kets=kets, gauges=gauges, cache=cache):
            if (s, a) not in cache:
                nb = layout["nbrs"][s][a]
                lam = gauges[(min(s, nb), max(s, nb))]
                cache[(s, a)] = gauge_tensor(c0, lam[0], lam[1], kets[s].legs[a][2], dt)
            return cache[(s, a)]

        terms = [((a, b), hop) for a, b in layout["edges"]] + [((s,), onsite) for s in range(layout["n"])]
        for targets, op in terms:
            sites, dang, tree_op, tree_norm = cluster_fn(list(targets))
            for o, tree in ((op, tree_op), (None, tree_norm)):
                tens, bonds, pos = cluster_network(layout, kets, bras, sites, dang, gauge_of, o, targets)
                nets.append({"tensors": tens, "bonds": bonds, "tree": tree, "positions": pos, "policy": policy,
                             "chi": chi})
        nterms.append(len(terms))
        keep.append((bras, cache))
    res = contract_many(ctxs, nets, prec, batch)
    out, q = [], 0
    for nt in nterms:
        ratios = []
        for _ in range(nt):
            (mn, ln), (md, ld) = res[q], res[q + 1]
            ratios.append(mn / md * math.exp(ln - ld))
            q += 2
        out.append((float(sum(ratios)), ratios))
    return out
