"""PEPS norm and energy networks assembled for libftn's contraction executor.

Marshalling only: this module builds bond lists and positions and calls the
C ABI (ftn_tensor_dagger, ftn_hubbard_term, ftn_contract); every contraction,
compression and reduction runs in libftn.

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


def energy(ctx, layout, kets, t, u, tree_fn, mode="local", policy="exact", chi=0, prec="f64"):
    """sum_t <h_t>/<Psi|Psi> over all nearest-neighbour hopping and on-site
    terms; each term and the norm are contracted with tree_fn(op_sites).
    Returns (energy, norm mantissa, norm log-scale).

    ``ctx`` may be a list of contexts (each on its own stream): the norm and
    the terms are independent contractions, so host threads, one per
    context, take them from a shared counter and run them concurrently on
    the GPU.  The kets, bras and operator tensors belong to the first
    context and are only read by the others.  The sum runs in term order,
    so the result does not depend on the schedule."""
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

    def run(c, job):
        tens, bonds, pos, tree = job
        return ftn.contract(c, tens, bonds, tree, positions=pos if glob else None, policy=policy, chi=chi, prec=prec)

    if len(ctxs) == 1:
        results = [run(c0, job) for job in jobs]
    else:
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
    nm, nl = results[0]
    total = 0.0
    for m, lg in results[1:]:
        total += m / nm * math.exp(lg - nl)
    return total, nm, nl
