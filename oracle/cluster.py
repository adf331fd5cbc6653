"""Cluster approximation of local energy terms (Sec. V, Fig. ftn_clusterc).

TEST INFRASTRUCTURE ONLY (see the package docstring).

For a term h_t on its target sites, the cluster is every site within graph
distance r of the targets.  The bra and ket of the cluster form their own
globally ordered network (Fig. 4b: bra cluster in reversed site order, then
the operator and the gauges, then the ket cluster; the arrows follow from that
order, which changes some of them with respect to the full network -- the
"partial trace" of the paper).  Every bond leaving the cluster is closed by the
simple-update gauges standing in for the rest of the network: the ket's and
the bra's dangling legs are joined through the diagonal weights lambda_k^2 of
that bond (lambda on the ket side times lambda on the bra side).  The term's
value is the ratio of the cluster network with the operator to the same
network without it, and the energy is the sum over terms.  Contractions are
those of :mod:`oracle.network` in the globally ordered formalism.
"""
from __future__ import annotations

import numpy as np

from .graded import GTensor, dagger
from .hubbard import hop_gate, onsite_gate
from .network import Network, contract_tree

__all__ = ["gauge_tensor", "cluster_network", "cluster_energy"]


def gauge_tensor(lam_even, lam_odd, dual_to_bra):
    """Even rank-2 tensor diag(lambda^2): leg 0 meets the bra leg, leg 1 the
    ket leg (``dual_to_bra`` is the ket leg's dual)."""
    w = np.concatenate([np.asarray(lam_even, float) ** 2, np.asarray(lam_odd, float) ** 2])
    d0, d1 = len(lam_even), len(lam_odd)
    return GTensor(np.diag(w), [(d0, d1, dual_to_bra), (d0, d1, 1 - dual_to_bra)], 0)


def cluster_network(layout, kets, sites, dangling, gauges, op=None, targets=()):
    """Globally ordered cluster network.  Ids: kets 0..m-1 (order of
    ``sites``), bras m..2m-1, the operator 2m (if given), then one gauge tensor
    per entry of ``dangling`` ((s, leg of s, t) with t outside)."""
    m = len(sites)
    loc = {s: i for i, s in enumerate(sites)}
    ks = [kets[s] for s in sites]
    bras = [dagger(k) for k in ks]
    tensors = list(ks) + bras
    bonds = []
    for s, a, t, b in layout["bonds"]:
        if s in loc and t in loc:
            i, j = loc[s], loc[t]
            bonds.append((i, a, j, b))
            bonds.append((m + i, ks[i].rank - 1 - a, m + j, ks[j].rank - 1 - b))
    targets = list(targets)
    for s in sites:
        if op is None or s not in targets:
            i = loc[s]
            bonds.append((m + i, 0, i, ks[i].rank - 1))
    nmid = 0
    if op is not None:
        tensors.append(op)
        nmid = 1
        k = len(targets)
        for q, s in enumerate(targets):
            i = loc[s]
            bonds.append((m + i, 0, 2 * m, q))
            bonds.append((2 * m, 2 * k - 1 - q, i, ks[i].rank - 1))
    for s, a, t in dangling:
        i = loc[s]
        lam = gauges[(min(s, t), max(s, t))]
        g = gauge_tensor(lam[0], lam[1], ks[i].legs[a][2])
        gid = len(tensors)
        tensors.append(g)
        nmid += 1
        bonds.append((m + i, ks[i].rank - 1 - a, gid, 0))
        bonds.append((gid, 1, i, a))
    pos = [m + nmid + i for i in range(m)] + [m - 1 - i for i in range(m)] + [m + q for q in range(nmid)]
    return Network(tensors, bonds, pos)


def cluster_energy(layout, kets, t, u, cluster_fn, gauges, policy="exact", chi=None):
    """Sum over hopping and on-site terms of the cluster-approximated <h_t>.
    ``cluster_fn(targets)`` gives the term's (sites, dangling bonds, tree of
    the network with the operator, tree of the network without it).  Returns
    (energy, per-term ratios)."""
    ratios = []
    terms = [((a, b), hop_gate(t)) for a, b in layout["edges"]] + [((s,), onsite_gate(u)) for s in range(layout["n"])]
    for targets, op in terms:
        sites, dang, tree_op, tree_norm = cluster_fn(list(targets))
        num = cluster_network(layout, kets, sites, dang, gauges, op, targets)
        den = cluster_network(layout, kets, sites, dang, gauges)
        rn, ln, _ = contract_tree(num, tree_op, mode="global", policy=policy, chi=chi, normalize=True)
        rd, ld, _ = contract_tree(den, tree_norm, mode="global", policy=policy, chi=chi, normalize=True)
        ratios.append(float(rn.data) / float(rd.data) * np.exp(ln - ld))
    return float(sum(ratios)), ratios
