"""Fermi-Hubbard terms, PEPS double-layer networks and exact diagonalisation.

Test infrastructure only (see the package docstring).

Local basis of a site (physical leg split 2+2, even states first):
0 = |0>, 1 = |up,down> = c+_up c+_dn |0>, 2 = |up> = c+_up |0>, 3 = |dn> = c+_dn |0>.
A PEPS amplitude psi(n_0 ... n_{N-1}) is the coefficient of the ordered
creation string S_0(n_0) S_1(n_1) ... S_{N-1}(n_{N-1}) |vac>, sites in global
order, which is what the ket network F(T^[0] T^[1] ...) produces with its
physical legs in site order.
"""
from __future__ import annotations

import numpy as np

from .graded import GTensor, dagger, embed_blocks, transpose
from .network import Network, contract_tree

__all__ = [
    "LOCAL_OCC",
    "jw_annihilators",
    "hop_gate",
    "onsite_gate",
    "ket_tensors",
    "norm_network",
    "term_network",
    "ket_amplitudes",
    "ed_energy",
    "energy_terms",
]

# local state -> (n_up, n_dn)
LOCAL_OCC = {0: (0, 0), 1: (1, 1), 2: (1, 0), 3: (0, 1)}


def jw_annihilators(nmodes):
    """Jordan-Wigner annihilation operators c_m = Z_0 ... Z_{m-1} a_m on
    2^nmodes states; basis index = sum_m n_m 2^{nmodes-1-m}, so that the basis
    vector of occupations n equals prod_m (c+_m)^{n_m} |vac> (m increasing)."""
    a = np.array([[0.0, 1.0], [0.0, 0.0]])
    z = np.diag([1.0, -1.0])
    eye = np.eye(2)
    ops = []
    for m in range(nmodes):
        op = np.ones((1, 1))
        for l in range(nmodes):
            op = np.kron(op, z if l < m else (a if l == m else eye))
        ops.append(op)
    return ops


def _fock_index(occ_list):
    bits = []
    for n_up, n_dn in occ_list:
        bits += [n_up, n_dn]
    idx = 0
    for b in bits:
        idx = 2 * idx + b
    return idx


def _two_site_hop_matrix(t):
    c = jw_annihilators(4)  # modes: i_up, i_dn, j_up, j_dn
    h = np.zeros((16, 16))
    for sig in (0, 1):
        ci, cj = c[sig], c[2 + sig]
        h += -t * (ci.T @ cj + cj.T @ ci)
    return h


def hop_gate(t):
    """Hopping term -t sum_sigma (c+_i c_j + h.c.) of Eq. (fermi-hubbard-ham) on
    a bond i < j, as an even 4-leg tensor O[i', j', j, i].

    Entries are the two-site matrix elements <n_i n_j| h |m_i m_j> in the
    ordered-string basis (site i's modes first), read from a Jordan-Wigner
    Fock-space matrix.  Legs: the two bra-side legs (outgoing) in site order,
    then the two ket-side legs (incoming) in reverse site order, so that in
    F(bra, O, ket) the operator sits between the layers.
    """
    h = _two_site_hop_matrix(t)
    o = np.zeros((4, 4, 4, 4))
    for ni in range(4):
        for nj in range(4):
            for mi in range(4):
                for mj in range(4):
                    o[ni, nj, mj, mi] = h[
                        _fock_index([LOCAL_OCC[ni], LOCAL_OCC[nj]]),
                        _fock_index([LOCAL_OCC[mi], LOCAL_OCC[mj]]),
                    ]
    legs = [(2, 2, 0), (2, 2, 0), (2, 2, 1), (2, 2, 1)]
    return GTensor(o, legs, 0)


def onsite_gate(u):
    """On-site term U n_up n_dn as an even 2-leg tensor O[i', i]."""
    c = jw_annihilators(2)
    h = u * (c[0].T @ c[0]) @ (c[1].T @ c[1])
    o = np.zeros((4, 4))
    for n in range(4):
        for m in range(4):
            o[n, m] = h[_fock_index([LOCAL_OCC[n]]), _fock_index([LOCAL_OCC[m]])]
    return GTensor(o, [(2, 2, 0), (2, 2, 1)], 0)


def ket_tensors(layout, blocks):
    return [embed_blocks(layout["legs"][s], 0, blocks[s]) for s in range(layout["n"])]


def _layers(layout, kets):
    n = layout["n"]
    bras = [dagger(k) for k in kets]
    bonds = []
    for s, ks, t, kt in layout["bonds"]:
        bonds.append((s, ks, t, kt))
        bonds.append((n + s, kets[s].rank - 1 - ks, n + t, kets[t].rank - 1 - kt))
    return bras, bonds


def norm_network(layout, kets):
    """<Psi|Psi> = F(bra_{N-1} ... bra_0 ket_0 ... ket_{N-1}) (Fig. 4a): the bra
    layer (daggers, reversed site order) precedes the ket layer.  Tensor ids:
    ket s -> s, bra s -> n + s."""
    n = layout["n"]
    bras, bonds = _layers(layout, kets)
    for s in range(n):
        bonds.append((n + s, 0, s, kets[s].rank - 1))
    pos = [n + s for s in range(n)] + [n - 1 - s for s in range(n)]
    return Network(list(kets) + bras, bonds, pos)


def term_network(layout, kets, op, sites):
    """<Psi|h_t|Psi> with the operator O (from :func:`hop_gate` or
    :func:`onsite_gate`) between the bra and ket layers.  Ids: ket s -> s,
    bra s -> n + s, operator -> 2n; ``sites`` are the (ordered) sites of O."""
    n = layout["n"]
    bras, bonds = _layers(layout, kets)
    sites = list(sites)
    for s in range(n):
        if s not in sites:
            bonds.append((n + s, 0, s, kets[s].rank - 1))
    k = len(sites)
    for q, s in enumerate(sites):
        bonds.append((n + s, 0, 2 * n, q))  # bra side of O, in site order
        bonds.append((2 * n, 2 * k - 1 - q, s, kets[s].rank - 1))  # ket side, reversed
    pos = [n + 1 + s for s in range(n)] + [n - 1 - s for s in range(n)] + [n]
    return Network(list(kets) + bras + [op], bonds, pos)


def ket_amplitudes(layout, kets, mode="local"):
    """psi(n_0 ... n_{N-1}): the ket network contracted in site order, so its
    open physical legs come out in site order."""
    n = layout["n"]
    net = Network(kets, layout["bonds"], list(range(n)))
    tree = []
    cur = 0
    for s in range(1, n):
        tree.append((cur, s))
        cur = n + s - 1
    if n == 1:
        return kets[0]
    res, _, ids = contract_tree(net, tree, mode=mode)
    want = [(s, kets[s].rank - 1) for s in range(n)]
    perm = [ids.index(w) for w in want]
    return transpose(res, perm)


def ed_energy(psi, n, edges, t, u):
    """<psi|H|psi>/<psi|psi> for the Hubbard Hamiltonian of Eq.
    (fermi-hubbard-ham) built densely by Jordan-Wigner on 2n modes
    (site s: modes 2s = up, 2s+1 = down)."""
    c = jw_annihilators(2 * n)
    dim = 4**n
    h = np.zeros((dim, dim))
    for a, b in edges:
        for sig in (0, 1):
            ca, cb = c[2 * a + sig], c[2 * b + sig]
            h += -t * (ca.T @ cb + cb.T @ ca)
    for s in range(n):
        h += u * (c[2 * s].T @ c[2 * s]) @ (c[2 * s + 1].T @ c[2 * s + 1])
    vec = np.zeros(dim)
    for idx in np.ndindex(*([4] * n)):
        vec[_fock_index([LOCAL_OCC[v] for v in idx])] = psi.data[idx]
    return float(vec @ h @ vec / (vec @ vec))


def energy_terms(layout, kets, t, u, tree_fn, mode="local", policy="exact", chi=None):
    """Sum over terms of <h_t>/<Psi|Psi>, each term and the norm contracted by
    the tree ``tree_fn(op_sites)`` (a double-layer SSA tree).  Returns
    (energy, norm_mantissa, norm_log_scale, per-term ratios)."""
    nt, nlog, _ = contract_tree(norm_network(layout, kets), tree_fn(()), mode=mode, policy=policy, chi=chi, normalize=True)
    norm_m = float(nt.data)
    ratios = []
    hop = hop_gate(t)
    for a, b in layout["edges"]:
        net = term_network(layout, kets, hop, (a, b))
        r, lg, _ = contract_tree(net, tree_fn((a, b)), mode=mode, policy=policy, chi=chi, normalize=True)
        ratios.append(float(r.data) / norm_m * np.exp(lg - nlog))
    on = onsite_gate(u)
    for s in range(layout["n"]):
        net = term_network(layout, kets, on, (s,))
        r, lg, _ = contract_tree(net, tree_fn((s,)), mode=mode, policy=policy, chi=chi, normalize=True)
        ratios.append(float(r.data) / norm_m * np.exp(lg - nlog))
    return float(sum(ratios)), norm_m, nlog, ratios
