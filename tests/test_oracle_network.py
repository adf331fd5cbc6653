"""Pins of the oracle's network executor: brute force, order independence,
global == local on a DAG, norm = sum psi^2, and exact diagonalisation.

Config of the 2x2 norm: open 2x2 square lattice, physical dimension 4 (even
{0, updown}, odd {up, down}), bond D = 2 (1 even + 1 odd), N(0,1) entries,
even site tensors.
"""
import numpy as np
import pytest

import oracle as O
import workloads as W


def setup_2x2(D=(1, 1), seed=0):
    n, edges = W.square_lattice(2, 2)
    lay = W.peps_layout(n, edges, D, (2, 2))
    kets = O.ket_tensors(lay, W.random_peps(lay, seed))
    return n, edges, lay, kets


@pytest.mark.parametrize("D,seed", [((1, 1), 0), ((2, 1), 1), ((1, 2), 2)])
def test_norm_brute_force_local_global(D, seed):
    n, edges, lay, kets = setup_2x2(D, seed)
    net = O.norm_network(lay, kets)
    assert O.arrows_from_positions(net)
    bf = O.brute_force_global(net)
    psi = O.ket_amplitudes(lay, kets)
    assert bf > 0
    assert abs(bf - np.sum(psi.data**2)) <= 1e-12 * abs(bf)
    edges8 = [(b[0], b[2]) for b in net.bonds]
    trees = [W.connected_random_tree(2 * n, edges8, s) for s in range(40)]
    trees += [W.random_tree(2 * n, s) for s in range(20)]
    for mode in ("local", "global"):
        for tr in trees:
            r, lg, _ = O.contract_tree(net, tr, mode=mode)
            assert abs(float(r.data) - bf) <= 1e-12 * abs(bf), (mode, tr)


def test_norm_two_orders_two_conventions():
    """Row-first and column-first site orders, in both formalisms."""
    n, edges, lay, kets = setup_2x2()
    net = O.norm_network(lay, kets)
    bf = O.brute_force_global(net)
    for order in ([0, 1, 2, 3], [0, 2, 1, 3]):
        tree = W.double_layer_tree(n, W.site_sweep_tree(order))
        for mode in ("local", "global"):
            r, lg, _ = O.contract_tree(net, tree, mode=mode, normalize=True)
            assert abs(float(r.data) * np.exp(lg) - bf) <= 1e-12 * bf


def test_local_formalism_on_non_dag_arrows():
    """Reversing one bond's arrow (flipping both duals) while inserting the
    bond parity on that bond leaves the local value unchanged (Fig. 3b)."""
    n, edges, lay, kets = setup_2x2((2, 1), 4)
    net = O.norm_network(lay, kets)
    ref = float(O.contract_tree(net, W.connected_random_tree(8, [(b[0], b[2]) for b in net.bonds], 0))[0].data)
    t1, l1, t2, l2 = net.bonds[0]
    ts = list(net.tensors)
    a = ts[t1]
    a = O.flip_legs(a, [l1])
    a = O.GTensor(a.data, [lg if k != l1 else (lg[0], lg[1], 1 - lg[2]) for k, lg in enumerate(a.legs)], a.parity)
    b = ts[t2]
    b = O.GTensor(b.data, [lg if k != l2 else (lg[0], lg[1], 1 - lg[2]) for k, lg in enumerate(b.legs)], b.parity)
    ts[t1], ts[t2] = a, b
    net2 = O.Network(ts, net.bonds)
    for s in range(10):
        tr = W.connected_random_tree(8, [(b[0], b[2]) for b in net.bonds], s)
        assert abs(float(O.contract_tree(net2, tr)[0].data) - ref) <= 1e-12 * abs(ref)


@pytest.mark.parametrize("D,seed,U", [((1, 1), 0, 8.0), ((2, 1), 3, 4.0), ((1, 2), 5, 6.0)])
def test_energy_matches_exact_diagonalisation(D, seed, U):
    """<psi|H|psi>/<psi|psi> from a dense Jordan-Wigner Hamiltonian in the
    256-state Fock space equals the sum of per-term network contractions."""
    n, edges, lay, kets = setup_2x2(D, seed)
    psi = O.ket_amplitudes(lay, kets)
    e_ed = O.ed_energy(psi, n, edges, 1.0, U)
    for mode in ("local", "global"):
        for order in ([0, 1, 2, 3], [3, 1, 2, 0]):
            st = W.site_sweep_tree(order)
            e, *_ = O.energy_terms(lay, kets, 1.0, U, lambda ops: W.double_layer_tree(n, st, ops), mode=mode)
            assert abs(e - e_ed) <= 1e-11 * abs(e_ed), (mode, order)


def test_ed_hopping_sign_with_jw_string():
    """Single-bond check on 2x2 where the bond (0, 2) skips site 1: the JW
    string of the skipped site must enter; a gate without it differs."""
    n, edges, lay, kets = setup_2x2((1, 1), 7)
    psi = O.ket_amplitudes(lay, kets)
    e_ed = O.ed_energy(psi, n, [(0, 2)], 1.0, 0.0)
    st = W.site_sweep_tree([0, 1, 2, 3])
    norm, nlog = None, None
    nt, nlog, _ = O.contract_tree(O.norm_network(lay, kets), W.double_layer_tree(n, st), normalize=True)
    net = O.term_network(lay, kets, O.hop_gate(1.0), (0, 2))
    r, lg, _ = O.contract_tree(net, W.double_layer_tree(n, st, (0, 2)), normalize=True)
    val = float(r.data) / float(nt.data) * np.exp(lg - nlog)
    assert abs(val - e_ed) <= 1e-11 * abs(e_ed)


def test_planted_mistakes_are_caught(monkeypatch):
    """Mutations planted in the oracle (on the CPU) must break a pin."""
    n, edges, lay, kets = setup_2x2((1, 1), 0)
    net = O.norm_network(lay, kets)
    bf = O.brute_force_global(net)
    tr = W.connected_random_tree(8, [(b[0], b[2]) for b in net.bonds], 3)
    import oracle.graded as G
    import oracle.network as N

    good_transpose = G.transpose

    # 1. transposition sign dropped
    def no_sign_transpose(t, perm):
        return G.GTensor(np.transpose(t.data, perm), [t.legs[p] for p in perm], t.parity)

    monkeypatch.setattr(G, "transpose", no_sign_transpose)
    bad = float(O.contract_tree(net, tr)[0].data)
    monkeypatch.setattr(G, "transpose", good_transpose)
    assert abs(bad - bf) > 1e-6 * abs(bf)

    # 2. arrow (bond parity) ignored in the local formalism
    good_contract = N.contract

    def no_arrow(x, y, ax, ay, arrows=True, flip_x=(), flip_y=()):
        return good_contract(x, y, ax, ay, arrows=False, flip_x=flip_x, flip_y=flip_y)

    monkeypatch.setattr(N, "contract", no_arrow)
    vals = [float(O.contract_tree(net, W.connected_random_tree(8, [(b[0], b[2]) for b in net.bonds], s))[0].data) for s in range(10)]
    monkeypatch.setattr(N, "contract", good_contract)
    assert max(abs(v - bf) for v in vals) > 1e-6 * abs(bf)

    # 3. gate with its ket-side legs in site order instead of reversed
    psi = O.ket_amplitudes(lay, kets)
    e_ed = O.ed_energy(psi, n, edges, 1.0, 8.0)
    good_gate = O.hubbard.hop_gate

    def swapped_gate(t):
        g = good_gate(t)
        return G.GTensor(np.transpose(g.data, [0, 1, 3, 2]), g.legs, 0)

    monkeypatch.setattr(O.hubbard, "hop_gate", swapped_gate)
    st = W.site_sweep_tree([0, 1, 2, 3])
    e_bad, *_ = O.energy_terms(lay, kets, 1.0, 8.0, lambda ops: W.double_layer_tree(n, st, ops))
    monkeypatch.setattr(O.hubbard, "hop_gate", good_gate)
    assert abs(e_bad - e_ed) > 1e-6
