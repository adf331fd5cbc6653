"""Pins of the oracle's cluster approximation (Sec. V) against facts that do
not come from it:

* a cluster that covers the whole graph has no dangling bond, so its energy
  is the exact energy (the full-network contraction, and exact
  diagonalisation on 2x2);
* an exact-environment identity: a leaf site whose tensor puts weight
  lambda_k on one physical state of parity p(k) has the double layer
  diag(lambda^2) -- exactly the gauge that closes its bond -- so a cluster
  whose every dangling bond leads to such a leaf reproduces the exact term
  (path 0-1-2-3 and a star), and a planted sign flip on the odd gauge
  entries breaks it;
* the cluster network contracted along its tree equals the literal
  global-formalism brute force.
"""
import numpy as np
import pytest

import oracle as O
import workloads as W
from oracle.network import brute_force_global, contract_tree


def cfn(lay, r):
    def f(targets):
        sites = W.cluster_sites(lay, targets, r)
        return (sites, W.dangling_bonds(lay, sites), W.cluster_tree(lay, sites, targets, True),
                W.cluster_tree(lay, sites, targets, False))
    return f


def exact_terms(lay, kets):
    n = lay["n"]
    st = W.site_sweep_tree(list(range(n)))
    return O.energy_terms(lay, kets, 1.0, 8.0, lambda ops: W.double_layer_tree(n, st, ops), mode="global")


def test_whole_graph_cluster_is_exact_2x2():
    n, e = W.square_lattice(2, 2)
    lay = W.peps_layout(n, e, (1, 1), (2, 2))
    kets = O.ket_tensors(lay, W.random_peps(lay, 0))
    ce, _ = O.cluster_energy(lay, kets, 1.0, 8.0, cfn(lay, 2), W.bond_gauges(lay))
    ex = exact_terms(lay, kets)[0]
    ed = O.ed_energy(O.ket_amplitudes(lay, kets), n, e, 1.0, 8.0)
    assert abs(ce - ex) <= 1e-12 * abs(ex) and abs(ce - ed) <= 1e-10 * abs(ed)


def test_whole_graph_cluster_is_exact_regular_graph():
    n, e = W.random_regular_graph(6, 3, 2)
    lay = W.peps_layout(n, e, (1, 1), (2, 2))
    kets = O.ket_tensors(lay, W.random_peps(lay, 4))
    ce, rat = O.cluster_energy(lay, kets, 1.0, 8.0, cfn(lay, 6), W.bond_gauges(lay))
    ex, _, _, rex = exact_terms(lay, kets)
    assert np.allclose(rat, rex, rtol=1e-11, atol=1e-12)


def leafy(lay, blocks, gauges, leaves):
    """Ket tensors with every site in ``leaves`` (one virtual leg) replaced by
    the exact-environment tensor T[k, p] = lambda_k on the first physical state
    of parity p(k)."""
    kets = O.ket_tensors(lay, blocks)
    for leaf in leaves:
        nb = lay["nbrs"][leaf][0]
        lam = gauges[(min(leaf, nb), max(leaf, nb))]
        legs = lay["legs"][leaf]
        assert legs[0][:2] == (1, 1), "one even and one odd virtual state"
        d = np.zeros([a + b for a, b, _ in legs])
        d[0, 0] = lam[0][0]  # even virtual state -> first even physical state
        d[1, legs[1][0]] = lam[1][0]  # odd virtual state -> first odd physical state
        kets[leaf] = O.GTensor(d, legs, 0)
    return kets


def one_term(lay, kets, gauges, targets, op, r, gfun=None):
    import oracle.cluster as OC

    orig = OC.gauge_tensor
    if gfun is not None:
        OC.gauge_tensor = gfun
    try:
        sites, dang, tro, trn = cfn(lay, r)(list(targets))
        num = OC.cluster_network(lay, kets, sites, dang, gauges, op, targets)
        den = OC.cluster_network(lay, kets, sites, dang, gauges)
        rn, ln, _ = contract_tree(num, tro, mode="global", normalize=True)
        rd, ld, _ = contract_tree(den, trn, mode="global", normalize=True)
        return float(rn.data) / float(rd.data) * np.exp(ln - ld)
    finally:
        OC.gauge_tensor = orig


@pytest.mark.parametrize("seed", [3, 4])
def test_exact_environment_path(seed):
    n, e = 4, [(0, 1), (1, 2), (2, 3)]
    lay = W.peps_layout(n, e, (1, 1), (2, 2))
    gs = W.bond_gauges(lay, decay=0.6)
    kets = leafy(lay, W.random_peps(lay, seed), gs, [0, 3])
    rex = exact_terms(lay, kets)[3]
    got = one_term(lay, kets, gs, (1, 2), O.hop_gate(1.0), 0)
    assert abs(got - rex[1]) <= 1e-12 * abs(rex[1])


def test_exact_environment_star():
    n, e = 4, [(0, 1), (0, 2), (0, 3)]
    lay = W.peps_layout(n, e, (1, 1), (2, 2))
    gs = W.bond_gauges(lay, decay=0.7)
    kets = leafy(lay, W.random_peps(lay, 5), gs, [1, 2, 3])
    _, _, _, rex = exact_terms(lay, kets)
    # terms: hop (0,1), (0,2), (0,3), then U_0..U_3
    assert abs(one_term(lay, kets, gs, (0,), O.onsite_gate(8.0), 0) - rex[3]) <= 1e-12 * abs(rex[3])
    assert abs(one_term(lay, kets, gs, (0, 2), O.hop_gate(1.0), 0) - rex[1]) <= 1e-12 * abs(rex[1])


def test_planted_odd_gauge_sign_breaks_the_identity():
    import oracle.cluster as OC

    n, e = 4, [(0, 1), (1, 2), (2, 3)]
    lay = W.peps_layout(n, e, (1, 1), (2, 2))
    gs = W.bond_gauges(lay, decay=0.6)
    kets = leafy(lay, W.random_peps(lay, 3), gs, [0, 3])
    rex = exact_terms(lay, kets)[3]
    orig = OC.gauge_tensor
    got = one_term(lay, kets, gs, (1, 2), O.hop_gate(1.0), 0, gfun=lambda a, b, d: flipped_with(orig, a, b, d))
    assert abs(got - rex[1]) > 1e-3


def flipped_with(orig, le, lo, d):
    g = orig(le, lo, d)
    data = g.data.copy()
    data[len(le):, len(le):] *= -1
    return O.GTensor(data, g.legs, g.parity)


def test_cluster_network_tree_equals_brute_force():
    n, e = W.square_lattice(2, 3)
    lay = W.peps_layout(n, e, (1, 1), (2, 2))
    kets = O.ket_tensors(lay, W.random_peps(lay, 6))
    gs = W.bond_gauges(lay)
    for targets, op in (((1,), O.onsite_gate(8.0)), ((0, 1), O.hop_gate(1.0))):
        sites, dang, tro, _ = cfn(lay, 0)(list(targets))
        net = O.cluster_network(lay, kets, sites, dang, gs, op, targets)
        r, lg, _ = contract_tree(net, tro, mode="global", normalize=True)
        bf = brute_force_global(net)
        assert abs(float(r.data) * np.exp(lg) - bf) <= 1e-12 * abs(bf)
