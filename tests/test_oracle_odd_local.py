"""Odd-parity tensors in the locally ordered formalism (Sec. II.D): each odd
tensor gets a size-1 odd dummy leg, the network is contracted as an even one
and the dummy legs left on the result are sorted by decreasing tensor index.
Pinned against the brute-force globally ordered value (tensors in index
order, arrows of the DAG of that order) on random networks with cycles and
an even number of odd tensors; sorting the dummy legs the other way breaks
the pin."""
import numpy as np
import pytest

import oracle as O
import oracle.network as ON
import workloads as W


def rand_net(seed, m=5, extra=3):
    g = np.random.default_rng(seed)
    edges = [(i, i + 1) for i in range(m - 1)]
    while len(edges) < m - 1 + extra:
        a, b = sorted(int(x) for x in g.choice(m, 2, replace=False))
        if (a, b) not in edges:
            edges.append((a, b))
    legs = [[] for _ in range(m)]
    bonds = []
    for a, b in edges:
        d0, d1 = int(g.integers(1, 3)), int(g.integers(1, 3))
        la, lb = len(legs[a]), len(legs[b])
        legs[a].append((d0, d1, 1))  # the earlier tensor holds the '-' leg
        legs[b].append((d0, d1, 0))
        bonds.append((a, la, b, lb))
    odd = set(int(x) for x in g.choice(m, 2 * int(g.integers(1, m // 2 + 1)), replace=False))
    blocks = [W.random_blocks(legs[i], 1 if i in odd else 0, 100 * seed + i) for i in range(m)]
    tens = [O.embed_blocks(legs[i], 1 if i in odd else 0, blocks[i]) for i in range(m)]
    return ON.Network(tens, bonds, list(range(m))), legs, blocks, sorted(odd)


def trees_of(net, k=4):
    edges = [(b[0], b[2]) for b in net.bonds]
    return [W.connected_random_tree(len(net.tensors), edges, s) for s in range(k)]


@pytest.mark.parametrize("seed", range(12))
def test_local_odd_equals_global_brute_force(seed):
    net, *_ = rand_net(seed)
    bf = O.brute_force_global(net)
    for tr in trees_of(net):
        g, _, _ = O.contract_tree(net, tr, mode="global")
        v, _, _ = O.contract_tree(net, tr, mode="local")
        assert abs(float(g.data) - bf) <= 1e-10 * abs(bf)
        assert abs(float(v.data) - bf) <= 1e-10 * abs(bf), (seed, tr)


def test_reversed_dummy_order_breaks_the_pin(monkeypatch):
    monkeypatch.setattr(ON, "DUMMY_ORDER_DESCENDING", False)
    wrong = 0
    for seed in range(12):
        net, *_ = rand_net(seed)
        bf = O.brute_force_global(net)
        for tr in trees_of(net):
            v, _, _ = O.contract_tree(net, tr, mode="local")
            wrong += abs(float(v.data) - bf) > 1e-10 * abs(bf)
    assert wrong > 0


def test_odd_tensor_count_odd_gives_zero():
    """A closed network with an odd number of odd tensors has odd total
    parity: its value is zero in both formalisms."""
    net, legs, blocks, odd = rand_net(3)
    i = next(k for k in range(len(legs)) if k not in odd)
    t = O.embed_blocks(legs[i], 1, W.random_blocks(legs[i], 1, 77))
    tens = list(net.tensors)
    tens[i] = t
    net2 = ON.Network(tens, net.bonds, net.positions)
    assert abs(O.brute_force_global(net2)) == 0.0
    for tr in trees_of(net2, 2):
        assert abs(float(O.contract_tree(net2, tr, mode="local")[0].data)) == 0.0
