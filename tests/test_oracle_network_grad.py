"""Pins of the oracle's network gradient (oracle.network_grad): reverse mode
through the contraction tree and its compressions.

* the value is the value of oracle.contract_tree (same walk), in the
  locally and in the globally ordered formalism;
* exact contraction is linear in every tensor, so v = sum(T_i * dv/dT_i) for
  each input tensor T_i (Euler's identity for a function linear in T_i);
* with late or early compression at a truncating chi (gaps checked), the
  gradient equals central finite differences of oracle.contract_tree on 20
  seeded entries (the check of the fPEPS gradient workload, on a small
  lattice the oracle contracts in milliseconds);
* a planted mistake in the compression adjoint (the SVD rule without its
  projection terms) fails the finite differences at network level.
"""
import numpy as np
import pytest

import oracle as O
import oracle.network_grad as NG
import workloads as W


def setup(lx, ly, D, seed):
    n, edges = W.square_lattice(lx, ly)
    lay = W.peps_layout(n, edges, D, (2, 2))
    kets = O.ket_tensors(lay, W.random_peps(lay, seed))
    net = O.norm_network(lay, kets)
    tree = W.double_layer_tree(n, W.site_sweep_tree(list(range(n))))
    return net, tree


def value(net, tree, policy, chi, mode="local"):
    return float(O.contract_tree(net, tree, mode=mode, policy=policy, chi=chi)[0].data)


def allowed_entries(t):
    par = [O.index_parity(d0, d1) for d0, d1, _ in t.legs]
    out = []
    for idx in np.ndindex(*t.data.shape):
        if sum(int(par[k][i]) for k, i in enumerate(idx)) % 2 == t.parity:
            out.append(idx)
    return out


def fd_check(net, tree, policy, chi, grads, samples=20, seed=0, h=1e-6, scale=None, mode="local"):
    rng = np.random.default_rng(seed)
    worst = 0.0
    if scale is None:
        scale = max(np.max(np.abs(g.data)) for g in grads)
    for _ in range(samples):
        i = int(rng.integers(len(net.tensors)))
        ents = allowed_entries(net.tensors[i])
        idx = ents[int(rng.integers(len(ents)))]
        vals = []
        for sgn in (1.0, -1.0):
            tensors = list(net.tensors)
            d = tensors[i].data.copy()
            d[idx] += sgn * h
            tensors[i] = O.GTensor(d, tensors[i].legs, tensors[i].parity)
            vals.append(value(O.Network(tensors, net.bonds, net.positions), tree, policy, chi, mode))
        fd = (vals[0] - vals[1]) / (2 * h)
        worst = max(worst, abs(fd - grads[i].data[idx]) / scale)
    return worst


@pytest.mark.parametrize("mode", ["local", "global"])
@pytest.mark.parametrize("lx,ly,D", [(2, 2, (1, 1)), (2, 3, (1, 1)), (2, 2, (2, 1))])
@pytest.mark.parametrize("policy,chi", [("exact", None), ("late", 2), ("early", 2)])
def test_value_is_the_executor_value(lx, ly, D, policy, chi, mode):
    net, tree = setup(lx, ly, D, 1)
    v, _, _ = NG.contract_tree_grad(net, tree, policy, chi, mode=mode)
    assert v == value(net, tree, policy, chi, mode)


@pytest.mark.parametrize("mode", ["local", "global"])
@pytest.mark.parametrize("lx,ly,D", [(2, 2, (1, 1)), (2, 3, (1, 1)), (2, 2, (2, 1))])
def test_exact_gradient_satisfies_euler_identity(lx, ly, D, mode):
    net, tree = setup(lx, ly, D, 2)
    v, grads, _ = NG.contract_tree_grad(net, tree, mode=mode)
    for t, g in zip(net.tensors, grads):
        assert abs(float(np.sum(t.data * g.data)) - v) <= 1e-12 * abs(v)


@pytest.mark.parametrize("mode", ["local", "global"])
@pytest.mark.parametrize("lx,ly,D,chi", [(2, 2, (1, 1), 2), (2, 3, (1, 1), 2), (2, 2, (2, 1), 3)])
@pytest.mark.parametrize("policy", ["late", "early"])
def test_truncated_gradient_matches_finite_differences(lx, ly, D, chi, policy, mode):
    net, tree = setup(lx, ly, D, 3)
    v, grads, gap = NG.contract_tree_grad(net, tree, policy, chi, mode=mode)
    assert gap is not None and gap > 1e-4  # truncation happens, away from a degeneracy
    assert v != value(net, tree, "exact", None, mode)
    assert fd_check(net, tree, policy, chi, grads, mode=mode) < 1e-6


def test_planted_mistake_fails_the_finite_differences(monkeypatch):
    net, tree = setup(2, 3, (1, 1), 3)
    _, good, _ = NG.contract_tree_grad(net, tree, "late", 2)
    scale = max(np.max(np.abs(g.data)) for g in good)
    assert fd_check(net, tree, "late", 2, good) < 1e-6
    import oracle.compress_adjoint as CA

    good_svd = CA._svd_backward

    def svd_without_projections(u, s, v, du, ds, dv, keep):
        # the SVD rule without its (I - U U^T) and (I - V V^T) terms
        full = good_svd(u, s, v, du, ds, dv, keep)
        sinv = np.zeros(len(s))
        sinv[:keep] = 1.0 / s[:keep]
        full = full - (np.eye(u.shape[0]) - u @ u.T) @ du @ np.diag(sinv) @ v.T
        return full - u @ np.diag(sinv) @ dv.T @ (np.eye(v.shape[0]) - v @ v.T)

    monkeypatch.setattr(CA, "_svd_backward", svd_without_projections)
    _, bad, _ = NG.contract_tree_grad(net, tree, "late", 2)
    assert fd_check(net, tree, "late", 2, bad, scale=scale) > 1e-3
