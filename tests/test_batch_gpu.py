"""Batched contraction of many networks (ftn_contract_batch): every network
of a batch gives exactly (bit for bit) what it gives alone through
ftn_contract -- the batch merges job tables but keeps each network's plans,
tiles and reduction orders -- and the batched energies agree with the
oracle.  Covered: cluster networks of random 3-regular graphs (globally
ordered) in FP64, TF32x3 and F16X3, exact and late policies (the batched
compression stages), intermediates above the one-CTA normalisation size,
locally and globally ordered networks with different trees, policies and chi
in one batch, and the error paths."""
import pytest

import oracle as O
import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def F():
    import torch

    from paper_2410_02215_gb300 import ftn

    assert torch.cuda.is_available()
    ftn.lib()
    return ftn


@pytest.fixture(scope="module")
def ctx(F):
    c = F.Context()
    yield c
    c.synchronize()
    c.close()


def cfn(lay, r):
    def f(targets):
        sites = W.cluster_sites(lay, targets, r)
        return (sites, W.dangling_bonds(lay, sites), W.cluster_tree(lay, sites, targets, True),
                W.cluster_tree(lay, sites, targets, False))
    return f


def cluster_nets(F, ctx, n, D, seed, r, policy, chi, dt, limit=None):
    """Cluster networks (with and without the operator) of the first
    ``limit`` terms of a random 3-regular graph; returns (networks, the
    tensors they borrow)."""
    from paper_2410_02215_gb300 import peps

    n, e = W.random_regular_graph(n, 3, seed)
    lay = W.peps_layout(n, e, D, (2, 2))
    blocks, gs = W.random_peps(lay, seed), W.bond_gauges(lay)
    kets = [F.Tensor.from_blocks(ctx, lay["legs"][s], 0, blocks[s], dt) for s in range(n)]
    bras = [F.dagger(ctx, k) for k in kets]
    hop = F.hubbard_term(ctx, 0, 1.0, 0.0, dt)
    onsite = F.hubbard_term(ctx, 1, 0.0, 8.0, dt)
    cache = {}

    def gauge_of(s, a):
        if (s, a) not in cache:
            nb = lay["nbrs"][s][a]
            lam = gs[(min(s, nb), max(s, nb))]
            cache[(s, a)] = peps.gauge_tensor(ctx, lam[0], lam[1], kets[s].legs[a][2], dt)
        return cache[(s, a)]

    f = cfn(lay, r)
    nets = []
    terms = [((a, b), hop) for a, b in lay["edges"]] + [((s,), onsite) for s in range(n)]
    for targets, op in terms[:limit]:
        sites, dang, t_op, t_norm = f(list(targets))
        for o, tree in ((op, t_op), (None, t_norm)):
            tens, bonds, pos = peps.cluster_network(lay, kets, bras, sites, dang, gauge_of, o, targets)
            nets.append({"tensors": tens, "bonds": bonds, "tree": tree, "positions": pos, "policy": policy,
                         "chi": chi})
    return nets, (kets, bras, cache, hop, onsite)


def singles(F, ctx, nets, prec):
    return [F.contract(ctx, j["tensors"], j["bonds"], j["tree"], positions=j.get("positions"),
                       policy=j.get("policy", "exact"), chi=j.get("chi", 0), prec=prec) for j in nets]


@pytest.mark.parametrize("prec", ["f64", "tf32x3", "f16x3"])
@pytest.mark.parametrize("policy,chi", [("exact", 0), ("late", 4)])
def test_batch_equals_single_cluster_networks(F, ctx, prec, policy, chi):
    dt = F.F64 if prec == "f64" else F.F32
    nets, keep = cluster_nets(F, ctx, 12, (2, 1), 3, 1, policy, chi, dt)
    ref = singles(F, ctx, nets, prec)
    assert F.contract_batch(ctx, nets, prec=prec) == ref
    # the same networks split over two batches
    assert F.contract_batch(ctx, nets[:7], prec=prec) + F.contract_batch(ctx, nets[7:], prec=prec) == ref


@pytest.mark.parametrize("prec", ["f64", "tf32x3", "f16x3"])
def test_batch_large_intermediates_and_compression(F, ctx, prec):
    """D = 6 (4+2) bonds, late compression to chi = 32: merged-site
    intermediates of ~10^6 entries (the multi-CTA normalisation), batched
    Gram / Cholesky / Jacobi / projector stages, tensor-core tiles of several
    widths."""
    dt = F.F64 if prec == "f64" else F.F32
    nets, keep = cluster_nets(F, ctx, 8, (4, 2), 11, 1, "late", 32, dt, limit=5)
    assert F.contract_batch(ctx, nets, prec=prec) == singles(F, ctx, nets, prec)


def test_batch_mixed_networks(F, ctx):
    """Locally and globally ordered norm / term networks of a 3x3 lattice
    with different trees, policies and chi in one batch."""
    from paper_2410_02215_gb300 import peps

    n, e = W.square_lattice(3, 3)
    lay = W.peps_layout(n, e, (1, 1), (2, 2))
    blocks = W.random_peps(lay, 4)
    kets = [F.Tensor.from_blocks(ctx, lay["legs"][s], 0, blocks[s]) for s in range(n)]
    bras = [F.dagger(ctx, k) for k in kets]
    hop = F.hubbard_term(ctx, 0, 1.0, 0.0, F.F64)
    nets = []
    for q, (glob, policy, chi) in enumerate([(True, "exact", 0), (False, "exact", 0), (True, "late", 2),
                                             (False, "early", 3), (True, "early", 2), (False, "late", 3)]):
        order = list(range(n)) if q < 3 else [4, 3, 5, 1, 7, 0, 2, 6, 8]
        if q % 2 == 0:
            tens, bonds, pos = peps.norm_network(ctx, lay, kets, bras)
            tree = W.double_layer_tree(n, W.site_sweep_tree(order))
        else:
            a, b = lay["edges"][q]
            tens, bonds, pos = peps.term_network(lay, kets, bras, hop, (a, b))
            tree = W.double_layer_tree(n, W.site_sweep_tree(order), (a, b))
        nets.append({"tensors": tens, "bonds": bonds, "tree": tree, "positions": pos if glob else None,
                     "policy": policy, "chi": chi})
    assert F.contract_batch(ctx, nets) == singles(F, ctx, nets, "f64")


def test_batch_cluster_energy_matches_oracle(F, ctx):
    import torch

    from paper_2410_02215_gb300 import peps

    n, e = W.random_regular_graph(10, 3, 7)
    lay = W.peps_layout(n, e, (1, 1), (2, 2))
    blocks, gs = W.random_peps(lay, 7), W.bond_gauges(lay)
    ref, rref = O.cluster_energy(lay, O.ket_tensors(lay, blocks), 1.0, 8.0, cfn(lay, 2), gs, policy="late", chi=4)
    kets = [F.Tensor.from_blocks(ctx, lay["legs"][s], 0, blocks[s]) for s in range(n)]
    en, rat = peps.cluster_energy(ctx, lay, kets, 1.0, 8.0, cfn(lay, 2), gs, policy="late", chi=4, batch=16)
    assert max(abs(x - y) for x, y in zip(rat, rref)) <= 1e-9 * max(abs(y) for y in rref)  # normwise over terms
    assert abs(en - ref) <= 1e-9 * abs(ref)
    # several instances at once, batches spread over two streams
    c2 = F.Context(stream=torch.cuda.Stream())
    try:
        out = peps.cluster_energies([ctx, c2], [(lay, kets, cfn(lay, 2), gs)] * 2, 1.0, 8.0, policy="late", chi=4,
                                    batch=32)
        assert out[0] == (en, rat) and out[1] == (en, rat)
    finally:
        c2.synchronize()
        c2.close()


def test_batch_energy_equals_single(F, ctx):
    from paper_2410_02215_gb300 import peps

    n, e = W.square_lattice(3, 3)
    lay = W.peps_layout(n, e, (2, 2), (2, 2))
    blocks = W.random_peps(lay, 2)
    kets = [F.Tensor.from_blocks(ctx, lay["legs"][s], 0, blocks[s]) for s in range(n)]

    def tf(ops):
        return W.double_layer_tree(n, W.site_sweep_tree(list(range(n))), ops)

    a = peps.energy(ctx, lay, kets, 1.0, 8.0, tf, mode="global", policy="late", chi=8)
    b = peps.energy(ctx, lay, kets, 1.0, 8.0, tf, mode="global", policy="late", chi=8, batch=8)
    assert a == b


def test_batch_errors(F, ctx):
    nets, keep = cluster_nets(F, ctx, 8, (1, 1), 5, 1, "exact", 0, F.F64, limit=3)
    assert F.contract_batch(ctx, []) == []
    bad = dict(nets[1])
    bad["tree"] = [(0, 0)] + list(bad["tree"][1:])  # a tensor paired with itself
    with pytest.raises(F.FtnError):
        F.contract_batch(ctx, [nets[0], bad, nets[2]])
    with pytest.raises(F.FtnError):
        F.contract_batch(ctx, nets, prec="tf32x3")  # FP64 tensors on a tensor-core precision
    # the context is still usable
    assert F.contract_batch(ctx, nets) == singles(F, ctx, nets, "f64")
