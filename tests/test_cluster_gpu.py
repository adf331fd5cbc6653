"""Parity of the cluster approximation (Sec. V) on the GPU with the oracle:
random 3-regular graphs, radius 0-2, every hopping and on-site term as the
ratio of its cluster network with and without the operator, contracted in
the globally ordered formalism.  Tolerances: FP64 1e-10 per term (relative
normwise over the terms, and relative on the energy); the mixed path (FP32 tensors, TF32x3 GEMMs, FP64
compression) 1e-6 relative on the energy."""
import numpy as np
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


def setup(n, D, seed):
    n, e = W.random_regular_graph(n, 3, seed)
    lay = W.peps_layout(n, e, D, (2, 2))
    return lay, W.random_peps(lay, seed), W.bond_gauges(lay)


@pytest.mark.parametrize("D,r", [((1, 1), 0), ((1, 1), 1), ((2, 1), 1), ((1, 1), 2)])
def test_cluster_energy_matches_oracle(F, ctx, D, r):
    from paper_2410_02215_gb300 import peps

    lay, blocks, gs = setup(10, D, 3)
    ref, rref = O.cluster_energy(lay, O.ket_tensors(lay, blocks), 1.0, 8.0, cfn(lay, r), gs)
    kets = [F.Tensor.from_blocks(ctx, lay["legs"][s], 0, blocks[s]) for s in range(lay["n"])]
    e, rat = peps.cluster_energy(ctx, lay, kets, 1.0, 8.0, cfn(lay, r), gs)
    assert max(abs(x - y) for x, y in zip(rat, rref)) <= 1e-10 * max(abs(y) for y in rref)
    assert abs(e - ref) <= 1e-10 * abs(ref)


def test_cluster_energy_streams_and_mixed(F, ctx):
    import torch

    from paper_2410_02215_gb300 import peps

    lay, blocks, gs = setup(12, (2, 1), 5)
    kets = [F.Tensor.from_blocks(ctx, lay["legs"][s], 0, blocks[s]) for s in range(lay["n"])]
    e1, r1 = peps.cluster_energy(ctx, lay, kets, 1.0, 8.0, cfn(lay, 1), gs)
    extra = [F.Context(stream=torch.cuda.Stream()) for _ in range(3)]
    try:
        e4, r4 = peps.cluster_energy([ctx] + extra, lay, kets, 1.0, 8.0, cfn(lay, 1), gs)
        assert (e4, r4) == (e1, r1)
        k32 = [F.Tensor.from_blocks(ctx, lay["legs"][s], 0, blocks[s], F.F32) for s in range(lay["n"])]
        e32, _ = peps.cluster_energy([ctx] + extra, lay, k32, 1.0, 8.0, cfn(lay, 1), gs, prec="tf32x3")
        assert abs(e32 - e1) <= 1e-6 * abs(e1)
    finally:
        for c in extra:
            c.synchronize()
            c.close()


def test_compressed_cluster_matches_oracle(F, ctx):
    """Late compression to chi = 4 inside radius-2 clusters: the same tree,
    policy and chi give the same truncations on both sides."""
    from paper_2410_02215_gb300 import peps

    lay, blocks, gs = setup(10, (1, 1), 7)
    ref, rref = O.cluster_energy(lay, O.ket_tensors(lay, blocks), 1.0, 8.0, cfn(lay, 2), gs, policy="late", chi=4)
    kets = [F.Tensor.from_blocks(ctx, lay["legs"][s], 0, blocks[s]) for s in range(lay["n"])]
    e, rat = peps.cluster_energy(ctx, lay, kets, 1.0, 8.0, cfn(lay, 2), gs, policy="late", chi=4)
    assert max(abs(x - y) for x, y in zip(rat, rref)) <= 1e-9 * max(abs(y) for y in rref)
