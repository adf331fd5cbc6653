"""The network gradient on the GPU (ftn_contract_grad) against the oracle's
(oracle.network_grad, pinned by finite differences and Euler's identity in
tests/test_oracle_network_grad.py): PEPS norm networks on 2x2 and 2x3 open
lattices with the site-sweep double-layer tree and on a 3x3 lattice with the
boundary-MPS row sweep, exact, late and early
compression at a truncating chi, in the locally and the globally ordered
formalism.  Value at 1e-10 (and equal to ftn_contract's normalised value),
every gradient entry at 1e-9 of the largest."""
import numpy as np
import pytest

import oracle as O
import oracle.network_grad as NG
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


def setup(lx, ly, D, seed, boundary=False):
    n, edges = W.square_lattice(lx, ly)
    lay = W.peps_layout(n, edges, D, (2, 2))
    kets = O.ket_tensors(lay, W.random_peps(lay, seed))
    net = O.norm_network(lay, kets)
    site_tree = W.boundary_mps_tree(lx, ly) if boundary else W.site_sweep_tree(list(range(n)))
    return net, W.double_layer_tree(n, site_tree)


def dense(t):
    return O.embed_blocks(t.legs, t.parity, t.to_blocks())


@pytest.mark.parametrize("mode", ["local", "global"])
@pytest.mark.parametrize("lx,ly,D,chi", [(2, 2, (1, 1), 2), (2, 3, (1, 1), 2), (2, 2, (2, 1), 3)])
@pytest.mark.parametrize("policy", ["exact", "late", "early"])
def test_network_grad_against_oracle(F, ctx, lx, ly, D, chi, policy, mode):
    net, tree = setup(lx, ly, D, 3)
    c = None if policy == "exact" else chi
    v_o, g_o, _ = NG.contract_tree_grad(net, tree, policy, c, mode=mode)
    tensors = [F.Tensor.from_blocks(ctx, t.legs, t.parity, sorted(O.extract_blocks(t).items())) for t in net.tensors]
    pos = list(net.positions) if mode == "global" else None
    v, grads = F.contract_grad(ctx, tensors, net.bonds, tree, positions=pos, policy=policy, chi=c or 0)
    assert abs(v - v_o) <= 1e-10 * abs(v_o)
    m, lg = F.contract(ctx, tensors, net.bonds, tree, positions=pos, policy=policy, chi=c or 0)
    assert abs(m * np.exp(lg) - v) <= 1e-12 * abs(v)
    scale = max(np.max(np.abs(g.data)) for g in g_o)
    for t, gg, go in zip(net.tensors, grads, g_o):
        assert gg.legs == t.legs or list(gg.legs) == list(t.legs)
        assert np.max(np.abs(dense(gg).data - go.data)) <= 1e-9 * scale


@pytest.mark.parametrize("mode", ["local", "global"])
@pytest.mark.parametrize("lx,ly,D,chi", [(2, 3, (2, 1), 4)])
def test_boundary_mps_gradient_against_oracle(F, ctx, lx, ly, D, chi, mode):
    """The boundary-MPS row sweep (one tensor per column, horizontal bonds
    capped at chi by late compression)."""
    net, tree = setup(lx, ly, D, 3, boundary=True)
    v_o, g_o, gap = NG.contract_tree_grad(net, tree, "late", chi, mode=mode)
    assert gap is not None and gap > 1e-3
    tensors = [F.Tensor.from_blocks(ctx, t.legs, t.parity, sorted(O.extract_blocks(t).items())) for t in net.tensors]
    pos = list(net.positions) if mode == "global" else None
    v, grads = F.contract_grad(ctx, tensors, net.bonds, tree, positions=pos, policy="late", chi=chi)
    assert abs(v - v_o) <= 1e-10 * abs(v_o)
    scale = max(np.max(np.abs(g.data)) for g in g_o)
    for gg, go in zip(grads, g_o):
        assert np.max(np.abs(dense(gg).data - go.data)) <= 1e-9 * scale


@pytest.mark.parametrize("mode", ["local", "global"])
def test_boundary_mps_gradient_finite_differences(F, ctx, mode):
    """3x3, D = 2 (1+1), chi = 3: some compressed blocks are square and rank
    deficient (their boundary tensor came out of an earlier truncation), where
    the oracle's QR rule, which inverts R, is off (its own finite-difference
    error here is ~2e-4); the GPU takes blocks of fewer than 5/4 K rows as
    their own factor and needs no inverse.  Its gradient against central
    differences of ftn_contract on 20 seeded entries (h = 1e-6)."""
    net, tree = setup(3, 3, (1, 1), 3, boundary=True)
    tensors = [F.Tensor.from_blocks(ctx, t.legs, t.parity, sorted(O.extract_blocks(t).items())) for t in net.tensors]
    pos = list(net.positions) if mode == "global" else None
    v, grads = F.contract_grad(ctx, tensors, net.bonds, tree, positions=pos, policy="late", chi=3)
    host = [dict(g.to_blocks()) for g in grads]
    scale = max(float(np.max(np.abs(b))) for d in host for b in d.values())
    rng = np.random.default_rng(0)
    worst, h = 0.0, 1e-6
    for _ in range(20):
        i = int(rng.integers(len(tensors)))
        tb = dict(tensors[i].to_blocks())
        key = sorted(tb)[int(rng.integers(len(tb)))]
        idx = tuple(int(rng.integers(d)) for d in tb[key].shape)
        vals = []
        for sg in (1.0, -1.0):
            pb = {k: b.copy() for k, b in tb.items()}
            pb[key][idx] += sg * h
            t = F.Tensor.from_blocks(ctx, tensors[i].legs, tensors[i].parity, sorted(pb.items()))
            m, lg = F.contract(ctx, tensors[:i] + [t] + tensors[i + 1:], net.bonds, tree, positions=pos,
                               policy="late", chi=3)
            vals.append(m * np.exp(lg))
        worst = max(worst, abs((vals[0] - vals[1]) / (2 * h) - float(host[i][key][idx])) / scale)
    assert worst < 1e-6, worst


@pytest.mark.parametrize("mode", ["local", "global"])
@pytest.mark.parametrize("case", ["exact", "late", "early", "boundary"])
def test_checkpointed_gradient_is_bit_identical(F, ctx, case, mode):
    """checkpoint = k keeps the walk's state every k steps and replays each
    segment in the backward: the value and every gradient entry equal those
    of the fully taped walk (checkpoint = 0) bit for bit, for segments of one
    step up to past the whole tree."""
    if case == "boundary":
        net, tree = setup(3, 3, (1, 1), 3, boundary=True)
        policy, chi = "late", 3
    else:
        net, tree = setup(2, 3, (1, 1), 3)
        policy, chi = case, (0 if case == "exact" else 2)
    tensors = [F.Tensor.from_blocks(ctx, t.legs, t.parity, sorted(O.extract_blocks(t).items())) for t in net.tensors]
    pos = list(net.positions) if mode == "global" else None
    v0, g0 = F.contract_grad(ctx, tensors, net.bonds, tree, positions=pos, policy=policy, chi=chi)
    ref = [g.download() for g in g0]
    steps = len(tree)
    for k in sorted({1, 2, 3, 5, steps - 1, steps, steps + 4}):
        v, gk = F.contract_grad(ctx, tensors, net.bonds, tree, positions=pos, policy=policy, chi=chi, checkpoint=k)
        assert v == v0, k
        for r, gg in zip(ref, gk):
            assert np.array_equal(r, gg.download()), k


def test_checkpoint_argument_checked(F, ctx):
    net, tree = setup(2, 2, (1, 1), 3)
    tensors = [F.Tensor.from_blocks(ctx, t.legs, t.parity, sorted(O.extract_blocks(t).items())) for t in net.tensors]
    with pytest.raises(F.FtnError) as e:
        F.contract_grad(ctx, tensors, net.bonds, tree, checkpoint=-1)
    assert e.value.status == -1
    v, grads = F.contract_grad(ctx, tensors, net.bonds, tree, checkpoint=1)  # the context is still usable
    assert np.isfinite(v) and len(grads) == len(tensors)


def test_network_grad_rejects_odd_tensors(F, ctx):
    la = [(1, 1, 0), (1, 1, 1)]
    a = F.Tensor.from_blocks(ctx, la, 1, W.random_blocks(la, 1, 1))
    b = F.Tensor.from_blocks(ctx, [(1, 1, 1), (1, 1, 0)], 1, W.random_blocks([(1, 1, 1), (1, 1, 0)], 1, 2))
    with pytest.raises(F.FtnError) as e:
        F.contract_grad(ctx, [a, b], [(0, 0, 1, 0), (0, 1, 1, 1)], [(0, 1)])
    assert e.value.status == -8
