"""The adjoints behind torch.autograd.Function: the compression
(compress_autograd: ftn_compress forward, ftn_compress_grad backward)
chained with the differentiable tensordot, against the oracle's compression
adjoint; and a network's value (network_value_autograd over
ftn_contract_grad) against contract_grad itself, with and without
checkpointing, and under a scaled loss."""
import numpy as np
import pytest

import oracle as O
import oracle.compress_adjoint as CA
import oracle.network_grad as NG
import workloads as W

pytestmark = pytest.mark.gpu

CASES = [
    ([(2, 1, 0), (2, 2, 1), (1, 2, 0), (3, 2, 1)], [(2, 2, 0), (2, 1, 1), (3, 2, 0)], [1, 3], [0, 2], 0, 0),
    ([(6, 5, 0), (4, 3, 1), (3, 2, 0)], [(3, 2, 1), (5, 4, 0), (3, 3, 1)], [2], [0], 0, 0),
    ([(1, 1, 1), (3, 3, 0), (2, 1, 1)], [(3, 3, 1), (2, 2, 0)], [1], [0], 1, 1),
]


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


def dense_flat(F, ctx, legs, parity, flat):
    t = F.Tensor.wrap(ctx, legs, parity, flat.detach().contiguous(), F.F64)
    return O.embed_blocks(t.legs, t.parity, t.to_blocks())


def flat_of(F, ctx, t):
    return F.Tensor.from_blocks(ctx, t.legs, t.parity, sorted(O.extract_blocks(t).items())).view().clone()


def pick_chi(x, y, ax, ay):
    _, _, info = O.compress(x, y, ax, ay, chi=10**6)
    sv = info["singular_values"]
    best = max(range(1, len(sv)), key=lambda c: (sv[c - 1] - sv[c]) / sv[0])
    assert (sv[best - 1] - sv[best]) / sv[0] > 1e-3
    return best


@pytest.mark.parametrize("case", range(len(CASES)))
def test_compress_autograd_against_oracle(F, ctx, case):
    """L = sum(G * op(X', Y')) through compress_autograd and
    tensordot_autograd; torch's backward gives dL/dX and dL/dY."""
    lx, ly, ax, ay, px, py = CASES[case]
    x = O.embed_blocks(lx, px, W.random_blocks(lx, px, 40 + case))
    y = O.embed_blocks(ly, py, W.random_blocks(ly, py, 50 + case))
    chi = pick_chi(x, y, ax, ay)
    c = O.contract(x, y, ax, ay)
    g = O.embed_blocks(c.legs, c.parity, W.random_blocks(c.legs, c.parity, 60 + case))
    xd = flat_of(F, ctx, x).requires_grad_(True)
    yd = flat_of(F, ctx, y).requires_grad_(True)
    x_before, y_before = xd.detach().clone(), yd.detach().clone()
    xn, lxn, pxn, yn, lyn, pyn = F.compress_autograd(ctx, xd, x.legs, px, yd, y.legs, py, ax, ay, chi)
    cd, lc, pc = F.tensordot_autograd(ctx, xn, lxn, pxn, yn, lyn, pyn, [len(lxn) - 1], [0])
    assert [tuple(l) for l in lc] == [tuple(l) for l in c.legs] and pc == c.parity
    loss = (flat_of(F, ctx, g) * cd).sum()
    loss.backward()
    xo, yo, _ = O.compress(x, y, ax, ay, chi)
    ox = O.contract_grad(xo, yo, [xo.rank - 1], [0], g, wrt="x")
    oy = O.contract_grad(xo, yo, [xo.rank - 1], [0], g, wrt="y")
    rx, ry = CA.compress_grad(x, y, ax, ay, chi, ox, oy)
    scale = max(np.max(np.abs(rx.data)), np.max(np.abs(ry.data)))
    ex = np.max(np.abs(dense_flat(F, ctx, x.legs, px, xd.grad).data - rx.data)) / scale
    ey = np.max(np.abs(dense_flat(F, ctx, y.legs, py, yd.grad).data - ry.data)) / scale
    assert max(ex, ey) <= 1e-9, (ex, ey)
    # the forward works on copies: the leaves are unchanged
    assert bool((xd.detach() == x_before).all()) and bool((yd.detach() == y_before).all())


def network(lx, ly, D, seed):
    n, edges = W.square_lattice(lx, ly)
    lay = W.peps_layout(n, edges, D, (2, 2))
    net = O.norm_network(lay, O.ket_tensors(lay, W.random_peps(lay, seed)))
    return net, W.double_layer_tree(n, W.site_sweep_tree(list(range(n))))


@pytest.mark.parametrize("checkpoint", [0, 2])
def test_network_value_autograd(F, ctx, checkpoint):
    """value and leaf gradients equal contract_grad's bit for bit (the
    forward runs it), a scaled loss scales them exactly, and the value matches
    the oracle's."""
    net, tree = network(2, 3, (1, 1), 3)
    datas = [flat_of(F, ctx, t).requires_grad_(True) for t in net.tensors]
    legs = [t.legs for t in net.tensors]
    pars = [t.parity for t in net.tensors]
    v = F.network_value_autograd(ctx, datas, legs, pars, net.bonds, tree, policy="late", chi=2,
                                 checkpoint=checkpoint)
    (3.0 * v).backward()
    tensors = [F.Tensor.from_blocks(ctx, t.legs, t.parity, sorted(O.extract_blocks(t).items())) for t in net.tensors]
    v_ref, g_ref = F.contract_grad(ctx, tensors, net.bonds, tree, policy="late", chi=2)
    assert float(v.detach()) == v_ref
    for d, gr in zip(datas, g_ref):
        assert np.array_equal(d.grad.cpu().numpy(), 3.0 * gr.download())
    v_o, _, _ = NG.contract_tree_grad(net, tree, "late", 2, mode="local")
    assert abs(float(v.detach()) - v_o) <= 1e-10 * abs(v_o)
