"""Pins of the oracle's contraction gradient (brute force over unit tensors)
against facts that do not come from it: the bosonic reduction to an einsum
closed form, the adjoint identity <dX, X> = <G, C> = <dY, Y> of a bilinear
form, and a planted mistake (dropping the fermionic signs) that must fail."""
import string

import numpy as np
import pytest

import oracle as O
import workloads as W


def graded(legs, parity, seed):
    return O.embed_blocks(legs, parity, W.random_blocks(legs, parity, seed))


def einsum_grad_bosonic(x, y, ax, ay, g, out_perm, wrt):
    """Closed form for d1 = 0 on every leg: C[xf..., yf...] = sum_k X Y, so
    dX = einsum(G, Y) and dY = einsum(X, G) with the contracted letters shared."""
    letters = iter(string.ascii_letters)
    lx = [next(letters) for _ in range(x.rank)]
    ly = [None] * y.rank
    for a, b in zip(ax, ay):
        ly[b] = lx[a]
    for k in range(y.rank):
        if ly[k] is None:
            ly[k] = next(letters)
    lc = [lx[k] for k in range(x.rank) if k not in ax] + [ly[k] for k in range(y.rank) if k not in ay]
    if out_perm is not None:
        lc = [lc[p] for p in out_perm]
    if wrt == "x":
        return np.einsum(f"{''.join(lc)},{''.join(ly)}->{''.join(lx)}", g.data, y.data)
    return np.einsum(f"{''.join(lx)},{''.join(lc)}->{''.join(ly)}", x.data, g.data)


CASES = [
    # X legs, Y legs, ax, ay, out_perm
    ([(2, 1, 0), (2, 1, 1), (1, 2, 0)], [(2, 1, 0), (2, 2, 1)], [1], [0], None),
    ([(1, 2, 1), (2, 1, 0), (2, 2, 1)], [(2, 2, 0), (1, 2, 0), (1, 1, 1)], [0, 2], [1, 0], [1, 0]),
    ([(2, 1, 0), (1, 1, 1), (2, 1, 0), (1, 2, 1)], [(1, 2, 0), (1, 1, 0), (2, 1, 1)], [3, 1], [0, 1], [2, 0, 1]),
]


@pytest.mark.parametrize("ci", range(len(CASES)))
@pytest.mark.parametrize("wrt", ["x", "y"])
def test_bosonic_reduction_matches_einsum(ci, wrt):
    lx, ly, ax, ay, perm = CASES[ci]
    lx = [(d0 + d1, 0, du) for d0, d1, du in lx]
    ly = [(d0 + d1, 0, du) for d0, d1, du in ly]
    x, y = graded(lx, 0, 1 + ci), graded(ly, 0, 11 + ci)
    c = O.contract_forward(x, y, ax, ay, out_perm=perm)
    g = O.GTensor(W.rng(21 + ci).standard_normal(c.data.shape), c.legs, c.parity)
    got = O.contract_grad(x, y, ax, ay, g, wrt=wrt, out_perm=perm)
    ref = einsum_grad_bosonic(x, y, ax, ay, g, perm, wrt)
    assert np.allclose(got.data, ref, rtol=0, atol=1e-12)


@pytest.mark.parametrize("ci", range(len(CASES)))
@pytest.mark.parametrize("px,py", [(0, 0), (1, 0), (0, 1), (1, 1)])
def test_adjoint_identity(ci, px, py):
    lx, ly, ax, ay, perm = CASES[ci]
    x, y = graded(lx, px, 3 + ci), graded(ly, py, 13 + ci)
    c = O.contract_forward(x, y, ax, ay, out_perm=perm)
    g = O.embed_blocks(c.legs, c.parity, W.random_blocks(c.legs, c.parity, 23 + ci))
    dx = O.contract_grad(x, y, ax, ay, g, wrt="x", out_perm=perm)
    dy = O.contract_grad(x, y, ax, ay, g, wrt="y", out_perm=perm)
    form = float(np.sum(g.data * c.data))
    assert abs(float(np.sum(dx.data * x.data)) - form) <= 1e-12 * abs(form)
    assert abs(float(np.sum(dy.data * y.data)) - form) <= 1e-12 * abs(form)


def test_planted_sign_mistake_is_detected():
    """The sign-less einsum gradient differs from the fermionic one as soon
    as odd sectors are present: the pins above would catch a dropped sign."""
    lx, ly, ax, ay, perm = CASES[1]
    x, y = graded(lx, 1, 5), graded(ly, 0, 15)
    c = O.contract_forward(x, y, ax, ay, out_perm=perm)
    g = O.embed_blocks(c.legs, c.parity, W.random_blocks(c.legs, c.parity, 25))
    got = O.contract_grad(x, y, ax, ay, g, wrt="x", out_perm=perm)
    wrong = einsum_grad_bosonic(x, y, ax, ay, g, perm, "x")
    assert np.max(np.abs(got.data - wrong)) > 1e-3
