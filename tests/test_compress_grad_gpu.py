"""The adjoint of the GPU compression (ftn_compress_grad) against the
oracle's (oracle.compress_adjoint, pinned by finite differences of the
forward oracle in tests/test_oracle_compress_adjoint.py).

Each case compresses X and Y with a truncation at the largest relative gap of
the pooled spectrum and takes the gradient of a loss that does not depend on
the gauge of the new bond -- sum(G * op(X', Y')) or row-weighted squared norms
of X' and Y' -- with the cotangents formed from each implementation's own
(X', Y').  Cases: blocks with fewer rows than bond states (the side is its own
factor on the GPU; the wide QR rule in the oracle), tall blocks (factored by
Gram and Cholesky), one and two bond legs, odd tensors.  Also: the inputs
are left unchanged, a cotangent of the wrong shape is rejected, and a bond
state that no entry of X reaches (a rank-deficient sector: no gradient
there) is reported as unsupported.
"""
import numpy as np
import pytest

import oracle as O
import oracle.compress_adjoint as CA
import workloads as W

pytestmark = pytest.mark.gpu

CASES = [
    ([(2, 1, 0), (2, 2, 1), (1, 2, 0), (3, 2, 1)], [(2, 2, 0), (2, 1, 1), (3, 2, 0)], [1, 3], [0, 2], 0, 0),
    ([(3, 2, 1), (2, 2, 0), (2, 1, 1)], [(1, 2, 0), (2, 2, 1), (2, 1, 0)], [1], [1], 1, 0),
    ([(1, 1, 1), (3, 3, 0), (2, 1, 1)], [(3, 3, 1), (2, 2, 0)], [1], [0], 1, 1),
    ([(6, 5, 0), (4, 3, 1), (3, 2, 0)], [(3, 2, 1), (5, 4, 0), (3, 3, 1)], [2], [0], 0, 0),
    ([(7, 6, 0), (3, 2, 1), (4, 3, 0), (2, 2, 1)], [(4, 3, 1), (2, 2, 0), (5, 4, 1), (3, 3, 0)], [2, 3], [0, 1], 0, 1),
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


def dense(t):
    return O.embed_blocks(t.legs, t.parity, t.to_blocks())


def pick_chi(x, y, ax, ay):
    _, _, info = O.compress(x, y, ax, ay, chi=10**6)
    sv = info["singular_values"]
    best = max(range(1, len(sv)), key=lambda c: (sv[c - 1] - sv[c]) / sv[0])
    assert (sv[best - 1] - sv[best]) / sv[0] > 1e-3
    return best


def cotangents(kind, x, y, ax, ay, xn, yn, seed):
    rng = np.random.default_rng(seed)
    if kind == "bilinear":
        c = O.contract(x, y, ax, ay)
        g = O.embed_blocks(c.legs, c.parity, W.random_blocks(c.legs, c.parity, seed))
        return (O.contract_grad(xn, yn, [xn.rank - 1], [0], g, wrt="x"),
                O.contract_grad(xn, yn, [xn.rank - 1], [0], g, wrt="y"))
    xm = xn.data.reshape(-1, xn.data.shape[-1])
    ym = yn.data.reshape(yn.data.shape[0], -1)
    w = rng.uniform(0.5, 1.5, xm.shape[0])
    v = rng.uniform(0.5, 1.5, ym.shape[1])
    return (O.GTensor((2.0 * w[:, None] * xm).reshape(xn.data.shape), xn.legs, xn.parity),
            O.GTensor((2.0 * v[None, :] * ym).reshape(yn.data.shape), yn.legs, yn.parity))


def upload(F, ctx, t):
    return F.Tensor.from_blocks(ctx, t.legs, t.parity, sorted(O.extract_blocks(t).items()))


@pytest.mark.parametrize("case", range(len(CASES)))
@pytest.mark.parametrize("kind", ["bilinear", "norms"])
def test_compress_grad_against_oracle(F, ctx, case, kind):
    lx, ly, ax, ay, px, py = CASES[case]
    x = O.embed_blocks(lx, px, W.random_blocks(lx, px, 6 + case))
    y = O.embed_blocks(ly, py, W.random_blocks(ly, py, 16 + case))
    chi = pick_chi(x, y, ax, ay)
    xg, yg = upload(F, ctx, x), upload(F, ctx, y)
    xn_t, yn_t, _ = F.compress(ctx, upload(F, ctx, x), upload(F, ctx, y), ax, ay, chi)
    xn, yn = dense(xn_t), dense(yn_t)
    gx, gy = cotangents(kind, x, y, ax, ay, xn, yn, 30 + case)
    dx, dy = F.compress_grad(ctx, xg, yg, ax, ay, chi, upload(F, ctx, gx), upload(F, ctx, gy))
    xo, yo, _ = O.compress(x, y, ax, ay, chi)
    ox, oy = cotangents(kind, x, y, ax, ay, xo, yo, 30 + case)
    rx, ry = CA.compress_grad(x, y, ax, ay, chi, ox, oy)
    scale = max(np.max(np.abs(rx.data)), np.max(np.abs(ry.data)))
    assert dx.legs == list(x.legs) or dx.legs == x.legs
    ex = np.max(np.abs(dense(dx).data - rx.data)) / scale
    ey = np.max(np.abs(dense(dy).data - ry.data)) / scale
    assert max(ex, ey) <= 1e-9, (ex, ey)
    # the inputs are borrowed and left as they were
    assert np.array_equal(dense(xg).data, x.data) and np.array_equal(dense(yg).data, y.data)


def test_compress_grad_errors(F, ctx):
    lx, ly, ax, ay, px, py = CASES[3]
    x = O.embed_blocks(lx, px, W.random_blocks(lx, px, 3))
    y = O.embed_blocks(ly, py, W.random_blocks(ly, py, 4))
    chi = pick_chi(x, y, ax, ay)
    xn_t, yn_t, _ = F.compress(ctx, upload(F, ctx, x), upload(F, ctx, y), ax, ay, chi)
    # a cotangent with X's legs instead of X''s
    with pytest.raises(F.FtnError) as e:
        F.compress_grad(ctx, upload(F, ctx, x), upload(F, ctx, y), ax, ay, chi, upload(F, ctx, x),
                        upload(F, ctx, dense(yn_t)))
    assert e.value.status == -2
    # a bond state of X that no entry reaches: the even sector's factor loses
    # a row (rank deficient: the gradient is not defined there)
    bx = {kk: v.copy() for kk, v in W.random_blocks(lx, px, 3)}
    for kk, v in bx.items():
        if kk[-1] == 0:
            v[..., 0] = 0.0
    xz_t = F.Tensor.from_blocks(ctx, lx, px, sorted(bx.items()))
    xnz, ynz, _ = F.compress(ctx, F.Tensor.from_blocks(ctx, lx, px, sorted(bx.items())), upload(F, ctx, y), ax, ay,
                             10**6)
    with pytest.raises(F.FtnError) as e:
        F.compress_grad(ctx, xz_t, upload(F, ctx, y), ax, ay, 10**6, upload(F, ctx, dense(xnz)),
                        upload(F, ctx, dense(ynz)))
    assert e.value.status == -8
    # the context is still usable
    dx, dy = F.compress_grad(ctx, upload(F, ctx, x), upload(F, ctx, y), ax, ay, chi, upload(F, ctx, dense(xn_t)),
                             upload(F, ctx, dense(yn_t)))
    assert np.isfinite(dense(dx).data).all() and np.isfinite(dense(dy).data).all()
