"""Pins of the oracle's adjoint of the sector QR/SVD compression
(oracle.compress_adjoint), with nothing but the forward oracle and the
contraction adjoint as references:

* without truncation op(X', Y') = op(X, Y) exactly, so the gradient of
  L = sum(G * op(X', Y')) through the compression equals the gradient of the
  plain contraction (oracle.adjoint, pinned by its definition);
* with truncation (a gap at the cut) the gradients of two losses that do not
  depend on the gauge of the new bond -- the contraction above and
  row-weighted squared norms of X' and Y' -- equal central finite differences
  of the forward oracle, entry by entry;
* planted mistakes in the backward rules (a dropped projection term of the SVD
  rule, the QR rule without its symmetrisation) fail the finite differences.
"""
import numpy as np
import pytest

import oracle as O
import oracle.compress_adjoint as CA
import workloads as W


def rand_t(legs, parity, seed):
    return O.embed_blocks(legs, parity, W.random_blocks(legs, parity, seed))


CASES = [
    # X legs, Y legs, ax, ay, px, py; the first X block of the second parity
    # sector has fewer rows than bond states (the wide QR branch)
    ([(2, 1, 0), (2, 2, 1), (1, 2, 0), (3, 2, 1)], [(2, 2, 0), (2, 1, 1), (3, 2, 0)], [1, 3], [0, 2], 0, 0),
    ([(3, 2, 1), (2, 2, 0), (2, 1, 1)], [(1, 2, 0), (2, 2, 1), (2, 1, 0)], [1], [1], 1, 0),
    ([(1, 1, 1), (3, 3, 0), (2, 1, 1)], [(3, 3, 1), (2, 2, 0)], [1], [0], 1, 1),
]


def pick_chi(x, y, ax, ay):
    """A truncation that keeps some and drops some singular values, at the
    largest relative gap."""
    _, _, info = O.compress(x, y, ax, ay, chi=10**6)
    sv = info["singular_values"]
    best = max(range(1, len(sv)), key=lambda c: (sv[c - 1] - sv[c]) / sv[0])
    assert (sv[best - 1] - sv[best]) / sv[0] > 1e-3
    return best


def bilinear_loss(x, y, ax, ay, chi, g):
    xn, yn, _ = O.compress(x, y, ax, ay, chi)
    return float(np.sum(g.data * O.contract(xn, yn, [xn.rank - 1], [0]).data)), xn, yn


def bilinear_cotangents(xn, yn, g):
    gx = O.contract_grad(xn, yn, [xn.rank - 1], [0], g, wrt="x")
    gy = O.contract_grad(xn, yn, [xn.rank - 1], [0], g, wrt="y")
    return gx, gy


def norm_loss(x, y, ax, ay, chi, w, v):
    xn, yn, _ = O.compress(x, y, ax, ay, chi)
    xm = xn.data.reshape(-1, xn.data.shape[-1])
    ym = yn.data.reshape(yn.data.shape[0], -1)
    return float(np.sum(w[:, None] * xm**2) + np.sum(v[None, :] * ym**2)), xn, yn


def norm_cotangents(xn, yn, w, v):
    xm = xn.data.reshape(-1, xn.data.shape[-1])
    ym = yn.data.reshape(yn.data.shape[0], -1)
    gx = O.GTensor((2.0 * w[:, None] * xm).reshape(xn.data.shape), xn.legs, xn.parity)
    gy = O.GTensor((2.0 * v[None, :] * ym).reshape(yn.data.shape), yn.legs, yn.parity)
    return gx, gy


def finite_differences(loss, x, y, h=1e-6):
    out = []
    for t, which in ((x, 0), (y, 1)):
        d = np.zeros(t.data.shape)
        for idx in CA._allowed(t):
            vals = []
            for sgn in (1.0, -1.0):
                e = t.data.copy()
                e[idx] += sgn * h
                tt = O.GTensor(e, t.legs, t.parity)
                vals.append(loss(tt, y) if which == 0 else loss(x, tt))
            d[idx] = (vals[0] - vals[1]) / (2 * h)
        out.append(d)
    return out


def result_cotangent(x, y, ax, ay, seed):
    c = O.contract(x, y, ax, ay)
    return O.embed_blocks(c.legs, c.parity, W.random_blocks(c.legs, c.parity, seed))


@pytest.mark.parametrize("case", CASES)
def test_factors_match_the_forward_oracle(case):
    lx, ly, ax, ay, px, py = case
    x, y = rand_t(lx, px, 1), rand_t(ly, py, 2)
    chi = pick_chi(x, y, ax, ay)
    _, _, info = O.compress(x, y, ax, ay, chi)
    _, _, sec, k = CA.compress_factors(x, y, ax, ay, chi)
    assert k == info["kept"]
    for pi in (0, 1):
        ref = info["sector_sv"][pi]
        got = None if sec[pi][3] is None else sec[pi][3][5]
        assert (ref is None and got is None) or np.array_equal(ref, got)


@pytest.mark.parametrize("case", CASES)
def test_without_truncation_equals_the_contraction_gradient(case):
    lx, ly, ax, ay, px, py = case
    x, y = rand_t(lx, px, 3), rand_t(ly, py, 4)
    g = result_cotangent(x, y, ax, ay, 5)
    xn, yn, _ = O.compress(x, y, ax, ay, chi=10**6)
    gx, gy = bilinear_cotangents(xn, yn, g)
    dx, dy = CA.compress_grad(x, y, ax, ay, 10**6, gx, gy)
    rx = O.contract_grad(x, y, ax, ay, g, wrt="x")
    ry = O.contract_grad(x, y, ax, ay, g, wrt="y")
    scale = max(np.max(np.abs(rx.data)), np.max(np.abs(ry.data)))
    assert np.max(np.abs(dx.data - rx.data)) <= 1e-10 * scale
    assert np.max(np.abs(dy.data - ry.data)) <= 1e-10 * scale


def check_against_fd(x, y, ax, ay, chi, kind, seed):
    rng = np.random.default_rng(seed)
    if kind == "bilinear":
        g = result_cotangent(x, y, ax, ay, seed)
        _, xn, yn = bilinear_loss(x, y, ax, ay, chi, g)
        gx, gy = bilinear_cotangents(xn, yn, g)
        loss = lambda a, b: bilinear_loss(a, b, ax, ay, chi, g)[0]  # noqa: E731
    else:
        xn, yn, _ = O.compress(x, y, ax, ay, chi)
        w = rng.uniform(0.5, 1.5, int(np.prod(xn.data.shape[:-1])))
        v = rng.uniform(0.5, 1.5, int(np.prod(yn.data.shape[1:])))
        gx, gy = norm_cotangents(xn, yn, w, v)
        loss = lambda a, b: norm_loss(a, b, ax, ay, chi, w, v)[0]  # noqa: E731
    dx, dy = CA.compress_grad(x, y, ax, ay, chi, gx, gy)
    fx, fy = finite_differences(loss, x, y)
    scale = max(np.max(np.abs(fx)), np.max(np.abs(fy)))
    return max(np.max(np.abs(dx.data - fx)), np.max(np.abs(dy.data - fy))) / scale


@pytest.mark.parametrize("case", CASES)
@pytest.mark.parametrize("kind", ["bilinear", "norms"])
def test_truncated_gradient_matches_finite_differences(case, kind):
    lx, ly, ax, ay, px, py = case
    x, y = rand_t(lx, px, 6), rand_t(ly, py, 7)
    chi = pick_chi(x, y, ax, ay)
    assert check_against_fd(x, y, ax, ay, chi, kind, 8) < 1e-6


def test_planted_mistakes_fail_the_finite_differences(monkeypatch):
    lx, ly, ax, ay, px, py = CASES[0]
    x, y = rand_t(lx, px, 6), rand_t(ly, py, 7)
    chi = pick_chi(x, y, ax, ay)
    assert check_against_fd(x, y, ax, ay, chi, "norms", 8) < 1e-6
    good_svd = CA._svd_backward

    def svd_without_projections(u, s, v, du, ds, dv, keep):
        # the SVD rule without its (I - U U^T) and (I - V V^T) terms
        full = good_svd(u, s, v, du, ds, dv, keep)
        sinv = np.zeros(len(s))
        sinv[:keep] = 1.0 / s[:keep]
        full = full - (np.eye(u.shape[0]) - u @ u.T) @ du @ np.diag(sinv) @ v.T
        return full - u @ np.diag(sinv) @ dv.T @ (np.eye(v.shape[0]) - v @ v.T)

    monkeypatch.setattr(CA, "_svd_backward", svd_without_projections)
    assert check_against_fd(x, y, ax, ay, chi, "norms", 8) > 1e-3
    monkeypatch.setattr(CA, "_svd_backward", good_svd)
    monkeypatch.setattr(CA, "_copyltu", lambda b: np.tril(b))  # QR rule without the symmetrisation
    assert check_against_fd(x, y, ax, ay, chi, "norms", 8) > 1e-3
