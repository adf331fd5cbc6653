"""Pins of the oracle's sector QR/SVD compression and approximate contraction.

* chi >= rank reproduces the exact product (Sec. II.A decomposition is exact);
* Eckart-Young: the Frobenius error equals sqrt(sum of discarded s^2);
* the pooled singular values equal numpy.linalg.svd of each dense sector
  block of the bond product;
* approximate contraction converges to the exact value as chi grows.
"""
import numpy as np
import pytest

import oracle as O
import workloads as W


def rand_t(legs, parity, seed):
    return O.embed_blocks(legs, parity, W.random_blocks(legs, parity, seed))


CASES = [
    # X legs, Y legs, ax, ay, px, py
    ([(2, 1, 0), (2, 2, 1), (1, 2, 0), (3, 2, 1)], [(2, 2, 0), (2, 1, 1), (3, 2, 0)], [1, 3], [0, 2], 0, 0),
    ([(3, 2, 1), (2, 2, 0), (2, 1, 1)], [(1, 2, 0), (2, 2, 1), (2, 1, 0)], [1], [1], 1, 0),
    ([(2, 2, 1), (3, 3, 0), (2, 1, 1), (1, 1, 0)], [(3, 3, 1), (1, 1, 1), (2, 2, 0)], [1, 3], [0, 1], 1, 1),
]


@pytest.mark.parametrize("case", CASES)
def test_full_rank_is_exact(case):
    lx, ly, ax, ay, px, py = case
    x, y = rand_t(lx, px, 1), rand_t(ly, py, 2)
    ref = O.contract(x, y, ax, ay)
    xn, yn, info = O.compress(x, y, ax, ay, chi=10**6)
    got = O.contract(xn, yn, [xn.rank - 1], [0])
    assert xn.check_symmetry() and yn.check_symmetry()
    assert np.allclose(got.data, ref.data, rtol=1e-12, atol=1e-12 * np.max(np.abs(ref.data)))


@pytest.mark.parametrize("case", CASES)
@pytest.mark.parametrize("chi", [1, 2, 3, 5])
def test_eckart_young(case, chi):
    lx, ly, ax, ay, px, py = case
    x, y = rand_t(lx, px, 3), rand_t(ly, py, 4)
    ref = O.contract(x, y, ax, ay)
    xn, yn, info = O.compress(x, y, ax, ay, chi=chi)
    assert sum(info["kept"]) == min(chi, len(info["singular_values"]))
    got = O.contract(xn, yn, [xn.rank - 1], [0])
    err = np.linalg.norm(got.data - ref.data)
    assert abs(err - np.sqrt(info["discarded_sq"])) <= 1e-10 * np.linalg.norm(ref.data)


@pytest.mark.parametrize("case", CASES)
def test_sector_singular_values(case):
    """Singular values of each parity sector equal those of the dense sector
    block of the matricised product op(X, Y)."""
    lx, ly, ax, ay, px, py = case
    x, y = rand_t(lx, px, 5), rand_t(ly, py, 6)
    ref = O.contract(x, y, ax, ay)
    nfx = x.rank - len(ax)
    rows = int(np.prod(ref.data.shape[:nfx]))
    m = ref.data.reshape(rows, -1)
    from oracle.compress import _multi_parity

    rpar = _multi_parity(ref.legs[:nfx])
    cpar = _multi_parity(ref.legs[nfx:])
    _, _, info = O.compress(x, y, ax, ay, chi=10**6)
    for pi in (0, 1):
        blk = m[np.ix_(rpar == (px ^ pi), cpar == (py ^ pi))]
        want = np.linalg.svd(blk, compute_uv=False) if blk.size else np.zeros(0)
        got = info["sector_sv"][pi]
        got = np.zeros(0) if got is None else got
        k = min(len(want), len(got))
        assert np.allclose(np.sort(got)[::-1][:k], want[:k], rtol=1e-12, atol=1e-12 * want.max(initial=1))
        # beyond the rank of the block the core has only zeros
        assert np.all(np.abs(np.sort(got)[::-1][k:]) <= 1e-10 * max(want.max(initial=1), 1))


@pytest.mark.parametrize("lx,ly", [(2, 3), (3, 3)])
def test_approximate_contraction_converges(lx, ly):
    n, edges = W.square_lattice(lx, ly)
    lay = W.peps_layout(n, edges, (1, 1), (2, 2))
    kets = O.ket_tensors(lay, W.random_peps(lay, 1))
    net = O.norm_network(lay, kets)
    st = W.site_sweep_tree(list(range(n)))
    tree = W.double_layer_tree(n, st)
    ex, exl, _ = O.contract_tree(net, tree, normalize=True)
    exact = float(ex.data) * np.exp(exl)
    errs = []
    for chi in (2, 4, 8, 16, 64):
        for policy in ("late", "early"):
            r, lg, _ = O.contract_tree(net, tree, policy=policy, chi=chi, normalize=True)
            errs.append((chi, policy, abs(float(r.data) * np.exp(lg) - exact) / abs(exact)))
    assert all(e <= 1e-10 for c, p, e in errs if c == 64)
    assert any(e > 1e-8 for c, p, e in errs if c == 2)
    for mode in ("global",):
        r, lg, _ = O.contract_tree(net, tree, mode=mode, policy="late", chi=64, normalize=True)
        assert abs(float(r.data) * np.exp(lg) - exact) <= 1e-10 * abs(exact)
    # approximate: global and local agree at a truncating chi as well
    a, al, _ = O.contract_tree(net, tree, mode="local", policy="late", chi=4, normalize=True)
    b, bl, _ = O.contract_tree(net, tree, mode="global", policy="late", chi=4, normalize=True)
    assert abs(float(a.data) * np.exp(al) - float(b.data) * np.exp(bl)) <= 1e-9 * abs(float(a.data) * np.exp(al))
