"""Parity of ftn_compress (GPU, FP64) with the oracle's sector QR/SVD
compression.  Compared: the gauge-invariant product op(X', Y'), the kept
sector dimensions and the discarded weight (tolerance 1e-10 relative)."""
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


def dense(t):
    return O.embed_blocks(t.legs, t.parity, t.to_blocks())


CASES = [
    # X legs, Y legs, ax, ay, px, py
    ([(2, 1, 0), (2, 2, 1), (1, 2, 0), (3, 2, 1)], [(2, 2, 0), (2, 1, 1), (3, 2, 0)], [1, 3], [0, 2], 0, 0),
    ([(3, 2, 1), (2, 2, 0), (2, 1, 1)], [(1, 2, 0), (2, 2, 1), (2, 1, 0)], [1], [1], 1, 0),
    ([(2, 2, 1), (3, 3, 0), (2, 1, 1), (1, 1, 0)], [(3, 3, 1), (1, 1, 1), (2, 2, 0)], [1, 3], [0, 1], 1, 1),
    # tall on both sides, bond of 2 legs (16 + 16 states)
    ([(8, 8, 0), (4, 4, 1), (4, 4, 0), (6, 5, 1)], [(4, 4, 0), (8, 8, 0), (6, 5, 0), (3, 3, 1)], [1, 3], [0, 2], 0, 0),
    # bond wider than one side
    ([(1, 1, 0), (8, 8, 1)], [(8, 8, 0), (5, 7, 1), (4, 4, 0)], [1], [0], 0, 1),
]


def run(F, ctx, case, chi, arrows=True, seed=0):
    lx, ly, ax, ay, px, py = case
    bx, by = W.random_blocks(lx, px, 11 + seed), W.random_blocks(ly, py, 12 + seed)
    X, Y = O.embed_blocks(lx, px, bx), O.embed_blocks(ly, py, by)
    xr, yr, info_r = O.compress(X, Y, ax, ay, chi, arrows=arrows)
    ref = O.contract(xr, yr, [xr.rank - 1], [0])
    x = F.Tensor.from_blocks(ctx, lx, px, bx)
    y = F.Tensor.from_blocks(ctx, ly, py, by)
    xg, yg, info = F.compress(ctx, x, y, ax, ay, chi, arrows=arrows)
    got = O.contract(dense(xg), dense(yg), [xg.rank - 1], [0])
    return ref, got, info_r, info, xg, yg


@pytest.mark.parametrize("ci", range(len(CASES)))
@pytest.mark.parametrize("chi", [1, 3, 7, 10**6])
def test_compress_matches_oracle(F, ctx, ci, chi):
    ref, got, info_r, info, xg, yg = run(F, ctx, CASES[ci], chi)
    assert got.legs == ref.legs
    scale = max(np.max(np.abs(ref.data)), 1e-300)
    assert np.max(np.abs(got.data - ref.data)) <= 1e-10 * scale
    assert tuple(info.kept) == tuple(info_r["kept"])
    assert abs(info.discarded_sq - info_r["discarded_sq"]) <= 1e-10 * max(info.total_sq, 1e-300)
    sv = info_r["singular_values"]
    assert abs(info.s_max - sv[0]) <= 1e-12 * sv[0]
    # the new leg: incoming on X', outgoing on Y', dims = kept
    assert xg.legs[-1] == (info.kept[0], info.kept[1], 1)
    assert yg.legs[0] == (info.kept[0], info.kept[1], 0)


@pytest.mark.parametrize("ci", [0, 2])
def test_compress_without_arrow_parity(F, ctx, ci):
    ref, got, info_r, info, _, _ = run(F, ctx, CASES[ci], 4, arrows=False, seed=3)
    assert np.max(np.abs(got.data - ref.data)) <= 1e-10 * np.max(np.abs(ref.data))


def test_compress_full_rank_reproduces_product(F, ctx):
    """chi at or above the rank: op(X', Y') equals op(X, Y) itself."""
    lx, ly, ax, ay, px, py = CASES[3]
    bx, by = W.random_blocks(lx, px, 5), W.random_blocks(ly, py, 6)
    exact = O.contract(O.embed_blocks(lx, px, bx), O.embed_blocks(ly, py, by), ax, ay)
    x = F.Tensor.from_blocks(ctx, lx, px, bx)
    y = F.Tensor.from_blocks(ctx, ly, py, by)
    xg, yg, info = F.compress(ctx, x, y, ax, ay, 10**6)
    got = O.contract(dense(xg), dense(yg), [xg.rank - 1], [0])
    assert np.max(np.abs(got.data - exact.data)) <= 1e-10 * np.max(np.abs(exact.data))
    assert info.discarded_sq <= 1e-20 * info.total_sq


def test_compress_rank_deficient(F, ctx):
    """X of low rank across the bond: numerically zero singular values are
    never kept and the product stays exact."""
    g = W.rng(9)
    lx = [(6, 6, 0), (5, 5, 1)]
    # X = A B with an inner dimension of 2 per sector -> rank <= 4
    bx = []
    for bits in W.block_bits(lx, 0):
        shp = W.block_shape(lx, bits)
        bx.append((bits, g.standard_normal((shp[0], 2)) @ g.standard_normal((2, shp[1]))))
    ly = [(5, 5, 0), (4, 3, 1)]
    by = W.random_blocks(ly, 0, 4)
    exact = O.contract(O.embed_blocks(lx, 0, bx), O.embed_blocks(ly, 0, by), [1], [0])
    x = F.Tensor.from_blocks(ctx, lx, 0, bx)
    y = F.Tensor.from_blocks(ctx, ly, 0, by)
    xg, yg, info = F.compress(ctx, x, y, [1], [0], 10**6)
    assert sum(info.kept) <= 4
    got = O.contract(dense(xg), dense(yg), [xg.rank - 1], [0])
    assert np.max(np.abs(got.data - exact.data)) <= 1e-10 * np.max(np.abs(exact.data))


def _low_rank_blocks(g, legs, parity, inner, noise=0.0):
    out = []
    for bits in W.block_bits(legs, parity):
        shp = W.block_shape(legs, bits)
        blk = g.standard_normal((shp[0], inner)) @ g.standard_normal((inner, shp[1]))
        if noise:
            blk = blk + noise * g.standard_normal(shp)
        out.append((bits, blk))
    return out


def test_compress_zero_bond_columns(F, ctx):
    """Bond states that X never reaches: the Gram matrix has zero rows and
    columns, the R factor exact zero rows; the core is formed from the
    nonzero rows only and the result matches the oracle."""
    g = W.rng(21)
    lx = [(40, 36, 0), (24, 20, 1)]
    bx = []
    for bits in W.block_bits(lx, 0):
        blk = g.standard_normal(W.block_shape(lx, bits))
        blk[:, ::3] = 0.0  # every third bond state unused
        bx.append((bits, blk))
    ly = [(24, 20, 0), (30, 31, 1)]
    by = W.random_blocks(ly, 0, 22)
    X, Y = O.embed_blocks(lx, 0, bx), O.embed_blocks(ly, 0, by)
    for chi in (5, 10**6):
        xr, yr, info_r = O.compress(X, Y, [1], [0], chi)
        ref = O.contract(xr, yr, [1], [0])
        xg, yg, info = F.compress(ctx, F.Tensor.from_blocks(ctx, lx, 0, bx), F.Tensor.from_blocks(ctx, ly, 0, by),
                                  [1], [0], chi)
        got = O.contract(dense(xg), dense(yg), [1], [0])
        assert np.max(np.abs(got.data - ref.data)) <= 1e-10 * np.max(np.abs(ref.data))
        if chi == 5:
            assert tuple(info.kept) == tuple(info_r["kept"])
        else:
            assert sum(info.kept) == 16 + 13  # the numerical rank: nonzero bond states per sector


@pytest.mark.parametrize("noise", [0.0, 1e-15])
def test_compress_rounding_level_rank_deficiency(F, ctx, noise):
    """A bond of 64 + 64 states carried by rank-6 sectors (plus optional
    rounding-level noise): rows of the core at the rounding level are
    numerically zero for the Jacobi; the kept part and the product match."""
    g = W.rng(31)
    lx = [(150, 140, 0), (64, 64, 1)]
    ly = [(64, 64, 0), (70, 90, 1)]
    bx = _low_rank_blocks(g, lx, 0, 6, noise)
    by = W.random_blocks(ly, 0, 32)
    X, Y = O.embed_blocks(lx, 0, bx), O.embed_blocks(ly, 0, by)
    exact = O.contract(X, Y, [1], [0])
    for chi in (8, 10**6):
        xr, yr, info_r = O.compress(X, Y, [1], [0], chi)
        ref = O.contract(xr, yr, [1], [0])
        xg, yg, info = F.compress(ctx, F.Tensor.from_blocks(ctx, lx, 0, bx), F.Tensor.from_blocks(ctx, ly, 0, by),
                                  [1], [0], chi)
        got = O.contract(dense(xg), dense(yg), [1], [0])
        assert np.max(np.abs(got.data - ref.data)) <= 1e-10 * np.max(np.abs(ref.data))
        assert info.jacobi_sweeps < 40
        if chi == 8:
            assert tuple(info.kept) == tuple(info_r["kept"])
        else:
            assert sum(info.kept) == 12
            assert np.max(np.abs(got.data - exact.data)) <= 1e-10 * np.max(np.abs(exact.data))


@pytest.mark.parametrize("chi", [40, 10**6])
def test_compress_wide_bond_cluster_jacobi(F, ctx, chi):
    """A 128 + 128 bond between two tall full-rank sides: 128 x 128 cores,
    rotated by a 16-CTA cluster."""
    lx = [(300, 260, 0), (128, 128, 1)]
    ly = [(128, 128, 0), (280, 270, 1)]
    bx, by = W.random_blocks(lx, 0, 41), W.random_blocks(ly, 0, 42)
    X, Y = O.embed_blocks(lx, 0, bx), O.embed_blocks(ly, 0, by)
    xr, yr, info_r = O.compress(X, Y, [1], [0], chi)
    ref = O.contract(xr, yr, [1], [0])
    xg, yg, info = F.compress(ctx, F.Tensor.from_blocks(ctx, lx, 0, bx), F.Tensor.from_blocks(ctx, ly, 0, by), [1],
                              [0], chi)
    got = O.contract(dense(xg), dense(yg), [1], [0])
    assert np.max(np.abs(got.data - ref.data)) <= 1e-10 * np.max(np.abs(ref.data))
    assert tuple(info.kept) == tuple(info_r["kept"])
    assert abs(info.discarded_sq - info_r["discarded_sq"]) <= 1e-10 * info.total_sq
