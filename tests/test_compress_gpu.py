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


def _orth(g, n, k):
    q, r = np.linalg.qr(g.standard_normal((n, k)))
    return q * np.sign(np.diag(r))


def _graded_with_spectrum(legs, parity, bond_first, spectra, seed):
    """A dense graded tensor whose bond-parity sector matrices have prescribed
    singular values.  The bond is one leg, last (bond_first False: the
    matrix is [free | bond]) or first (True: [bond | free]), so the
    matricisation of the compression is a plain reshape up to column signs,
    which leave singular values unchanged.  spectra[pi] lists the singular
    values of sector pi (as many as the smaller side allows)."""
    g = W.rng(seed)
    free = legs[1:] if bond_first else legs[:-1]
    bond = legs[0] if bond_first else legs[-1]
    fdims = [a + b for a, b, _ in free]
    fpar = np.zeros(1, np.int64)
    for d0, d1, _ in free:
        fpar = (fpar[:, None] + O.index_parity(d0, d1)[None, :]).reshape(-1) & 1
    bpar = O.index_parity(bond[0], bond[1])
    mat = np.zeros((int(np.prod(fdims)), bond[0] + bond[1]))
    for pi in (0, 1):
        rows = np.nonzero(fpar == (parity ^ pi))[0]
        cols = np.nonzero(bpar == pi)[0]
        k = min(len(rows), len(cols))
        s = np.asarray(spectra[pi][:k], dtype=np.float64)
        mat[np.ix_(rows, cols)] = (_orth(g, len(rows), k) * s) @ _orth(g, len(cols), k).T
    if bond_first:
        data = mat.T.reshape([bond[0] + bond[1]] + fdims)
    else:
        data = mat.reshape(fdims + [bond[0] + bond[1]])
    t = O.GTensor(data, legs, parity)
    assert t.check_symmetry()
    return t


def _spectrum(kind, n):
    if kind == "log12":
        return np.logspace(0, -12, n)
    return 0.5 ** np.arange(n)  # the stand-in gauges of the cluster workload


@pytest.mark.parametrize("kind", ["log12", "half"])
@pytest.mark.parametrize("chi", [10**6, 30, 9])
@pytest.mark.parametrize("other", ["ill", "gauss", "orthonormal"])
@pytest.mark.parametrize("px", [0, 1])
def test_compress_ill_conditioned(F, ctx, kind, chi, other, px):
    """X's sector blocks U diag(sigma) V^T with sigma spanning 1 ... 1e-12 (or
    0.5^k), against Y ill-conditioned the same way, N(0, 1), or with
    orthonormal sector blocks: chi above the rank (the exact product must
    survive) and chi cutting inside the spectrum, against the oracle at 1e-10
    relative.  (A Gram matrix of X carries only rounding noise in its
    directions below ~1e-8 of the largest; a one-sided ill-conditioned bond
    exposes that.)"""
    lx = [(6, 6, 0), (5, 5, 1), (24, 24, 0)]
    ly = [(24, 24, 1), (7, 7, 0), (6, 6, 1)]
    X = _graded_with_spectrum(lx, px, False, {0: _spectrum(kind, 24), 1: 0.7 * _spectrum(kind, 24)}, 5 + px)
    if other == "ill":
        Y = _graded_with_spectrum(ly, 0, True, {0: 0.9 * _spectrum(kind, 24), 1: _spectrum(kind, 24)}, 7 + px)
    elif other == "gauss":
        Y = O.embed_blocks(ly, 0, W.random_blocks(ly, 0, 9 + px))
    else:
        Y = _graded_with_spectrum(ly, 0, True, {0: np.ones(24), 1: np.ones(24)}, 7 + px)
    xr, yr, info_r = O.compress(X, Y, [2], [0], chi)
    ref = O.contract(xr, yr, [xr.rank - 1], [0])
    x = F.Tensor.from_blocks(ctx, lx, px, sorted(O.extract_blocks(X).items()))
    y = F.Tensor.from_blocks(ctx, ly, 0, sorted(O.extract_blocks(Y).items()))
    xg, yg, info = F.compress(ctx, x, y, [2], [0], chi)
    got = O.contract(dense(xg), dense(yg), [xg.rank - 1], [0])
    err = np.max(np.abs(got.data - ref.data)) / np.max(np.abs(ref.data))
    assert err <= 1e-10, err
    if chi >= 48:
        exact = O.contract(X, Y, [2], [0])
        assert np.max(np.abs(got.data - exact.data)) <= 1e-10 * np.max(np.abs(exact.data))
    elif info_r["gap"] > 1e-12 * info_r["singular_values"][0]:
        # the kept set is decided by more than rounding
        assert tuple(info.kept) == tuple(info_r["kept"])
        assert abs(info.discarded_sq - info_r["discarded_sq"]) <= 1e-10 * info.total_sq


@pytest.mark.parametrize("rows_odd,k", [(260, 128), (264, 128), (268, 128), (270, 128), (256, 128), (260, 64),
                                         (161, 128)])
def test_compress_qr_chunk_tails(F, ctx, rows_odd, k):
    """The Householder QR splits a tall sector into chunks of at least K rows
    and merges their factors: last chunks of 4, 8, 12 and 14 rows (after whose
    rank the leftover rounding noise shrinks towards underflow), one chunk,
    two chunks, and the shortest side still factored (5/4 K rows).  The
    odd-parity sector of X has singular values over 1 ... 1e-10, so its Gram
    factor has pivots in the unresolved band and the side goes to the
    Householder QR (checked through the profile labels)."""
    lx = [(300, rows_odd, 0), (k, k, 1)]
    ly = [(k, k, 0), (280, 270, 1)]
    bx, by = dict(W.random_blocks(lx, 0, 41)), W.random_blocks(ly, 0, 42)
    g = W.rng(43)
    u = np.linalg.qr(g.standard_normal((rows_odd, k)))[0]
    v = np.linalg.qr(g.standard_normal((k, k)))[0]
    bx[(1, 1)] = (u * np.logspace(0, -10, k)) @ v.T
    bx = sorted(bx.items())
    X, Y = O.embed_blocks(lx, 0, bx), O.embed_blocks(ly, 0, by)
    xr, yr, info_r = O.compress(X, Y, [1], [0], 10**6)
    ref = O.contract(xr, yr, [1], [0])
    ctx.profile(True)
    try:
        xg, yg, info = F.compress(ctx, F.Tensor.from_blocks(ctx, lx, 0, bx), F.Tensor.from_blocks(ctx, ly, 0, by),
                                  [1], [0], 10**6)
        labels = {r["label"]: r["launches"] for r in ctx.profile_read()}
    finally:
        ctx.profile(False)
    got = O.contract(dense(xg), dense(yg), [1], [0])
    assert np.max(np.abs(got.data - ref.data)) <= 1e-10 * np.max(np.abs(ref.data))
    assert tuple(info.kept) == tuple(info_r["kept"])
    assert labels.get("householder_qr", 0) > 0


@pytest.mark.parametrize("rows,other", [(139, 128), (400, 12), (128, 128), (1100, 12)])
def test_compress_side_as_own_factor(F, ctx, rows, other):
    """Sides that are not factored: fewer than 5/4 K rows (139 x 128), or a
    partner side of at most K/8 rows (400 x 128 against 12 rows), are their own
    R factor; a side beyond 1024 rows is factored whatever its partner.  Each
    against the oracle at 1e-10 with chi above the rank, and with chi = 7."""
    k = 128
    lx = [(rows, rows, 0), (k, k, 1)]
    ly = [(k, k, 0), (other, other, 1)]
    bx, by = W.random_blocks(lx, 0, 51), W.random_blocks(ly, 0, 52)
    X, Y = O.embed_blocks(lx, 0, bx), O.embed_blocks(ly, 0, by)
    for chi in (10**6, 7):
        xr, yr, info_r = O.compress(X, Y, [1], [0], chi)
        ref = O.contract(xr, yr, [1], [0])
        xg, yg, info = F.compress(ctx, F.Tensor.from_blocks(ctx, lx, 0, bx), F.Tensor.from_blocks(ctx, ly, 0, by),
                                  [1], [0], chi)
        if info_r["gap"] is not None:  # a cut decided by more than rounding
            assert info_r["gap"] > 1e-6 * info_r["singular_values"][0]
        got = O.contract(dense(xg), dense(yg), [1], [0])
        assert np.max(np.abs(got.data - ref.data)) <= 1e-10 * np.max(np.abs(ref.data))
        assert tuple(info.kept) == tuple(info_r["kept"])


@pytest.mark.parametrize("small,redo", [(1e-8, True), (1e-14, False)])
def test_compress_gram_residual_decides(F, ctx, small, redo):
    """Sector blocks with singular values 1 (x12) and ``small`` (x12): the
    Gram matrix's pivots for the small directions are at rounding level, so the
    semi-definite Cholesky drops them; the residual certificate |A T|_F then
    decides.  At 1e-8 the dropped directions matter (|E|^2 ~ 1e-16 |A|^2 >
    1e-24 |A|^2): the side is factored again by Householder TSQR and the job's
    cores decomposed again.  At 1e-14 they are below the certificate's 1e-12
    and the Gram factor stands.  Both against the oracle at 1e-10."""
    lx = [(6, 6, 0), (5, 5, 1), (24, 24, 0)]
    ly = [(24, 24, 1), (7, 7, 0), (6, 6, 1)]
    spec = np.concatenate([np.ones(12), np.full(12, small)])
    X = _graded_with_spectrum(lx, 0, False, {0: spec, 1: 0.7 * spec}, 11)
    Y = O.embed_blocks(ly, 0, W.random_blocks(ly, 0, 13))
    xr, yr, _ = O.compress(X, Y, [2], [0], 10**6)
    ref = O.contract(xr, yr, [xr.rank - 1], [0])
    x = F.Tensor.from_blocks(ctx, lx, 0, sorted(O.extract_blocks(X).items()))
    y = F.Tensor.from_blocks(ctx, ly, 0, sorted(O.extract_blocks(Y).items()))
    ctx.profile(True)
    try:
        xg, yg, _ = F.compress(ctx, x, y, [2], [0], 10**6)
        labels = {r["label"]: r["launches"] for r in ctx.profile_read()}
    finally:
        ctx.profile(False)
    got = O.contract(dense(xg), dense(yg), [xg.rank - 1], [0])
    assert np.max(np.abs(got.data - ref.data)) <= 1e-10 * np.max(np.abs(ref.data))
    assert labels.get("householder_qr", 0) == 0  # no pivot in the unresolved band
    assert (labels.get("householder_qr_redo", 0) > 0) == redo
