"""Parity of the CUDA sign-permute and tensordot path (through the C ABI)
with the CPU oracle.

Tolerances (normwise: max |got - ref| / max |ref| over the compared entries):
FP64 1e-10; TF32x3 1e-5; BF16x3 5e-5; TF32 5e-3; BF16 5e-2 (the operand
rounding of each format times a sqrt(K)-grown accumulation).
"""
import numpy as np
import pytest

import oracle as O
import workloads as W

pytestmark = pytest.mark.gpu

TOL = {"f64": 1e-10, "tf32x3": 1e-5, "f16x3": 1e-5, "bf16x3": 5e-5, "tf32": 5e-3, "bf16": 5e-2}


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


def dense(t_blocks, legs, parity):
    return O.embed_blocks(legs, parity, t_blocks)


def relerr(got, ref):
    den = np.max(np.abs(ref)) if ref.size else 1.0
    return float(np.max(np.abs(got - ref), initial=0.0) / max(den, 1e-300))


def upload(F, ctx, legs, parity, blocks, prec):
    return F.Tensor.from_blocks(ctx, legs, parity, blocks, F.F64 if prec == "f64" else F.F32)


LEGSETS = [
    [(2, 1, 0), (1, 2, 1), (2, 2, 0), (1, 1, 1)],
    [(1, 1, 1), (3, 1, 0), (2, 3, 1), (1, 2, 0), (2, 1, 1)],
    [(3, 0, 1), (2, 2, 0), (0, 2, 1), (1, 3, 0)],
    [(5, 3, 0), (4, 7, 1), (2, 1, 0), (33, 31, 1), (1, 1, 0), (2, 2, 1)],
]


@pytest.mark.parametrize("li", range(len(LEGSETS)))
@pytest.mark.parametrize("parity", [0, 1])
@pytest.mark.parametrize("dt", ["f64", "f32"])
def test_transpose_parity(F, ctx, li, parity, dt):
    legs = LEGSETS[li]
    blocks = W.random_blocks(legs, parity, 100 + li)
    t = F.Tensor.from_blocks(ctx, legs, parity, blocks, F.F64 if dt == "f64" else F.F32)
    ref_in = dense(blocks, legs, parity)
    if dt == "f32":
        ref_in = O.GTensor(ref_in.data.astype(np.float32).astype(np.float64), ref_in.legs, parity)
    for s in range(4):
        perm = W.random_perm(len(legs), 7 * s + li)
        out = F.transpose(ctx, t, perm)
        got = dense(out.to_blocks(), out.legs, out.parity)
        ref = O.transpose(ref_in, perm)
        assert out.legs == ref.legs
        assert np.array_equal(got.data, ref.data)  # sign flips and moves only: exact


def test_dagger_parity(F, ctx):
    legs = LEGSETS[1]
    blocks = W.random_blocks(legs, 1, 5)
    t = F.Tensor.from_blocks(ctx, legs, 1, blocks)
    d = F.dagger(ctx, t)
    ref = O.dagger(dense(blocks, legs, 1))
    assert d.legs == ref.legs
    assert np.array_equal(dense(d.to_blocks(), d.legs, d.parity).data, ref.data)


def random_pair_case(seed):
    g = W.rng(seed)
    n = int(g.integers(0, 4))
    ra, rb = n + int(g.integers(0, 4)), n + int(g.integers(0, 4))
    ra, rb = max(ra, 1), max(rb, 1)
    n = min(n, ra, rb)

    def leg():
        return (int(g.integers(0, 5)), int(g.integers(0, 5)), int(g.integers(0, 2)))

    la = [leg() for _ in range(ra)]
    lb = [leg() for _ in range(rb)]
    ax = [int(v) for v in g.permutation(ra)[:n]]
    ay = [int(v) for v in g.permutation(rb)[:n]]
    for a, b in zip(ax, ay):
        lb[b] = (la[a][0], la[a][1], 1 - la[a][2])
    pa, pb = int(g.integers(0, 2)), int(g.integers(0, 2))
    rc = ra + rb - 2 * n
    perm = [int(v) for v in g.permutation(rc)] if g.integers(0, 2) else None
    flip_a = int(g.integers(0, 1 << ra))
    flip_b = int(g.integers(0, 1 << rb))
    return la, lb, ax, ay, pa, pb, perm, flip_a, flip_b


@pytest.mark.parametrize("prec", ["f64", "tf32x3", "f16x3", "bf16x3", "tf32", "bf16"])
def test_tensordot_random_small(F, ctx, prec):
    """Random ranks, sector sizes (incl. empty sectors), parities, arrows,
    extra bond parities and output permutations."""
    for seed in range(40):
        la, lb, ax, ay, pa, pb, perm, fa, fb = random_pair_case(seed)
        ba, bb = W.random_blocks(la, pa, 2 * seed), W.random_blocks(lb, pb, 2 * seed + 1)
        A, B = dense(ba, la, pa), dense(bb, lb, pb)
        ref = O.contract(A, B, ax, ay, flip_x=[k for k in range(len(la)) if fa >> k & 1],
                         flip_y=[k for k in range(len(lb)) if fb >> k & 1])
        if perm is not None:
            ref = O.transpose(ref, perm)
        a, b = upload(F, ctx, la, pa, ba, prec), upload(F, ctx, lb, pb, bb, prec)
        c = F.tensordot(ctx, a, b, ax, ay, flip_a=fa, flip_b=fb, out_perm=perm, prec=prec)
        got = dense(c.to_blocks(), c.legs, c.parity)
        assert c.legs == ref.legs and c.parity == ref.parity
        assert relerr(got.data, ref.data) <= TOL[prec], (seed, relerr(got.data, ref.data))
    ctx.synchronize()


@pytest.mark.parametrize("name", ["T1", "T2", "T3", "T4"])
@pytest.mark.parametrize("prec", ["f64", "tf32x3", "f16x3", "bf16x3", "tf32"])
def test_tensordot_cases_reduced(F, ctx, name, prec):
    """The four microbenchmark contractions with every sector dimension halved:
    full element-wise comparison (several tiles and ragged tails)."""
    case = W.tensordot_case(name, seed=1, shrink=2 if name != "T4" else 4)
    ba = W.random_blocks(case["legs_a"], 0, case["seed_a"])
    bb = W.random_blocks(case["legs_b"], 0, case["seed_b"])
    ref = O.transpose(O.contract(dense(ba, case["legs_a"], 0), dense(bb, case["legs_b"], 0), case["axes_a"],
                                 case["axes_b"]), case["out_perm"])
    a, b = upload(F, ctx, case["legs_a"], 0, ba, prec), upload(F, ctx, case["legs_b"], 0, bb, prec)
    c = F.tensordot(ctx, a, b, case["axes_a"], case["axes_b"], out_perm=case["out_perm"], prec=prec)
    got = dense(c.to_blocks(), c.legs, c.parity)
    assert relerr(got.data, ref.data) <= TOL[prec]
    ctx.synchronize()


_FULL_REF = {}


def full_size_reference(name):
    """Dense oracle result of a full-size microbenchmark contraction (cached:
    the same reference serves every precision)."""
    if name not in _FULL_REF:
        case = W.tensordot_case(name, seed=0)
        ba = W.random_blocks(case["legs_a"], 0, case["seed_a"])
        bb = W.random_blocks(case["legs_b"], 0, case["seed_b"])
        ref = O.transpose(O.contract(dense(ba, case["legs_a"], 0), dense(bb, case["legs_b"], 0), case["axes_a"],
                                     case["axes_b"]), case["out_perm"])
        _FULL_REF[name] = (case, ba, bb, ref)
    return _FULL_REF[name]


def packed_like(t, ref):
    """The oracle's dense result packed in the GPU tensor's block layout."""
    blocks = O.extract_blocks(ref)
    flat = np.zeros(t.numel, dtype=np.float64)
    for m, off in t.block_table():
        blk = blocks[t.bits_of(m)]
        flat[off:off + blk.size] = blk.reshape(-1)
    return flat


@pytest.mark.parametrize("name", ["T1", "T2", "T3", "T4"])
@pytest.mark.parametrize("prec", ["f64", "tf32x3", "f16x3"])
def test_tensordot_cases_full_size(F, ctx, name, prec):
    """Full-size microbenchmark shapes in the launch configuration the
    benchmark times (same permutations, tuned tile widths, contiguous tile
    ranges, staged permutes, merged GEMM groups): every output entry against
    the oracle."""
    case, ba, bb, ref = full_size_reference(name)
    a, b = upload(F, ctx, case["legs_a"], 0, ba, prec), upload(F, ctx, case["legs_b"], 0, bb, prec)
    c = F.tensordot(ctx, a, b, case["axes_a"], case["axes_b"], out_perm=case["out_perm"], prec=prec)
    assert c.legs == ref.legs and c.parity == ref.parity
    got = c.download().astype(np.float64)
    want = packed_like(c, ref)
    assert relerr(got, want) <= TOL[prec], relerr(got, want)
    ctx.synchronize()


@pytest.mark.parametrize("scale", [0.125, 1.0, 3000.0])
def test_f16x3_within_its_range(F, ctx, scale):
    """F16X3 keeps the FP32-level normwise accuracy while the largest operand
    entry lies in its stated range (here N(0,1) data times scale, so the
    largest entries are about 4 * scale)."""
    case = W.tensordot_case("T3", seed=3, shrink=2)
    ba = [(bits, blk * scale) for bits, blk in W.random_blocks(case["legs_a"], 0, case["seed_a"])]
    bb = [(bits, blk * scale) for bits, blk in W.random_blocks(case["legs_b"], 0, case["seed_b"])]
    ref = O.transpose(O.contract(dense(ba, case["legs_a"], 0), dense(bb, case["legs_b"], 0), case["axes_a"],
                                 case["axes_b"]), case["out_perm"])
    a, b = upload(F, ctx, case["legs_a"], 0, ba, "f16x3"), upload(F, ctx, case["legs_b"], 0, bb, "f16x3")
    c = F.tensordot(ctx, a, b, case["axes_a"], case["axes_b"], out_perm=case["out_perm"], prec="f16x3")
    got = dense(c.to_blocks(), c.legs, c.parity)
    assert relerr(got.data, ref.data) <= TOL["f16x3"]
    ctx.synchronize()


def test_errors_are_reported(F, ctx):
    la = [(2, 1, 0), (1, 2, 1)]
    a = F.Tensor.from_blocks(ctx, la, 0, W.random_blocks(la, 0, 1))
    b = F.Tensor.from_blocks(ctx, la, 0, W.random_blocks(la, 0, 2))
    with pytest.raises(F.FtnError) as e:
        F.tensordot(ctx, a, b, [0], [0])  # same duals
    assert e.value.status == -4
    with pytest.raises(F.FtnError) as e:
        F.tensordot(ctx, a, b, [0], [1])  # sector dims differ
    assert e.value.status == -2
    with pytest.raises(F.FtnError) as e:
        F.tensordot(ctx, a, b, [0], [1], prec="tf32")  # FP64 data on a TF32 path
    assert e.value.status == -8


def test_misaligned_wrapped_input_uses_fallback_permute(F, ctx):
    """A borrowed buffer that is not 16-byte aligned cannot feed the TMA-staged
    permute; the register-staged kernel must take over with the same result."""
    import torch

    case = W.tensordot_case("T2", seed=2, shrink=2)
    for prec, tdt in (("f64", torch.float64), ("tf32x3", torch.float32)):
        ba = W.random_blocks(case["legs_a"], 0, case["seed_a"])
        bb = W.random_blocks(case["legs_b"], 0, case["seed_b"])
        ref = O.transpose(O.contract(dense(ba, case["legs_a"], 0), dense(bb, case["legs_b"], 0), case["axes_a"],
                                     case["axes_b"]), case["out_perm"])
        a0 = upload(F, ctx, case["legs_a"], 0, ba, prec)
        store = torch.empty(a0.numel + 1, dtype=tdt, device="cuda")
        store[1:].copy_(a0.view())
        a = F.Tensor.wrap(ctx, case["legs_a"], 0, store[1:])
        assert a.ptr % 16 != 0
        b = upload(F, ctx, case["legs_b"], 0, bb, prec)
        c = F.tensordot(ctx, a, b, case["axes_a"], case["axes_b"], out_perm=case["out_perm"], prec=prec)
        got = dense(c.to_blocks(), c.legs, c.parity)
        assert relerr(got.data, ref.data) <= TOL[prec]
        t = F.transpose(ctx, a, list(reversed(range(len(case["legs_a"])))))
        want = O.transpose(dense(a0.to_blocks(), a0.legs, 0), list(reversed(range(len(case["legs_a"])))))
        assert np.array_equal(dense(t.to_blocks(), t.legs, t.parity).data, want.data)
    ctx.synchronize()


def test_misaligned_preallocated_output_is_rejected(F, ctx):
    """The epilogues and the permute write 16-byte vectors, so a caller's
    preallocated output must be 16-byte aligned: a misaligned one is refused
    before any launch, and an aligned one is accepted."""
    import torch

    case = W.tensordot_case("T3", seed=1, shrink=2)
    a = upload(F, ctx, case["legs_a"], 0, W.random_blocks(case["legs_a"], 0, 1), "tf32x3")
    b = upload(F, ctx, case["legs_b"], 0, W.random_blocks(case["legs_b"], 0, 2), "tf32x3")
    c = F.tensordot(ctx, a, b, case["axes_a"], case["axes_b"], out_perm=case["out_perm"], prec="tf32x3")
    store = torch.empty(c.numel + 4, dtype=torch.float32, device="cuda")
    bad = F.Tensor.wrap(ctx, c.legs, c.parity, store[1:1 + c.numel])
    assert bad.ptr % 16 != 0
    with pytest.raises(F.FtnError) as e:
        F.tensordot(ctx, a, b, case["axes_a"], case["axes_b"], out_perm=case["out_perm"], prec="tf32x3", out=bad)
    assert e.value.status == -1  # FTN_EINVAL
    with pytest.raises(F.FtnError):
        F.transpose(ctx, c, list(range(len(c.legs))), out=bad)
    good = F.Tensor.wrap(ctx, c.legs, c.parity, store[4:4 + c.numel])
    F.tensordot(ctx, a, b, case["axes_a"], case["axes_b"], out_perm=case["out_perm"], prec="tf32x3", out=good)
    assert np.array_equal(good.download(), c.download())
    ctx.synchronize()


NARROW = [
    # (A legs, B legs, axes A, axes B, out_perm): long contracted legs, few
    # output tiles (split-K with the ordered slab reduction) and narrow
    # column blocks (16- and 32-wide FP64 tiles); ragged sizes throughout
    ([(9, 7, 0), (64, 50, 1), (3, 2, 0)], [(64, 50, 0), (5, 6, 1)], [1], [0], None),
    ([(9, 7, 0), (64, 50, 1), (3, 2, 0)], [(64, 50, 0), (5, 6, 1)], [1], [0], [2, 0, 1]),
    ([(17, 15, 1), (40, 33, 0), (2, 3, 1)], [(2, 3, 0), (40, 33, 1), (20, 12, 0)], [1, 2], [1, 0], [1, 0]),
    ([(130, 70, 0), (8, 9, 1), (4, 4, 0)], [(8, 9, 0), (4, 4, 1), (30, 29, 1)], [1, 2], [0, 1], None),
    ([(3, 1, 0), (2, 2, 1), (96, 64, 0)], [(96, 64, 1), (2, 2, 0), (45, 50, 1)], [2, 1], [0, 1], [1, 0]),
]


@pytest.mark.parametrize("ci", range(len(NARROW)))
@pytest.mark.parametrize("parity", [(0, 0), (1, 0), (1, 1)])
def test_tensordot_f64_splitk_and_narrow_tiles(F, ctx, ci, parity):
    la, lb, ax, ay, perm = NARROW[ci]
    pa, pb = parity
    ba, bb = W.random_blocks(la, pa, 300 + ci), W.random_blocks(lb, pb, 400 + ci)
    ref = O.contract(dense(ba, la, pa), dense(bb, lb, pb), ax, ay)
    if perm is not None:
        ref = O.transpose(ref, perm)
    a, b = upload(F, ctx, la, pa, ba, "f64"), upload(F, ctx, lb, pb, bb, "f64")
    for _ in range(2):  # the second call runs from the cached plan
        c = F.tensordot(ctx, a, b, ax, ay, out_perm=perm, prec="f64")
        got = dense(c.to_blocks(), c.legs, c.parity)
        assert c.legs == ref.legs and c.parity == ref.parity
        assert relerr(got.data, ref.data) <= TOL["f64"]


@pytest.mark.parametrize("name", ["T1", "T4"])
def test_tile_width_tuning_keeps_every_bit(F, name):
    """The first use of a large tensor-core contraction times its GEMM at a few
    tile widths and keeps the fastest: a tuning context and one that keeps the
    default width give the same result bit for bit (every output element
    accumulates its K products in the same order whatever the tiling), and the
    tuned plan's later calls repeat it."""
    case = W.tensordot_case(name, seed=0)
    ba = W.random_blocks(case["legs_a"], 0, case["seed_a"])
    bb = W.random_blocks(case["legs_b"], 0, case["seed_b"])
    outs = []
    for tune in (True, False):
        c = F.Context()
        try:
            c.set_tuning(tune)
            a, b = upload(F, c, case["legs_a"], 0, ba, "f16x3"), upload(F, c, case["legs_b"], 0, bb, "f16x3")
            r = [F.tensordot(c, a, b, case["axes_a"], case["axes_b"], out_perm=case["out_perm"],
                             prec="f16x3").download() for _ in range(2)]
            assert np.array_equal(r[0], r[1])
            outs.append(r[0])
        finally:
            c.synchronize()
            c.close()
    assert np.array_equal(outs[0], outs[1])


@pytest.mark.parametrize("dt", ["f64", "f32"])
@pytest.mark.parametrize("parity", [0, 1])
def test_transpose_many_jobs(F, ctx, dt, parity):
    """2048 blocks of 64 entries (ten legs of dimension 1 + 1 around two
    larger ones): the shared-memory-staged permute runs one job per tile, so
    every CTA starts with a 32-way search over 2048 jobs and changes job on
    every tile; exact against the oracle for several leg orders."""
    legs = [(1, 1, q % 2) for q in range(5)] + [(32, 32, 0), (2, 2, 1)] + [(1, 1, q % 2) for q in range(5)]
    blocks = W.random_blocks(legs, parity, 41 + parity)
    assert len(blocks) == 2048
    t = F.Tensor.from_blocks(ctx, legs, parity, blocks, F.F64 if dt == "f64" else F.F32)
    ref_in = dense(blocks, legs, parity)
    if dt == "f32":
        ref_in = O.GTensor(ref_in.data.astype(np.float32).astype(np.float64), ref_in.legs, parity)
    for s in range(3):
        perm = W.random_perm(len(legs), 90 + s)
        out = F.transpose(ctx, t, perm)
        got = dense(out.to_blocks(), out.legs, out.parity)
        ref = O.transpose(ref_in, perm)
        assert np.array_equal(got.data, ref.data)
    ctx.synchronize()


@pytest.mark.parametrize("prec", ["tf32x3", "f16x3"])
def test_merged_group_of_many_members(F, ctx, prec):
    """B's 64 column blocks per bond sector, each 32 wide, form one merged
    group per row block (more members than a warp's lanes): the GEMM epilogue
    finds each 32-column chunk's member by walking the group.  Against the
    oracle."""
    la = [(64, 64, 0), (16, 16, 0), (4, 4, 0)]
    lb = [(4, 4, 1)] + [(2, 2, 0)] * 5 + [(1, 1, 0)] * 2
    ba, bb = W.random_blocks(la, 0, 61), W.random_blocks(lb, 0, 62)
    ref = O.contract(dense(ba, la, 0), dense(bb, lb, 0), [2], [0])
    a, b = upload(F, ctx, la, 0, ba, prec), upload(F, ctx, lb, 0, bb, prec)
    c = F.tensordot(ctx, a, b, [2], [0], prec=prec)
    got = dense(c.to_blocks(), c.legs, c.parity)
    assert relerr(got.data, ref.data) <= TOL[prec]
    ctx.synchronize()


@pytest.mark.parametrize("prec", ["tf32x3", "f16x3", "bf16x3"])
@pytest.mark.parametrize("perm", [None, [1, 0]])
def test_partial_last_round_and_ragged_columns(F, ctx, prec, perm):
    """A launch of 152 + 20 tiles of 128 x 128 (one full round on the 152
    SMs and 20 tiles in a second, partial one), one problem whose last
    column tile holds 40 valid columns.  Every output entry against the
    oracle, with and without an output permutation (fused epilogue writes)."""
    la = [(1664, 128, 0), (64, 64, 1)]
    lb = [(64, 64, 0), (1664, 296, 0)]
    ba, bb = W.random_blocks(la, 0, 21), W.random_blocks(lb, 0, 22)
    A, B = dense(ba, la, 0), dense(bb, lb, 0)
    ref = O.contract(A, B, [1], [0])
    if perm is not None:
        ref = O.transpose(ref, perm)
    a, b = upload(F, ctx, la, 0, ba, prec), upload(F, ctx, lb, 0, bb, prec)
    c = F.tensordot(ctx, a, b, [1], [0], out_perm=perm, prec=prec)
    assert relerr(c.download().astype(np.float64), packed_like(c, ref)) <= TOL[prec]
    ctx.synchronize()
