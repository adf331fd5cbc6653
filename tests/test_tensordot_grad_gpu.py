"""Parity of ftn_tensordot_grad (the adjoint of the fermionic tensordot,
through the C ABI) with the oracle's gradient by definition, the adjoint
identity on larger contractions, and the autograd path of the binding.
Tolerances as for the tensordot: FP64 1e-10, TF32x3 1e-5 (normwise)."""
import numpy as np
import pytest

import oracle as O
import workloads as W

pytestmark = pytest.mark.gpu

TOL = {"f64": 1e-10, "tf32x3": 1e-5, "f16x3": 1e-5}


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


def dense(F, t):
    return O.embed_blocks(t.legs, t.parity, t.to_blocks())


def relerr(got, ref):
    den = np.max(np.abs(ref)) if ref.size else 1.0
    return float(np.max(np.abs(got - ref), initial=0.0) / max(den, 1e-300))


def small_case(seed):
    """Random pair of graded tensors (ranks 1-4, sectors of 1-2 states),
    contracted legs, parities, bond-parity flips and an output permutation."""
    g = W.rng(7000 + seed)
    ra, rb = int(g.integers(1, 4)), int(g.integers(1, 4))
    n = int(g.integers(0, min(ra, rb) + 1))
    leg = lambda: (int(g.integers(1, 3)), int(g.integers(1, 3)), int(g.integers(0, 2)))  # noqa: E731
    la = [leg() for _ in range(ra)]
    lb = [leg() for _ in range(rb)]
    ax = [int(v) for v in g.permutation(ra)[:n]]
    ay = [int(v) for v in g.permutation(rb)[:n]]
    for a, b in zip(ax, ay):
        lb[b] = (la[a][0], la[a][1], 1 - la[a][2])
    pa, pb = int(g.integers(0, 2)), int(g.integers(0, 2))
    rc = ra + rb - 2 * n
    perm = [int(v) for v in g.permutation(rc)] if rc and g.integers(0, 2) else None
    fa, fb = int(g.integers(0, 1 << ra)), int(g.integers(0, 1 << rb))
    return la, lb, ax, ay, pa, pb, perm, fa, fb


@pytest.mark.parametrize("prec", ["f64", "tf32x3", "f16x3"])
def test_grad_matches_oracle_by_definition(F, ctx, prec):
    dt = F.F64 if prec == "f64" else F.F32
    for seed in range(24):
        la, lb, ax, ay, pa, pb, perm, fa, fb = small_case(seed)
        ba, bb = W.random_blocks(la, pa, 2 * seed), W.random_blocks(lb, pb, 2 * seed + 1)
        if prec != "f64":
            ba = [(k, v.astype(np.float32).astype(np.float64)) for k, v in ba]
            bb = [(k, v.astype(np.float32).astype(np.float64)) for k, v in bb]
        X, Y = O.embed_blocks(la, pa, ba), O.embed_blocks(lb, pb, bb)
        flx = [k for k in range(len(la)) if fa >> k & 1]
        fly = [k for k in range(len(lb)) if fb >> k & 1]
        c = O.contract_forward(X, Y, ax, ay, flip_x=flx, flip_y=fly, out_perm=perm)
        bg = W.random_blocks(c.legs, c.parity, 9000 + seed)
        if prec != "f64":
            bg = [(k, v.astype(np.float32).astype(np.float64)) for k, v in bg]
        G = O.embed_blocks(c.legs, c.parity, bg)
        ref_a = O.contract_grad(X, Y, ax, ay, G, wrt="x", flip_x=flx, flip_y=fly, out_perm=perm)
        ref_b = O.contract_grad(X, Y, ax, ay, G, wrt="y", flip_x=flx, flip_y=fly, out_perm=perm)
        a = F.Tensor.from_blocks(ctx, la, pa, ba, dt)
        b = F.Tensor.from_blocks(ctx, lb, pb, bb, dt)
        g = F.Tensor.from_blocks(ctx, c.legs, c.parity, bg, dt)
        da, db = F.tensordot_grad(ctx, a, b, g, ax, ay, fa, fb, perm, prec)
        assert da.legs == ref_a.legs and db.legs == ref_b.legs
        assert relerr(dense(F, da).data, ref_a.data) <= TOL[prec], seed
        assert relerr(dense(F, db).data, ref_b.data) <= TOL[prec], seed


@pytest.mark.parametrize("name", ["T3", "T4"])
def test_adjoint_identity_reduced_cases(F, ctx, name):
    """<dA, A> = <G, C> = <dB, B> for the microbenchmark shapes (halved)."""
    case = W.tensordot_case(name, seed=3, shrink=2)
    ba = W.random_blocks(case["legs_a"], 0, case["seed_a"])
    bb = W.random_blocks(case["legs_b"], 0, case["seed_b"])
    a = F.Tensor.from_blocks(ctx, case["legs_a"], 0, ba)
    b = F.Tensor.from_blocks(ctx, case["legs_b"], 0, bb)
    c = F.tensordot(ctx, a, b, case["axes_a"], case["axes_b"], out_perm=case["out_perm"], prec="f64")
    g = F.Tensor.from_blocks(ctx, c.legs, c.parity, W.random_blocks(c.legs, c.parity, 77))
    da, db = F.tensordot_grad(ctx, a, b, g, case["axes_a"], case["axes_b"], out_perm=case["out_perm"], prec="f64")
    form = float(np.dot(g.download(), c.download()))
    assert abs(float(np.dot(da.download(), a.download())) - form) <= 1e-12 * abs(form)
    assert abs(float(np.dot(db.download(), b.download())) - form) <= 1e-12 * abs(form)


def test_autograd_backward(F, ctx):
    import torch

    seed = 5
    while not small_case(seed)[2]:
        seed += 1
    la, lb, ax, ay, pa, pb, perm, fa, fb = small_case(seed)
    ba, bb = W.random_blocks(la, pa, 1), W.random_blocks(lb, pb, 2)
    a = F.Tensor.from_blocks(ctx, la, pa, ba)
    b = F.Tensor.from_blocks(ctx, lb, pb, bb)
    at = torch.tensor(a.download(), device="cuda", requires_grad=True)
    bt = torch.tensor(b.download(), device="cuda", requires_grad=True)
    c, lc, pc = F.tensordot_autograd(ctx, at, la, pa, bt, lb, pb, ax, ay, fa, fb, perm, "f64")
    w = torch.randn_like(c)
    (w * c).sum().backward()
    g = F.Tensor.wrap(ctx, lc, pc, w.detach().contiguous())
    da, db = F.tensordot_grad(ctx, a, b, g, ax, ay, fa, fb, perm, "f64")
    assert np.allclose(at.grad.cpu().numpy(), da.download(), rtol=0, atol=1e-12)
    assert np.allclose(bt.grad.cpu().numpy(), db.download(), rtol=0, atol=1e-12)


def test_grad_rejects_wrong_result_legs(F, ctx):
    la = [(2, 1, 0), (1, 2, 1)]
    lb = [(1, 2, 0), (2, 2, 1)]
    a = F.Tensor.from_blocks(ctx, la, 0, W.random_blocks(la, 0, 1))
    b = F.Tensor.from_blocks(ctx, lb, 0, W.random_blocks(lb, 0, 2))
    bad = [(2, 2, 1), (2, 1, 0)]  # C's legs in the wrong order
    g = F.Tensor.from_blocks(ctx, bad, 0, W.random_blocks(bad, 0, 3))
    with pytest.raises(F.FtnError):
        F.tensordot_grad(ctx, a, b, g, [1], [0])


@pytest.mark.parametrize("prec", ["tf32x3", "f16x3"])
@pytest.mark.parametrize("name", ["T1", "T2"])
def test_long_contraction_gradient_full_size(F, ctx, name, prec):
    """dB of T1 / T2 contracts over every free state of the environment
    (131072 / 16384 per sector): the tensor-core gradient runs it as K parts
    accumulated in FP32 and added in FP64.  TF32x3 vs FP64 gradients of the
    same FP32-rounded inputs, normwise 1e-5 (TF32x3 and F16X3)."""
    c = W.tensordot_case(name, seed=0)
    rnd = lambda legs, par, seed: [(k, v.astype(np.float32).astype(np.float64))  # noqa: E731
                                   for k, v in W.random_blocks(legs, par, seed)]
    ba, bb = rnd(c["legs_a"], 0, 1), rnd(c["legs_b"], 0, 2)
    a64 = F.Tensor.from_blocks(ctx, c["legs_a"], 0, ba)
    b64 = F.Tensor.from_blocks(ctx, c["legs_b"], 0, bb)
    r = F.tensordot(ctx, a64, b64, c["axes_a"], c["axes_b"], out_perm=c["out_perm"], prec="f64")
    bg = rnd(r.legs, r.parity, 3)
    g64 = F.Tensor.from_blocks(ctx, r.legs, r.parity, bg)
    ref = F.tensordot_grad(ctx, a64, b64, g64, c["axes_a"], c["axes_b"], out_perm=c["out_perm"], prec="f64")
    a32 = F.Tensor.from_blocks(ctx, c["legs_a"], 0, ba, F.F32)
    b32 = F.Tensor.from_blocks(ctx, c["legs_b"], 0, bb, F.F32)
    g32 = F.Tensor.from_blocks(ctx, r.legs, r.parity, bg, F.F32)
    got = F.tensordot_grad(ctx, a32, b32, g32, c["axes_a"], c["axes_b"], out_perm=c["out_perm"], prec=prec)
    for x, y in zip(got, ref):
        assert relerr(x.download().astype(np.float64), y.download()) <= TOL[prec]
