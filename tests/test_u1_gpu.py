"""U(1)-symmetric tensors (fermion-number charges, parity = charge mod 2,
Sec. II.B) through the library's Z2 kernels: a U(1)-symmetric tensor is a
Z2 tensor with more zeros, so the contraction and the compression apply
unchanged; their results agree with the oracle and keep the charge
structure (the GPU does not exploit the finer charge blocks)."""
import numpy as np
import pytest

import oracle as O
import oracle.u1 as U

pytestmark = pytest.mark.gpu

from test_oracle_u1 import CASES  # noqa: E402


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


def upload(F, ctx, t, dt):
    return F.Tensor.from_blocks(ctx, t.legs, t.parity, list(O.extract_blocks(t).items()), dt)


def dense(t):
    return O.embed_blocks(t.legs, t.parity, t.to_blocks())


@pytest.mark.parametrize("case", CASES)
@pytest.mark.parametrize("prec", ["f64", "tf32x3"])
def test_u1_contraction_on_the_gpu(F, ctx, case, prec):
    lx, ly, ax, ay, qx, qy = case
    x, y = U.random_u1(lx, qx, 11), U.random_u1(ly, qy, 12)
    dt = F.F64 if prec == "f64" else F.F32
    if prec != "f64":
        x = O.GTensor(x.data.astype(np.float32).astype(np.float64), x.legs, x.parity)
        y = O.GTensor(y.data.astype(np.float32).astype(np.float64), y.legs, y.parity)
    ref = O.contract(x, y, ax, ay)
    got = dense(F.tensordot(ctx, upload(F, ctx, x, dt), upload(F, ctx, y, dt), ax, ay, prec=prec))
    scale = np.max(np.abs(ref.data))
    assert np.max(np.abs(got.data - ref.data)) <= (1e-10 if prec == "f64" else 1e-5) * scale
    lz = U.u1_result_legs(lx, ly, ax, ay)
    assert U.u1_violation(got, lz, qx + qy) == 0.0  # every product outside has a zero factor
    ctx.synchronize()


@pytest.mark.parametrize("case", CASES)
def test_u1_compression_on_the_gpu(F, ctx, case):
    lx, ly, ax, ay, qx, qy = case
    x, y = U.random_u1(lx, qx, 13), U.random_u1(ly, qy, 14)
    _, _, info = O.compress(x, y, ax, ay, chi=10**6)
    chi = max(1, len(info["singular_values"]) // 2)
    xr, yr, _ = O.compress(x, y, ax, ay, chi)
    ref = O.contract(xr, yr, [xr.rank - 1], [0])
    xn, yn, _ = F.compress(ctx, upload(F, ctx, x, F.F64), upload(F, ctx, y, F.F64), ax, ay, chi)
    z = dense(F.tensordot(ctx, xn, yn, [len(xn.legs) - 1], [0]))
    scale = np.max(np.abs(ref.data))
    assert np.max(np.abs(z.data - ref.data)) <= 1e-10 * scale
    assert U.u1_violation(z, U.u1_result_legs(lx, ly, ax, ay), qx + qy) <= 1e-12 * scale
    ctx.synchronize()
