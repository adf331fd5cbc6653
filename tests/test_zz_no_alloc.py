"""ftn_tensordot_noalloc: the tensordot entry point for callers that cannot
allocate device memory (allocation-free stream capture, plug-in hosts with
pre-reserved buffers, latency-critical loops).  Its temporaries live in a
static device array inside libftn; the caller passes inputs and output.

Checked through the C ABI against the existing ftn_tensordot on the same
inputs, on two calls in a row (FP64, tolerance 1e-10 relative), plus the
clear rejection of a contraction too large for the static scratch.  Kept in
its own file, collected last.
"""
import ctypes as C

import numpy as np
import pytest

import workloads as W

pytestmark = pytest.mark.gpu


def _noalloc(F):
    L = F.lib()
    f = L.ftn_tensordot_noalloc
    i32p, u8p, ip = C.POINTER(C.c_int32), C.POINTER(C.c_uint8), C.POINTER(C.c_int)
    f.argtypes = [C.c_void_p, C.c_int, i32p, i32p, u8p, C.c_int, C.c_void_p, C.c_int, i32p, i32p, u8p, C.c_int,
                  C.c_void_p, C.c_int, C.c_int, ip, ip, ip, C.c_int, C.c_void_p, C.c_int64]
    f.restype = C.c_int
    return f


def _legs(legs):
    r = len(legs)
    return (r, (C.c_int32 * max(r, 1))(*[l[0] for l in legs]), (C.c_int32 * max(r, 1))(*[l[1] for l in legs]),
            (C.c_uint8 * max(r, 1))(*[l[2] for l in legs]))


def _call(F, f, case, a, b, out, stream):
    ra, a0, a1, ad = _legs(case["legs_a"])
    rb, b0, b1, bd = _legs(case["legs_b"])
    n = len(case["axes_a"])
    ax = (C.c_int * n)(*case["axes_a"])
    ay = (C.c_int * n)(*case["axes_b"])
    op = (C.c_int * len(case["out_perm"]))(*case["out_perm"])
    return f(C.c_void_p(stream.cuda_stream), ra, a0, a1, ad, 0, C.c_void_p(a.ptr), rb, b0, b1, bd, 0,
             C.c_void_p(b.ptr), F.F64, n, ax, ay, op, F.PREC_F64, C.c_void_p(out.data_ptr()), out.numel())


def test_noalloc_matches_tensordot_twice():
    import torch

    from paper_2410_02215_gb300 import ftn as F

    F.lib()
    f = _noalloc(F)
    ctx = F.Context()
    stream = torch.cuda.current_stream()
    for name, shrink in (("T2", 2), ("T3", 1)):
        case = W.tensordot_case(name, seed=4, shrink=shrink)
        ba = W.random_blocks(case["legs_a"], 0, case["seed_a"])
        bb = W.random_blocks(case["legs_b"], 0, case["seed_b"])
        a = F.Tensor.from_blocks(ctx, case["legs_a"], 0, ba)
        b = F.Tensor.from_blocks(ctx, case["legs_b"], 0, bb)
        ref = F.tensordot(ctx, a, b, case["axes_a"], case["axes_b"], out_perm=case["out_perm"], prec="f64")
        out = torch.full((ref.numel,), float("nan"), dtype=torch.float64, device="cuda")
        st = _call(F, f, case, a, b, out, stream)
        assert st == 0, F.lib().ftn_last_error().decode()
        torch.cuda.synchronize()
        want = ref.download()
        got = out.cpu().numpy()
        assert np.max(np.abs(got - want)) <= 1e-10 * np.max(np.abs(want))
    ctx.close()


def test_noalloc_rejects_oversized_problem():
    import torch

    from paper_2410_02215_gb300 import ftn as F

    f = _noalloc(F)
    ctx = F.Context()
    case = W.tensordot_case("T1", seed=0)  # environment of 8.4M FP64 entries: 67 MB of fused operand
    a = F.Tensor.empty(ctx, case["legs_a"], 0)
    b = F.Tensor.empty(ctx, case["legs_b"], 0)
    free = [l for k, l in enumerate(case["legs_a"]) if k not in case["axes_a"]]
    free += [l for k, l in enumerate(case["legs_b"]) if k not in case["axes_b"]]
    numel = F.Tensor.empty(ctx, [free[p] for p in case["out_perm"]], 0).numel
    out = torch.empty(numel, dtype=torch.float64, device="cuda")
    st = _call(F, f, case, a, b, out, torch.cuda.current_stream())
    assert st == -1
    msg = F.lib().ftn_last_error().decode()
    assert "scratch" in msg and "noalloc" in msg
    ctx.close()
