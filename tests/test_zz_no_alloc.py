"""ftn_tensordot_noalloc: the tensordot entry point for callers that cannot
allocate device memory (plug-in hosts that hand over only the buffers they
reserved up front, processes whose device memory belongs to another
framework's allocator).  Its temporaries live in a static device array inside
libftn; the caller passes inputs and output.

Checked through the C ABI against the existing ftn_tensordot on the same
inputs on two calls in a row (FP64, 1e-10 relative), against the oracle in
FP64 and on the tensor-core path (TF32x3, F16X3: TMA tensor maps into the
static array, 1e-5), for two different contractions issued back to back on
one stream, and for the clear rejection of a contraction too large for the
array and of an output buffer one element short.  Kept in its own file,
collected last.
"""
import ctypes as C

import numpy as np
import pytest

import oracle as O
import workloads as W

pytestmark = pytest.mark.gpu

TOL = {"f64": 1e-10, "tf32x3": 1e-5, "f16x3": 1e-5}


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


def _call(F, f, case, a, b, out, stream, prec="f64", capacity=None):
    ra, a0, a1, ad = _legs(case["legs_a"])
    rb, b0, b1, bd = _legs(case["legs_b"])
    n = len(case["axes_a"])
    ax = (C.c_int * n)(*case["axes_a"])
    ay = (C.c_int * n)(*case["axes_b"])
    op = (C.c_int * len(case["out_perm"]))(*case["out_perm"])
    dt = F.F64 if prec == "f64" else F.F32
    cap = out.numel() if capacity is None else capacity
    return f(C.c_void_p(stream.cuda_stream), ra, a0, a1, ad, 0, C.c_void_p(a.ptr), rb, b0, b1, bd, 0,
             C.c_void_p(b.ptr), dt, n, ax, ay, op, F.PREC_NAMES[prec], C.c_void_p(out.data_ptr()), cap)


def _inputs(F, ctx, name, shrink, prec="f64", seed=4):
    case = W.tensordot_case(name, seed=seed, shrink=shrink)
    ba = W.random_blocks(case["legs_a"], 0, case["seed_a"])
    bb = W.random_blocks(case["legs_b"], 0, case["seed_b"])
    dt = F.F64 if prec == "f64" else F.F32
    a = F.Tensor.from_blocks(ctx, case["legs_a"], 0, ba, dt)
    b = F.Tensor.from_blocks(ctx, case["legs_b"], 0, bb, dt)
    return case, ba, bb, a, b


def _oracle_packed(case, ba, bb, like):
    """The oracle's permuted contraction packed in the block layout of the
    library tensor ``like`` (same legs)."""
    ref = O.transpose(O.contract(O.embed_blocks(case["legs_a"], 0, ba), O.embed_blocks(case["legs_b"], 0, bb),
                                 case["axes_a"], case["axes_b"]), case["out_perm"])
    assert like.legs == ref.legs
    blocks = O.extract_blocks(ref)
    flat = np.zeros(like.numel, dtype=np.float64)
    for m, off in like.block_table():
        blk = blocks[like.bits_of(m)]
        flat[off:off + blk.size] = blk.reshape(-1)
    return flat


def _relerr(got, want):
    return float(np.max(np.abs(got - want)) / np.max(np.abs(want)))


def test_noalloc_matches_tensordot_twice():
    import torch

    from paper_2410_02215_gb300 import ftn as F

    F.lib()
    f = _noalloc(F)
    ctx = F.Context()
    stream = torch.cuda.current_stream()
    for name, shrink in (("T2", 2), ("T3", 1)):
        case, _, _, a, b = _inputs(F, ctx, name, shrink)
        ref = F.tensordot(ctx, a, b, case["axes_a"], case["axes_b"], out_perm=case["out_perm"], prec="f64")
        out = torch.full((ref.numel,), float("nan"), dtype=torch.float64, device="cuda")
        st = _call(F, f, case, a, b, out, stream)
        assert st == 0, F.lib().ftn_last_error().decode()
        torch.cuda.synchronize()
        want = ref.download()
        got = out.cpu().numpy()
        assert np.max(np.abs(got - want)) <= 1e-10 * np.max(np.abs(want))
    ctx.close()


@pytest.mark.parametrize("prec", ["f64", "tf32x3", "f16x3"])
def test_noalloc_against_oracle_back_to_back(prec):
    """Two different contractions (T1 and T4 at reduced size; on the tensor
    cores their operands are read through TMA maps into the static array)
    issued back to back on one stream without a host synchronisation in
    between, both checked against the oracle afterwards."""
    import torch

    from paper_2410_02215_gb300 import ftn as F

    f = _noalloc(F)
    ctx = F.Context()
    stream = torch.cuda.current_stream()
    tdt = torch.float64 if prec == "f64" else torch.float32
    runs = []
    for name, shrink in (("T1", 2), ("T4", 4)):
        case, ba, bb, a, b = _inputs(F, ctx, name, shrink, prec, seed=6)
        like = F.Tensor.empty(ctx, F._result_legs(case["legs_a"], case["legs_b"], case["axes_a"], case["axes_b"],
                                                  case["out_perm"]), 0)
        out = torch.full((like.numel,), float("nan"), dtype=tdt, device="cuda")
        runs.append((case, ba, bb, a, b, like, out))
    for case, _, _, a, b, _, out in runs:
        st = _call(F, f, case, a, b, out, stream, prec)
        assert st == 0, F.lib().ftn_last_error().decode()
    torch.cuda.synchronize()
    for case, ba, bb, _, _, like, out in runs:
        want = _oracle_packed(case, ba, bb, like)
        got = out.cpu().numpy().astype(np.float64)
        assert _relerr(got, want) <= TOL[prec], (case["name"], _relerr(got, want))
    ctx.close()


def test_noalloc_rejects_short_output():
    import torch

    from paper_2410_02215_gb300 import ftn as F

    f = _noalloc(F)
    ctx = F.Context()
    case, _, _, a, b = _inputs(F, ctx, "T3", 1)
    like = F.Tensor.empty(ctx, F._result_legs(case["legs_a"], case["legs_b"], case["axes_a"], case["axes_b"],
                                              case["out_perm"]), 0)
    out = torch.zeros(like.numel, dtype=torch.float64, device="cuda")
    st = _call(F, f, case, a, b, out, torch.cuda.current_stream(), capacity=like.numel - 1)
    assert st == -1
    assert "output buffer" in F.lib().ftn_last_error().decode()
    assert torch.count_nonzero(out).item() == 0  # nothing written
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
