"""Failure detection without a GPU fault.

* Bounded device waits: ftn_ctx_wait_selftest launches one kernel whose
  mbarrier wait (the same bounded-wait code as the tensor-core GEMM and the
  staged permute) can never complete; it gives up after a short limit, the
  next ftn_ctx_synchronize reports FTN_ETIMEOUT, and the context stays usable.
* Allocator failure: a context whose allocator callback returns NULL on
  demand reports FTN_ENOMEM from tensor creation and from a contraction, and
  works again (with correct results) once the allocator recovers.
"""
import ctypes as C
import time
import weakref

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


def _t3(F, ctx):
    case = W.tensordot_case("T3", seed=2)
    ba = W.random_blocks(case["legs_a"], 0, case["seed_a"])
    bb = W.random_blocks(case["legs_b"], 0, case["seed_b"])
    ref = O.transpose(O.contract(O.embed_blocks(case["legs_a"], 0, ba), O.embed_blocks(case["legs_b"], 0, bb),
                                 case["axes_a"], case["axes_b"]), case["out_perm"])
    a = F.Tensor.from_blocks(ctx, case["legs_a"], 0, ba)
    b = F.Tensor.from_blocks(ctx, case["legs_b"], 0, bb)
    return case, a, b, ref


def _check_t3(F, ctx, case, a, b, ref, prec="f64"):
    c = F.tensordot(ctx, a, b, case["axes_a"], case["axes_b"], out_perm=case["out_perm"], prec=prec)
    got = O.embed_blocks(c.legs, c.parity, c.to_blocks())
    assert np.max(np.abs(got.data - ref.data)) <= 1e-10 * np.max(np.abs(ref.data))


def test_bounded_wait_timeout_is_reported(F):
    ctx = F.Context()
    case, a, b, ref = _t3(F, ctx)
    ctx.synchronize()
    t0 = time.perf_counter()
    ctx.wait_selftest(2_000_000)  # 2 ms
    with pytest.raises(F.FtnError) as e:
        ctx.synchronize()
    assert e.value.status == -7 and "timed out" in str(e.value)
    assert time.perf_counter() - t0 < 5.0  # the kernel returned after its limit
    ctx.synchronize()  # the error word was cleared
    _check_t3(F, ctx, case, a, b, ref)  # the context still computes correctly
    ctx.synchronize()
    ctx.close()


def test_wait_selftest_argument_checks(F):
    ctx = F.Context()
    for bad in (0, 999, 10_000_000_001):
        with pytest.raises(F.FtnError) as e:
            ctx.wait_selftest(bad)
        assert e.value.status == -1
    ctx.synchronize()
    ctx.close()


def _failing_context(F, torch, state):
    """A Context whose allocator callback returns NULL while state['fail']."""
    dev, st = torch.cuda.current_device(), torch.cuda.current_stream()

    def _alloc(nbytes, user):
        if state["fail"]:
            state["refused"] += 1
            return None
        return torch.cuda.caching_allocator_alloc(int(nbytes), dev, st)

    def _free(ptr, user):
        if ptr:
            torch.cuda.caching_allocator_delete(ptr)

    ctx = F.Context.__new__(F.Context)
    ctx._torch, ctx.device, ctx.stream = torch, dev, st
    a, f = F.ALLOC_FN(_alloc), F.FREE_FN(_free)
    ctx._keep = [a, f]
    h = C.c_void_p()
    assert F.lib().ftn_ctx_create(C.c_void_p(st.cuda_stream), a, f, None, C.byref(h)) == 0
    ctx.handle = h
    ctx._tensors = weakref.WeakSet()
    return ctx


def test_allocator_failure_reports_enomem(F):
    import torch

    state = {"fail": False, "refused": 0}
    ctx = _failing_context(F, torch, state)
    case, a, b, ref = _t3(F, ctx)
    state["fail"] = True
    with pytest.raises(F.FtnError) as e:
        F.Tensor.empty(ctx, case["legs_a"], 0)
    assert e.value.status == -5
    with pytest.raises(F.FtnError) as e:
        F.tensordot(ctx, a, b, case["axes_a"], case["axes_b"], out_perm=case["out_perm"], prec="f64")
    assert e.value.status == -5
    assert state["refused"] >= 2
    state["fail"] = False
    ctx.synchronize()
    _check_t3(F, ctx, case, a, b, ref)
    ctx.synchronize()
    ctx.close()
