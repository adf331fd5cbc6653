"""A contraction captured into a CUDA graph on a context's stream and
replayed (the form the benchmark times): the replay writes the eager result
bit for bit, both for an FP64 plan (tiled and warp GEMM kernels) and a
split-precision one, and the context's device-block cache stays usable
around the capture (it is bypassed while the stream is captured, so no block
the graph refers to is handed out again)."""
import numpy as np
import pytest

import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def F():
    import torch

    from paper_2410_02215_gb300 import ftn

    assert torch.cuda.is_available()
    ftn.lib()
    return ftn


@pytest.mark.parametrize("prec", ["f64", "tf32x3"])
def test_capture_replay_matches_eager(F, prec):
    import torch

    ctx = F.Context()
    dt = F.F64 if prec == "f64" else F.F32
    # a wide sector GEMM (tiled kernel) and many small ones (warp kernel)
    la = [(40, 24, 0), (6, 2, 1), (3, 5, 0), (70, 66, 1)]
    lb = [(70, 66, 0), (6, 2, 0), (30, 34, 0)]
    a = F.Tensor.from_blocks(ctx, la, 0, W.random_blocks(la, 0, 3), dt)
    b = F.Tensor.from_blocks(ctx, lb, 1, W.random_blocks(lb, 1, 4), dt)
    ref = F.tensordot(ctx, a, b, [3, 1], [0, 1], prec=prec)
    want = ref.view().clone()
    out = F.tensordot(ctx, a, b, [3, 1], [0, 1], prec=prec)  # the buffer the graph writes
    old = ctx.stream
    side = torch.cuda.Stream()
    side.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(side):
        ctx.set_stream(side)
        F.tensordot(ctx, a, b, [3, 1], [0, 1], prec=prec, out=out)
    torch.cuda.current_stream().wait_stream(side)
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g):
        ctx.set_stream(torch.cuda.current_stream())
        F.tensordot(ctx, a, b, [3, 1], [0, 1], prec=prec, out=out)
    ctx.set_stream(old)
    out.view().zero_()
    g.replay()
    torch.cuda.synchronize()
    assert torch.equal(out.view(), want)
    # eager calls after the capture (cache in use again) still give the same result,
    # and replaying again after them does too
    for _ in range(3):
        again = F.tensordot(ctx, a, b, [3, 1], [0, 1], prec=prec)
        assert torch.equal(again.view(), want)
        del again
    out.view().zero_()
    g.replay()
    torch.cuda.synchronize()
    assert torch.equal(out.view(), want)
    del g
    ctx.synchronize()
    ctx.close()
    assert np.isfinite(want.cpu().numpy()).all()
