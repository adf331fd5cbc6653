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
    # a contraction with wide, long sector GEMMs (tiled kernels) and one with
    # small sector problems of short K (warp kernels)
    la = [(40, 24, 0), (6, 2, 1), (3, 5, 0), (70, 66, 1)]
    lb = [(70, 66, 0), (6, 2, 0), (30, 34, 0)]
    sa = [(3, 2, 0), (2, 2, 1), (4, 3, 0)]
    sb = [(2, 2, 0), (3, 4, 1)]
    cases = [
        (F.Tensor.from_blocks(ctx, la, 0, W.random_blocks(la, 0, 3), dt),
         F.Tensor.from_blocks(ctx, lb, 1, W.random_blocks(lb, 1, 4), dt), [3, 1], [0, 1]),
        (F.Tensor.from_blocks(ctx, sa, 1, W.random_blocks(sa, 1, 5), dt),
         F.Tensor.from_blocks(ctx, sb, 0, W.random_blocks(sb, 0, 6), dt), [1], [0]),
    ]

    def step(outs=None):
        return [F.tensordot(ctx, a, b, xa, xb, prec=prec, out=None if outs is None else outs[i])
                for i, (a, b, xa, xb) in enumerate(cases)]

    want = [r.view().clone() for r in step()]
    outs = step()  # the buffers the graph writes
    old = ctx.stream
    side = torch.cuda.Stream()
    side.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(side):
        ctx.set_stream(side)
        step(outs)
    torch.cuda.current_stream().wait_stream(side)
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g):
        ctx.set_stream(torch.cuda.current_stream())
        step(outs)
    ctx.set_stream(old)
    for o in outs:
        o.view().zero_()
    g.replay()
    torch.cuda.synchronize()
    assert all(torch.equal(o.view(), w) for o, w in zip(outs, want))
    # eager calls after the capture (cache in use again) still give the same
    # results, and replaying again after them does too
    for _ in range(3):
        again = step()
        assert all(torch.equal(r.view(), w) for r, w in zip(again, want))
        del again
    for o in outs:
        o.view().zero_()
    g.replay()
    torch.cuda.synchronize()
    assert all(torch.equal(o.view(), w) for o, w in zip(outs, want))
    del g
    ctx.synchronize()
    ctx.close()
    assert all(np.isfinite(w.cpu().numpy()).all() for w in want)
