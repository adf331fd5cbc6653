"""A batch of networks captured into a CUDA graph (ftn_contract_batch_async
under stream capture): the replayed graph writes exactly (bit for bit) what
ftn_contract_batch returns, in FP64 and F16X3, replay after replay; it reads
the networks' tensors at replay (a tensor changed in place changes the
values as ftn_contract_batch sees them); and the two things a capture cannot
hold -- building a contraction's plan, running a compression (its kept
dimensions are read back to the host) -- are refused with FTN_EUNSUPPORTED,
leaving the context usable."""
import numpy as np
import pytest

from test_batch_gpu import cluster_nets

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def F():
    import torch

    from paper_2410_02215_gb300 import ftn

    assert torch.cuda.is_available()
    ftn.lib()
    return ftn


def pairs(d, n):
    h = d.cpu().numpy()
    return [(float(h[2 * i]), float(h[2 * i + 1])) for i in range(n)]


@pytest.mark.parametrize("prec", ["f64", "f16x3"])
def test_captured_batch_replays_bit_identical(F, prec):
    import torch

    s = torch.cuda.Stream()
    c = F.Context(stream=s)
    try:
        dt = F.F64 if prec == "f64" else F.F32
        nets, keep = cluster_nets(F, c, 16, (2, 1), 3, 1, "exact", 0, dt, limit=12)
        ref = F.contract_batch(c, nets, prec)
        d_out = torch.zeros(2 * len(nets), dtype=torch.float64, device="cuda")
        F.contract_batch_async(c, nets, d_out, prec)  # not captured: also builds every plan
        c.synchronize()
        assert pairs(d_out, len(nets)) == ref
        g = torch.cuda.CUDAGraph()
        d2 = torch.zeros_like(d_out)
        with torch.cuda.graph(g, stream=s):
            F.contract_batch_async(c, nets, d2, prec)
        for _ in range(3):
            d2.zero_()
            g.replay()
            torch.cuda.synchronize()
            assert pairs(d2, len(nets)) == ref
        # the graph reads the tensors at replay: double one ket in place
        keep[0][0].view().mul_(2.0)
        torch.cuda.synchronize()
        ref2 = F.contract_batch(c, nets, prec)
        assert ref2 != ref
        g.replay()
        torch.cuda.synchronize()
        assert pairs(d2, len(nets)) == ref2
        del g
    finally:
        c.synchronize()
        c.close()


def test_capture_refuses_plan_building_and_compression(F):
    import torch

    s = torch.cuda.Stream()
    c = F.Context(stream=s)
    try:
        nets, keep = cluster_nets(F, c, 16, (2, 1), 3, 1, "exact", 0, F.F64, limit=2)
        d = torch.zeros(2 * len(nets), dtype=torch.float64, device="cuda")
        # no plan exists yet on this context
        with pytest.raises(F.FtnError) as e:
            with torch.cuda.graph(torch.cuda.CUDAGraph(), stream=s):
                F.contract_batch_async(c, nets, d, "f64")
        assert e.value.status == -8
        # bonds of 36 states above chi = 8: compressions, refused under capture
        nets2, keep2 = cluster_nets(F, c, 16, (4, 2), 5, 1, "late", 8, F.F64, limit=2)
        ref2 = F.contract_batch(c, nets2, "f64")  # builds the plans
        d2 = torch.zeros(2 * len(nets2), dtype=torch.float64, device="cuda")
        with pytest.raises(F.FtnError) as e:
            with torch.cuda.graph(torch.cuda.CUDAGraph(), stream=s):
                F.contract_batch_async(c, nets2, d2, "f64")
        assert e.value.status == -8
        # the context is still usable, uncaptured
        F.contract_batch_async(c, nets2, d2, "f64")
        c.synchronize()
        assert pairs(d2, len(nets2)) == ref2
        assert np.isfinite(np.array(F.contract_batch(c, nets, "f64"))).all()
    finally:
        c.synchronize()
        c.close()
