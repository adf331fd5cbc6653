"""Parity of ftn_contract (tree executor), ftn_hubbard_term and the PEPS
energy path with the oracle.

The 2x2 norm is the exact small case: open 2x2 square lattice, physical
dimension 4 (even {0, updown}, odd {up, down}), bond D = 2 (1 + 1), N(0,1)
entries, even site tensors, contracted in two orders and in both
formalisms.  Tolerances: FP64 1e-10 relative; TF32x3 1e-5 relative.
"""
import math

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


def setup(lx, ly, D, seed):
    n, edges = W.square_lattice(lx, ly)
    lay = W.peps_layout(n, edges, D, (2, 2))
    blocks = W.random_peps(lay, seed)
    return n, edges, lay, blocks


def gpu_kets(F, ctx, lay, blocks, dt):
    return [F.Tensor.from_blocks(ctx, lay["legs"][s], 0, blocks[s], dt) for s in range(lay["n"])]


@pytest.mark.parametrize("prec", ["f64", "tf32x3", "f16x3"])
def test_norm_2x2_orders_and_formalisms(F, ctx, prec):
    from paper_2410_02215_gb300 import peps

    n, edges, lay, blocks = setup(2, 2, (1, 1), 0)
    kets_o = O.ket_tensors(lay, blocks)
    bf = O.brute_force_global(O.norm_network(lay, kets_o))
    dt = F.F64 if prec == "f64" else F.F32
    kets = gpu_kets(F, ctx, lay, blocks, dt)
    tens, bonds, pos = peps.norm_network(ctx, lay, kets)
    tol = 1e-10 if prec == "f64" else 1e-5
    trees = [W.double_layer_tree(n, W.site_sweep_tree(o)) for o in ([0, 1, 2, 3], [0, 2, 1, 3])]
    trees += [W.connected_random_tree(2 * n, [(b[0], b[2]) for b in bonds], s) for s in range(6)]
    for tree in trees:
        for glob in (False, True):
            m, lg = F.contract(ctx, tens, bonds, tree, positions=pos if glob else None, prec=prec)
            val = m * math.exp(lg)
            assert abs(val - bf) <= tol * abs(bf), (tree, glob, val, bf)


def test_hubbard_term_tensors_match_fock_space(F, ctx):
    hop = F.hubbard_term(ctx, 0, 1.3, 0.0)
    on = F.hubbard_term(ctx, 1, 0.0, 4.5)
    ref_h = O.hop_gate(1.3)
    ref_u = O.onsite_gate(4.5)
    assert hop.legs == ref_h.legs and on.legs == ref_u.legs
    assert np.array_equal(O.embed_blocks(hop.legs, 0, hop.to_blocks()).data, ref_h.data)
    assert np.array_equal(O.embed_blocks(on.legs, 0, on.to_blocks()).data, ref_u.data)


@pytest.mark.parametrize("mode", ["local", "global"])
@pytest.mark.parametrize("D,seed", [((1, 1), 0), ((2, 1), 3)])
def test_energy_2x2_matches_exact_diagonalisation(F, ctx, mode, D, seed):
    from paper_2410_02215_gb300 import peps

    n, edges, lay, blocks = setup(2, 2, D, seed)
    kets_o = O.ket_tensors(lay, blocks)
    e_ed = O.ed_energy(O.ket_amplitudes(lay, kets_o), n, edges, 1.0, 8.0)
    kets = gpu_kets(F, ctx, lay, blocks, F.F64)
    st = W.site_sweep_tree([0, 1, 2, 3])
    e, nm, nl = peps.energy(ctx, lay, kets, 1.0, 8.0, lambda ops: W.double_layer_tree(n, st, ops), mode=mode)
    assert abs(e - e_ed) <= 1e-10 * abs(e_ed)


@pytest.mark.parametrize("policy", ["late", "early"])
@pytest.mark.parametrize("mode", ["local", "global"])
@pytest.mark.parametrize("chi", [2, 4])
def test_approximate_norm_matches_oracle(F, ctx, policy, mode, chi):
    """Approximate contraction with compression: the same tree, policy and
    chi give the same truncations, hence the same value."""
    from paper_2410_02215_gb300 import peps

    n, edges, lay, blocks = setup(2, 3, (1, 1), 1)
    kets_o = O.ket_tensors(lay, blocks)
    net_o = O.norm_network(lay, kets_o)
    tree = W.double_layer_tree(n, W.site_sweep_tree(list(range(n))))
    r, lg_o, _ = O.contract_tree(net_o, tree, mode=mode, policy=policy, chi=chi, normalize=True)
    ref = float(r.data) * math.exp(lg_o)
    kets = gpu_kets(F, ctx, lay, blocks, F.F64)
    tens, bonds, pos = peps.norm_network(ctx, lay, kets)
    m, lg = F.contract(ctx, tens, bonds, tree, positions=pos if mode == "global" else None, policy=policy, chi=chi)
    assert abs(m * math.exp(lg) - ref) <= 1e-9 * abs(ref)


def test_approximate_energy_3x3_matches_oracle(F, ctx):
    from paper_2410_02215_gb300 import peps

    n, edges, lay, blocks = setup(3, 3, (1, 1), 2)
    kets_o = O.ket_tensors(lay, blocks)
    st = W.site_sweep_tree(list(range(n)))
    tf = lambda ops: W.double_layer_tree(n, st, ops)  # noqa: E731
    e_ref, *_ = O.energy_terms(lay, kets_o, 1.0, 8.0, tf, policy="late", chi=8)
    kets = gpu_kets(F, ctx, lay, blocks, F.F64)
    e, _, _ = peps.energy(ctx, lay, kets, 1.0, 8.0, tf, policy="late", chi=8)
    assert abs(e - e_ref) <= 1e-9 * abs(e_ref)


def test_energy_4x4_compressed_fp64_and_mixed(F, ctx):
    """The energy workload of the benchmark (4x4 square lattice, D = 4 as 2+2,
    chi = 32, late compression): FP64 GPU vs the oracle (1e-9), and the
    mixed paths (FP32 tensors, TF32x3 or F16X3 sector GEMMs, FP64
    compression) vs the FP64 GPU path (1e-6)."""
    from paper_2410_02215_gb300 import peps

    n, edges, lay, blocks = setup(4, 4, (2, 2), 1)
    st = W.site_sweep_tree(list(range(n)))
    tf = lambda ops: W.double_layer_tree(n, st, ops)  # noqa: E731
    e_ref, *_ = O.energy_terms(lay, O.ket_tensors(lay, blocks), 1.0, 8.0, tf, policy="late", chi=32)
    k64 = gpu_kets(F, ctx, lay, blocks, F.F64)
    e64, _, _ = peps.energy(ctx, lay, k64, 1.0, 8.0, tf, policy="late", chi=32)
    assert abs(e64 - e_ref) <= 1e-9 * abs(e_ref)
    k32 = gpu_kets(F, ctx, lay, blocks, F.F32)
    for prec in ("tf32x3", "f16x3"):
        e32, _, _ = peps.energy(ctx, lay, k32, 1.0, 8.0, tf, policy="late", chi=32, prec=prec)
        assert abs(e32 - e64) <= 1e-6 * abs(e64), prec


def test_energy_concurrent_streams_match_sequential(F, ctx):
    """The norm and the terms run concurrently on three contexts with their
    own streams: the same value, bit for bit, as one context."""
    import torch

    from paper_2410_02215_gb300 import peps

    n, edges, lay, blocks = setup(3, 3, (1, 1), 2)
    st = W.site_sweep_tree(list(range(n)))
    tf = lambda ops: W.double_layer_tree(n, st, ops)  # noqa: E731
    kets = gpu_kets(F, ctx, lay, blocks, F.F64)
    e1, nm1, nl1 = peps.energy(ctx, lay, kets, 1.0, 8.0, tf, policy="late", chi=8)
    extra = [F.Context(stream=torch.cuda.Stream()) for _ in range(2)]
    try:
        for _ in range(2):
            e3, nm3, nl3 = peps.energy([ctx] + extra, lay, kets, 1.0, 8.0, tf, policy="late", chi=8)
            assert (e3, nm3, nl3) == (e1, nm1, nl1)
    finally:
        for c in extra:
            c.synchronize()
            c.close()


@pytest.mark.parametrize("seed", range(6))
def test_local_formalism_with_odd_tensors(F, ctx, seed):
    """Odd tensors in the locally ordered formalism (dummy legs, Sec. II.D):
    the GPU value equals the oracle's, the brute-force global value and the
    GPU's globally ordered contraction with the tensors in index order."""
    from test_oracle_odd_local import rand_net, trees_of

    net, legs, blocks, odd = rand_net(seed)
    bf = O.brute_force_global(net)
    tens = [F.Tensor.from_blocks(ctx, legs[i], 1 if i in odd else 0, blocks[i]) for i in range(len(legs))]
    for tr in trees_of(net, 3):
        ref, _, _ = O.contract_tree(net, tr, mode="local")
        m, lg = F.contract(ctx, tens, net.bonds, tr)
        mg, lgg = F.contract(ctx, tens, net.bonds, tr, positions=list(range(len(legs))))
        v, vg = m * math.exp(lg), mg * math.exp(lgg)
        assert abs(v - float(ref.data)) <= 1e-10 * abs(bf), (seed, tr, v, float(ref.data))
        assert abs(v - bf) <= 1e-10 * abs(bf)
        assert abs(vg - bf) <= 1e-10 * abs(bf)
    t32 = [F.Tensor.from_blocks(ctx, legs[i], 1 if i in odd else 0, blocks[i], F.F32) for i in range(len(legs))]
    m, lg = F.contract(ctx, t32, net.bonds, trees_of(net, 1)[0], prec="f16x3")
    assert abs(m * math.exp(lg) - bf) <= 1e-5 * abs(bf)
