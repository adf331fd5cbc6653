"""Energy reduction behind the C ABI and the split of the energy networks
across ranks, on the CPU (no GPU: ftn_energy_reduce is host arithmetic, and
the per-network values come from the oracle).

* ftn_energy_reduce against its definition <h_t> = value(num) / value(den)
  with value = mantissa * exp(log_scale), group sums in term order, and its
  argument checks.
* World size 2 over gloo: each rank contracts the strided half of the
  networks of a 2x2 Hubbard energy with the oracle, the values are
  all-reduced, and both ranks' energies equal the one-process result bit for
  bit (and the oracle's own energy to rounding).
"""
import math
import socket

import pytest

import oracle as O
import workloads as W


def _lib():
    from paper_2410_02215_gb300 import build, ftn

    build.build()
    ftn.lib()
    return ftn


def test_energy_reduce_definition():
    ftn = _lib()
    vals = [(2.0, 0.5), (-3.0, 1.25), (0.75, -2.0), (1.5, 0.0), (4.0, 3.0)]
    num, den, ge = [1, 2, 3, 4], [0, 0, 4, 4], [2, 4]
    en, rat = ftn.energy_reduce(vals, num, den, ge)
    want = [vals[a][0] / vals[b][0] * math.exp(vals[a][1] - vals[b][1]) for a, b in zip(num, den)]
    assert rat == want
    assert en == [want[0] + want[1], want[2] + want[3]]
    en, _ = ftn.energy_reduce(vals, num, den, [1, 1, 4])  # an empty group
    assert en == [want[0], 0.0, want[1] + want[2] + want[3]]


@pytest.mark.parametrize("bad", ["index", "zero", "groups"])
def test_energy_reduce_errors(bad):
    ftn = _lib()
    vals = [(2.0, 0.5), (0.0, 0.0), (1.0, 0.0)]
    num, den, ge = [0], [2], [1]
    if bad == "index":
        num = [3]
    elif bad == "zero":
        den = [1]
    else:
        ge = [2]
    with pytest.raises(ftn.FtnError) as e:
        ftn.energy_reduce(vals, num, den, ge)
    assert e.value.status == -1


def _hubbard_networks():
    n, edges = W.square_lattice(2, 2)
    lay = W.peps_layout(n, edges, (1, 1), (2, 2))
    kets = O.ket_tensors(lay, W.random_peps(lay, 3))
    st = W.site_sweep_tree(list(range(n)))
    tf = lambda ops: W.double_layer_tree(n, st, ops)  # noqa: E731
    nets = [(O.norm_network(lay, kets), tf(()))]
    hop, on = O.hop_gate(1.0), O.onsite_gate(8.0)
    nets += [(O.term_network(lay, kets, hop, (a, b)), tf((a, b))) for a, b in lay["edges"]]
    nets += [(O.term_network(lay, kets, on, (s,)), tf((s,))) for s in range(n)]
    nt = len(nets) - 1
    ref = O.energy_terms(lay, kets, 1.0, 8.0, tf)[0]
    return nets, list(range(1, nt + 1)), [0] * nt, [nt], ref


def _oracle_values(nets):
    out = []
    for net, tree in nets:
        t, lg, _ = O.contract_tree(net, tree, normalize=True)
        out.append((float(t.data), float(lg)))
    return out


def _rank_main(rank, world, port, q):
    import torch.distributed as dist

    from paper_2410_02215_gb300 import dist as D

    try:
        dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank, world_size=world)
        nets, num, den, ge, _ = _hubbard_networks()
        got = []
        en, rat = D.energy_sharded(nets, num, den, ge, rank, world, lambda sub: got.extend(sub) or _oracle_values(sub))
        dist.barrier()
        dist.destroy_process_group()
        q.put((rank, en, rat, len(got)))
    except BaseException as e:  # reported to the parent
        q.put((rank, repr(e), None, None))


def test_energy_split_across_two_gloo_ranks():
    import multiprocessing as mp

    _lib()
    nets, num, den, ge, ref = _hubbard_networks()
    from paper_2410_02215_gb300 import dist as D

    one, one_r = D.energy_sharded(nets, num, den, ge, 0, 1, _oracle_values)
    assert abs(one[0] - ref) <= 1e-12 * abs(ref)
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        port = s.getsockname()[1]
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = [q.get(timeout=300) for _ in procs]
    for p in procs:
        p.join(timeout=60)
    counts = 0
    for rank, en, rat, n_local in sorted(res, key=lambda r: r[0]):
        assert rat is not None, en
        assert en == one and rat == one_r  # bit for bit
        counts += n_local
    assert counts == len(nets)  # every network contracted exactly once
