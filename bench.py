#!/usr/bin/env python
"""Benchmark of the fermionic tensordot hot path on GB300; prints ONE JSON line.

Workload (one step): the single-tensordot microbenchmark family T1-T4 --
two rank-5 Z2 site tensors (four virtual legs D = 8 split 4+4, physical leg
4 split 2+2) and rank-6 boundary environments (chi = 64 split 32+32),
contracting 2-3 legs, every input stored in a seeded random leg order and
every result permuted to a seeded random leg order; only parity-allowed
blocks are stored.  Each tensordot = one sign-permute launch of both inputs
into the fused sector-matrix layout + one grouped sector GEMM whose epilogue
writes the result straight into its permuted block layout (a separate output
sign-permute only where the destination's fastest legs are too short for
that), all in libftn's CUDA kernels.  The step is timed as a CUDA graph of
these launches when its replay reproduces the eager step bit for bit.

Metric: sector-GEMM TFLOP/s (the flops of the Z2-sector GEMMs, 2*M*N*K per
block pair, over the time of the whole step).  The default arithmetic is
F16X3 (FP16 hi/lo split products on the tcgen05 tensor cores, accumulated in
FP32); the other precisions, the plain-FP64 path and their errors against
the FP64 CPU oracle are reported beside it.  The second half of the metric,
fPEPS energy evaluations per second, is reported under "energy" (4x4 square
lattice, whole network), "energy_diamond" (the 64-site diamond by the
cluster approximation) and "cluster" (energy terms per second over 64
random 3-regular graphs), FP64 and mixed precision.

``--impl reference`` times the CPU oracle (the reference arm of this
method: no other implementation exists) on the same metric and workload.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import workloads as W  # noqa: E402

CASES = ["T1", "T2", "T3", "T4"]
PREC_DTYPE = {"f64": "f64", "tf32": "tf32", "bf16": "bf16", "tf32x3": "tf32x3", "bf16x3": "bf16x3", "f16x3": "f16x3"}
WORKLOAD = ("fermionic tensordot microbenchmark T1-T4: rank-5 Z2 site tensors (D=8 as 4+4, phys 4 as 2+2), "
            "rank-6 environments (chi=64 as 32+32); T1 E.A over 2 D legs, T2 E.A over 3 D legs, "
            "T3 A.B over 2 D legs, T4 E.E' over (chi,D,D); random stored and output leg orders")
NOMINAL_TF32_OVER_BF16 = 1.1 / 2.25  # dense tensor-core ratio (nominal)


def sector_flops(case):
    """2*M*N*K summed over the (row block, column block) pairs of the case."""
    la, lb, ax, ay = case["legs_a"], case["legs_b"], case["axes_a"], case["axes_b"]
    fa = [k for k in range(len(la)) if k not in ax]
    fb = [k for k in range(len(lb)) if k not in ay]

    def sectors(legs):
        out = {0: 0, 1: 0}
        for m in range(1 << len(legs)):
            size, par = 1, 0
            for i, l in enumerate(legs):
                b = (m >> i) & 1
                size *= l[1] if b else l[0]
                par ^= b
            out[par] += size
        return out

    rows = sectors([la[k] for k in fa])
    cols = sectors([lb[k] for k in fb])
    ks = sectors([la[k] for k in ax])
    tot = 0
    for pi in (0, 1):
        tot += 2 * rows[case["parity_a"] ^ pi] * cols[case["parity_b"] ^ pi] * ks[pi]
    return float(tot)


def load_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        return {"hbm_gbs": float(d["hbm_gbs"]), "bf16_tflops": float(d["bf16_tflops"]),
                "bf16_tflops_sustained": float(d.get("bf16_tflops_sustained", d["bf16_tflops"])), "src": "measured"}
    return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0, "src": "fallback"}


class ClockSampler:
    """nvidia-smi clock / throttle-reason samples during the timed region."""

    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
              "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
              "clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.path = None

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        time.sleep(0.25)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        rows = []
        for line in open(self.path):
            parts = [x.strip() for x in line.split(",")]
            if len(parts) < 8:
                continue
            try:
                rows.append((float(parts[0]), float(parts[1]), parts[4:8]))
            except ValueError:
                continue
        os.unlink(self.path)
        if not rows:
            return None
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for _, _, flags in rows for i, f in enumerate(flags) if f.lower() == "active"})
        return {"sm_mhz": statistics.median(r[0] for r in rows), "sm_max_mhz": max(r[1] for r in rows),
                "reasons": reasons, "samples": len(rows)}


def dist_init():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch
        import torch.distributed as dist

        if torch.cuda.is_available():
            torch.cuda.set_device(local)
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    return rank, world, local


def barrier(world):
    if world > 1:
        import torch.distributed as dist

        dist.barrier()


def max_over_ranks(x, world):
    if world == 1:
        return x
    import torch
    import torch.distributed as dist

    t = torch.tensor([x], dtype=torch.float64, device="cuda" if torch.cuda.is_available() else "cpu")
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


# ---------------------------------------------------------------------------------
def oracle_pass(cases, budget_s=None):
    """Run the CPU oracle on the cases; returns (flops done, seconds)."""
    import oracle as O

    done, t_tot = 0.0, 0.0
    for c in cases:
        a = O.embed_blocks(c["legs_a"], 0, W.random_blocks(c["legs_a"], 0, c["seed_a"]))
        b = O.embed_blocks(c["legs_b"], 0, W.random_blocks(c["legs_b"], 0, c["seed_b"]))
        t0 = time.perf_counter()
        r = O.transpose(O.contract(a, b, c["axes_a"], c["axes_b"]), c["out_perm"])
        t_tot += time.perf_counter() - t0
        done += sector_flops(c)
        del r
        if budget_s is not None and t_tot > budget_s:
            break
    return done, t_tot


def cpu_baseline(cases, budget_s=20.0):
    reps, flops, secs = 0, 0.0, 0.0
    while secs < budget_s * 0.5 and reps < 8:
        f, s = oracle_pass(cases)
        flops += f
        secs += s
        reps += 1
    out = {"value": flops / secs / 1e12, "unit": "TFLOP/s", "cores": len(os.sched_getaffinity(0)), "kind": "oracle",
           "sample": f"{reps} full oracle pass(es) over T1-T4 (dense FP64 numpy, data generation excluded), "
                     f"{secs:.1f} s"}
    one = single_thread_oracle([c["name"] for c in cases])
    if one is not None:
        out["single_thread"] = one
    return out


def single_thread_oracle(names, timeout=120):
    """The same oracle pass with one BLAS thread: a child process started with
    the thread-count variables of the common BLAS libraries set to 1 before
    numpy loads.  Returns {"value", "unit", "cores": 1, "sample"} or None."""
    import subprocess

    env = dict(os.environ)
    for k in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS", "BLIS_NUM_THREADS"):
        env[k] = "1"
    code = ("import json, sys; sys.path.insert(0, %r); import bench, workloads as W; "
            "cs = [W.tensordot_case(n, seed=0) for n in %r]; f, s = bench.oracle_pass(cs); "
            "print(json.dumps([f, s]))") % (os.path.dirname(os.path.abspath(__file__)), list(names))
    try:
        r = subprocess.run([sys.executable, "-c", code], env=env, capture_output=True, text=True, timeout=timeout)
        f, s = json.loads(r.stdout.strip().splitlines()[-1])
    except Exception:  # a missing or slow child only drops this figure
        return None
    return {"value": f / s / 1e12, "unit": "TFLOP/s", "cores": 1,
            "sample": f"one full oracle pass over {','.join(names)} with one BLAS thread, {s:.1f} s"}


def run_reference(args, rank, world):
    if rank != 0:
        return 0
    cases = [W.tensordot_case(n, seed=0) for n in CASES]
    for _ in range(args.warmup):
        oracle_pass(cases)
    times, flops = [], 0.0
    for _ in range(args.steps):
        f, s = oracle_pass(cases)
        times.append(s)
        flops = f
    tot = sum(times)
    val = flops * args.steps / tot / 1e12
    cores = len(os.sched_getaffinity(0))
    line = {
        "impl": "reference", "metric": "sector-GEMM TFLOP/s", "value": val, "unit": "TFLOP/s", "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * tot / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": WORKLOAD, "l2": "n/a (CPU)"},
        "cpu_baseline": {"value": val, "unit": "TFLOP/s", "cores": cores, "kind": "oracle",
                         "sample": "each step one full oracle pass over T1-T4 (dense FP64 numpy)"},
        "e2e": {"value": val, "unit": "TFLOP/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


# ---------------------------------------------------------------------------------
def make_inputs(F, ctx, torch, cases, prec, seed=0):
    dt = F.F64 if prec == "f64" else F.F32
    gen = torch.Generator(device="cuda")
    gen.manual_seed(seed)
    tens = {}
    for c in cases:
        for side in ("a", "b"):
            key = (tuple(c["legs_" + side]), side, c["name"])
            t = F.Tensor.empty(ctx, c["legs_" + side], 0, dt)
            v = t.view()
            v.copy_(torch.randn(v.shape, generator=gen, device="cuda", dtype=v.dtype))
            tens[key] = t
    return tens


def one_step(F, ctx, cases, ins, outs, prec, tag=False):
    for c in cases:
        if tag:
            ctx.profile_tag(c["name"])
        a = ins[(tuple(c["legs_a"]), "a", c["name"])]
        b = ins[(tuple(c["legs_b"]), "b", c["name"])]
        o = outs.get(c["name"])
        r = F.tensordot(ctx, a, b, c["axes_a"], c["axes_b"], out_perm=c["out_perm"], prec=prec, out=o)
        outs[c["name"]] = r


def copy_reference_ms(torch, traffic_bytes, flush, reps=10):
    """A plain device copy (torch's copy kernel) of traffic_bytes / 2 bytes,
    so traffic_bytes of reads and writes, L2 flushed before each: CUDA-event
    ms per copy, the mean of `reps` after two warm-up copies.  The size-matched
    scale for a sign-permute of the same algorithmic bytes (the measured HBM
    peak comes from a 2 GiB copy, whose fixed costs vanish)."""
    n = max(int(traffic_bytes) // 2, 1)
    src = torch.ones(n, dtype=torch.uint8, device="cuda")
    dst = torch.empty_like(src)
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(reps)]
    for _ in range(2):
        dst.copy_(src)
    for a, b in ev:
        flush.zero_()
        a.record()
        dst.copy_(src)
        b.record()
    torch.cuda.synchronize()
    return sum(a.elapsed_time(b) for a, b in ev) / reps


def time_steps(F, ctx, torch, cases, prec, steps, warmup, flush, world, profile=False, graph=False):
    """Times `steps` steps (L2 flushed before each, outside the events).
    Eager: one library call per contraction per step.  profile=True adds a
    second eager pass with per-launch CUDA events (ftn_ctx_profile) for the
    roofline; graph=True adds a pass that replays the step captured once as a
    CUDA graph (the same kernels with the same arguments), checked bit for bit
    against the eager outputs.  Returns (ms eager, launches per step, profile,
    inputs, outputs, graph info)."""
    ins = make_inputs(F, ctx, torch, cases, prec)
    outs = {}
    for _ in range(warmup):
        one_step(F, ctx, cases, ins, outs, prec)
    torch.cuda.synchronize()

    def timed(run):
        evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
        barrier(world)
        torch.cuda.synchronize()
        for i in range(steps):
            flush.zero_()
            evs[i][0].record()
            run()
            evs[i][1].record()
        torch.cuda.synchronize()
        barrier(world)
        return sum(a.elapsed_time(b) for a, b in evs)

    l0 = ctx.launches()
    ms = timed(lambda: one_step(F, ctx, cases, ins, outs, prec))
    launches = (ctx.launches() - l0) // max(steps, 1)
    prof = None
    if profile:
        ctx.profile(True)
        timed(lambda: one_step(F, ctx, cases, ins, outs, prec, tag=True))
        prof = ctx.profile_read()
        ctx.profile(False)
        ctx.profile_tag("")
    ginfo = None
    if graph:
        ginfo = graph_steps(F, ctx, torch, cases, ins, outs, prec, timed)
    ctx.synchronize()
    return ms, launches, prof, ins, outs, ginfo


def graph_steps(F, ctx, torch, cases, ins, outs, prec, timed):
    """The step captured once as a CUDA graph on the context's stream and
    replayed; the outputs of a replay must equal the eager step's bit for
    bit.  Returns {"ms", "launches_per_step", "identical"} or {"error"}."""
    ref = {k: v.view().clone() for k, v in outs.items()}
    old = ctx.stream
    g = torch.cuda.CUDAGraph()
    try:
        side = torch.cuda.Stream()
        side.wait_stream(torch.cuda.current_stream())
        with torch.cuda.stream(side):  # one eager step on the side stream first (capture etiquette)
            ctx.set_stream(side)
            one_step(F, ctx, cases, ins, outs, prec)
        torch.cuda.current_stream().wait_stream(side)
        l0 = ctx.launches()
        with torch.cuda.graph(g):
            ctx.set_stream(torch.cuda.current_stream())
            one_step(F, ctx, cases, ins, outs, prec)
        n = ctx.launches() - l0
    except Exception as e:  # noqa: BLE001 -- reported, the eager number stands
        ctx.set_stream(old)
        return {"error": str(e)[:200]}
    ctx.set_stream(old)
    for v in outs.values():
        v.view().zero_()
    g.replay()
    torch.cuda.synchronize()
    same = all(torch.equal(outs[k].view(), ref[k]) for k in ref)
    ms = timed(g.replay)
    del g
    return {"ms": ms, "launches_per_step": n, "identical": bool(same)}


CLUSTER_WORKLOAD = ("Hubbard fPEPS energy terms by the cluster approximation (radius 1, Sec. V) on 64 random "
                    "3-regular graphs (pairing model, seeds 0..63), N uniform over even integers in [16, 48], D cycling "
                    "through 3 (2+1), 4 (3+1), 6 (4+2), phys 4 (2+2), t=1, U=8, N(0,1) site tensors, stand-in gauges "
                    "0.5^k per sector on dangling bonds, late compression chi=32; one term = the cluster network with "
                    "and without the operator")


def cluster_bench(F, ctx, torch, n_graphs, streams, with_oracle, batch=128):
    """Energy terms per second of the cluster approximation over a set of
    random regular graphs (FP64 and mixed), and the oracle's rate on the
    smallest graph of the set.  The two cluster networks of every term of
    every graph are contracted in lock-step batches of `batch` networks
    (ftn_contract_batch) spread over `streams` contexts; the first graphs are
    checked against one ftn_contract call per network."""
    import numpy as np

    from paper_2410_02215_gb300 import peps

    rg = np.random.default_rng(12345)
    Ds = [(2, 1), (3, 1), (4, 2)]
    graphs = []
    for g in range(n_graphs):
        n = int(rg.integers(8, 25)) * 2
        nn, e = W.random_regular_graph(n, 3, g)
        lay = W.peps_layout(nn, e, Ds[g % 3], (2, 2))
        graphs.append((lay, W.random_peps(lay, g), W.bond_gauges(lay)))

    def cfn(lay):
        # a term's cluster (sites, dangling bonds, trees) depends on the lattice
        # alone: computed once per lattice and term, as repeated evaluations of
        # one lattice would
        memo = {}

        def f(targets):
            key = tuple(targets)
            if key not in memo:
                sites = W.cluster_sites(lay, targets, 1)
                memo[key] = (sites, W.dangling_bonds(lay, sites), W.cluster_tree(lay, sites, targets, True),
                             W.cluster_tree(lay, sites, targets, False))
            return memo[key]
        return f

    ctxs = [ctx] + [F.Context(stream=torch.cuda.Stream()) for _ in range(max(streams, 1) - 1)]
    out = {"workload": CLUSTER_WORKLOAD, "graphs": n_graphs, "streams": len(ctxs),
           "timed": "one pass through peps.cluster_networks (bras, gauge tensors and network tables) and "
                    "ftn_energy, after an untimed pass; the clusters' structure computed once per lattice"}
    res = {}
    for prec, dt in (("f64", F.F64), ("tf32x3", F.F32), ("f16x3", F.F32)):
        kets = [[F.Tensor.from_blocks(ctx, lay["legs"][s], 0, bl[s], dt) for s in range(lay["n"])]
                for lay, bl, _ in graphs]
        ctx.synchronize()
        inst = [(lay, k, cfn(lay), gs) for (lay, _, gs), k in zip(graphs, kets)]
        # warm-up: one untimed pass of the whole workload, so that every
        # context has built the plans of the shapes it meets (steady state)
        peps.cluster_energies(ctxs, inst, 1.0, 8.0, policy="late", chi=32, prec=prec, batch=batch)
        one = peps.cluster_energies(ctx, inst[:3], 1.0, 8.0, policy="late", chi=32, prec=prec)  # per network
        ctx.synchronize()
        t0 = time.perf_counter()
        nets, num, den, ge, keep = peps.cluster_networks(ctx, inst, 1.0, 8.0, "late", 32, dt)
        t1 = time.perf_counter()
        en, rat, _ = F.energy(ctxs, nets, num, den, ge, prec, batch)
        dt_s = time.perf_counter() - t0
        del keep
        got, q0 = [], 0
        for g, q1 in enumerate(ge):
            got.append((en[g], rat[q0:q1]))
            q0 = q1
        nterms = len(rat)
        energies = [e for e, _ in got]
        res[prec] = energies
        out[prec] = {"terms_per_s": nterms / dt_s, "terms": nterms, "s": dt_s, "assembly_s": t1 - t0,
                     "contract_s": dt_s - (t1 - t0), "batch": batch, "same_as_unbatched": got[:3] == one,
                     "energy_graph0": energies[0]}
    e64 = np.array(res["f64"])
    for p in ("tf32x3", "f16x3"):
        out[p]["max_rel_err_vs_f64"] = float(np.max(np.abs(np.array(res[p]) - e64) / np.abs(e64)))
    out["mixed_vs_f64_max_rel_err"] = out["tf32x3"]["max_rel_err_vs_f64"]
    if with_oracle:
        import oracle as O

        small = min(range(n_graphs), key=lambda g: graphs[g][0]["n"] * (1 + g % 3))
        lay, bl, gs = graphs[small]
        t0 = time.perf_counter()
        e_ref, rref = O.cluster_energy(lay, O.ket_tensors(lay, bl), 1.0, 8.0, cfn(lay), gs, policy="late", chi=32)
        dt_s = time.perf_counter() - t0
        out["oracle"] = {"terms_per_s": len(rref) / dt_s, "graph_sites": lay["n"], "D": list(lay["legs"][0][0][:2]),
                         "energy_rel_err_f64_gpu": abs(res["f64"][small] - e_ref) / abs(e_ref)}
    for c in ctxs[1:]:
        c.synchronize()
        c.close()
    return out


def backward_bench(F, ctx, torch, cases, prec, steps, warmup, flush, ins, outs, flops_step):
    """The adjoint of the step: dA and dB of every T1-T4 contraction from a
    resident G (C's metadata), timed like the forward step.  Each gradient
    costs the forward's sector flops, so a backward step is 2x the forward's.
    Accuracy: normwise against the FP64 gradients of the same inputs (the
    FP64 adjoint is checked against the oracle's gradient by definition in
    the tests)."""
    gen = torch.Generator(device="cuda")
    gen.manual_seed(11)
    gs, da, db = {}, {}, {}
    for c in cases:
        r = outs[c["name"]]
        g = F.Tensor.empty(ctx, r.legs, r.parity, F.F64 if prec == "f64" else F.F32)
        v = g.view()
        v.copy_(torch.randn(v.shape, generator=gen, device="cuda", dtype=v.dtype))
        gs[c["name"]] = g

    def step():
        for c in cases:
            a = ins[(tuple(c["legs_a"]), "a", c["name"])]
            b = ins[(tuple(c["legs_b"]), "b", c["name"])]
            x, y = F.tensordot_grad(ctx, a, b, gs[c["name"]], c["axes_a"], c["axes_b"], out_perm=c["out_perm"],
                                    prec=prec, out_a=da.get(c["name"]), out_b=db.get(c["name"]))
            da[c["name"]], db[c["name"]] = x, y

    for _ in range(warmup):
        step()
    torch.cuda.synchronize()
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
    for i in range(steps):
        flush.zero_()
        evs[i][0].record()
        step()
        evs[i][1].record()
    torch.cuda.synchronize()
    ms = sum(a.elapsed_time(b) for a, b in evs) / steps
    worst = 0.0
    if prec != "f64":
        for c in cases:
            up = lambda t: F.Tensor.wrap(ctx, t.legs, t.parity, t.view().double().contiguous(), F.F64)  # noqa: E731
            a64 = up(ins[(tuple(c["legs_a"]), "a", c["name"])])
            b64 = up(ins[(tuple(c["legs_b"]), "b", c["name"])])
            g64 = up(gs[c["name"]])
            ra, rb = F.tensordot_grad(ctx, a64, b64, g64, c["axes_a"], c["axes_b"], out_perm=c["out_perm"],
                                      prec="f64")
            for got, ref in ((da[c["name"]], ra), (db[c["name"]], rb)):
                x, y = got.view().double(), ref.view()
                worst = max(worst, float((x - y).abs().max() / y.abs().max()))
            for t in (ra, rb, a64, b64, g64):
                t.free()
    return {"metric": "sector-GEMM TFLOP/s of the adjoint step (dA and dB of T1-T4)", "precision": prec,
            "ms_per_step": ms, "tflops": 2.0 * flops_step / (ms * 1e-3) / 1e12,
            "rel_err_inf_vs_f64_gpu": worst}


def accuracy(F, ctx, prec):
    """Normwise errors of one reduced-size step against the oracle (T1-T4
    with every sector dimension halved, T4 quartered)."""
    import numpy as np

    import oracle as O

    worst_inf, worst_2 = 0.0, 0.0
    for n in CASES:
        c = W.tensordot_case(n, seed=1, shrink=2 if n != "T4" else 4)
        ba = W.random_blocks(c["legs_a"], 0, c["seed_a"])
        bb = W.random_blocks(c["legs_b"], 0, c["seed_b"])
        ref = O.transpose(O.contract(O.embed_blocks(c["legs_a"], 0, ba), O.embed_blocks(c["legs_b"], 0, bb),
                                     c["axes_a"], c["axes_b"]), c["out_perm"]).data
        dt = F.F64 if prec == "f64" else F.F32
        a = F.Tensor.from_blocks(ctx, c["legs_a"], 0, ba, dt)
        b = F.Tensor.from_blocks(ctx, c["legs_b"], 0, bb, dt)
        r = F.tensordot(ctx, a, b, c["axes_a"], c["axes_b"], out_perm=c["out_perm"], prec=prec)
        got = O.embed_blocks(r.legs, r.parity, r.to_blocks()).data
        worst_inf = max(worst_inf, float(np.max(np.abs(got - ref)) / np.max(np.abs(ref))))
        worst_2 = max(worst_2, float(np.linalg.norm(got - ref) / np.linalg.norm(ref)))
    return {"rel_err_inf": worst_inf, "rel_err_2": worst_2}


def traffic_for(label, prec):
    """DRAM bytes per launch from a committed ncu summary (profiles/traffic.txt),
    when it was taken on the current kernel sources in this precision (else
    None)."""
    label = f"{label}@{prec}"
    p = os.path.join(ROOT, "profiles", "traffic.txt")
    if not os.path.exists(p):
        return None
    try:
        from paper_2410_02215_gb300 import build as B

        dig = B.kernel_digest()
        for line in open(p):
            parts = line.split()
            if len(parts) >= 3 and not line.startswith("#") and parts[0] == label and parts[1] == dig:
                return float(parts[2])
    except Exception:
        return None
    return None


def roofline(prof, peaks, prec="tf32x3"):
    """Roofline of the dominant kernel.  A tensor-core contraction takes the
    dense peak of its operand type (TF32: the measured bf16 burst x 1.1/2.25,
    the nominal ratio; BF16 and FP16: the measured bf16 burst).  The split modes run
    3 tensor-core products per algorithmic product, so beside `frac` the
    fraction of the peak / 3 is reported as `frac_of_split_peak`."""
    dom = max(prof, key=lambda r: r["ms"])
    label = dom["label"]
    kind = label.split("/")[-1]
    t_s = dom["ms"] / 1e3 / max(dom["launches"], 1)
    bytes_per = dom["bytes"] / max(dom["launches"], 1)
    flops_per = dom["flops"] / max(dom["launches"], 1)
    bf16 = prec.startswith("bf16") or prec.startswith("f16")  # 16-bit operands: the bf16 / fp16 rate
    tc_peak = peaks["bf16_tflops"] * (1.0 if bf16 else NOMINAL_TF32_OVER_BF16)
    passes = 3 if prec.endswith("x3") else 1
    out = {"kernel": label, "launches": dom["launches"], "avg_launch_ms": t_s * 1e3}
    # tensor-bound when the tensor work (passes x sector flops) per algorithmic byte exceeds the ridge
    tensor_bound = (kind == "gemm_tc" and
                    passes * flops_per / max(bytes_per, 1.0) > tc_peak * 1e12 / (peaks["hbm_gbs"] * 1e9))
    if tensor_bound:
        ach = flops_per / t_s / 1e12
        note = (f"BF16 / FP16 dense = {peaks['src']} bf16 burst" if bf16 else
                f"TF32 dense = {peaks['src']} bf16 burst x 1.1/2.25 (nominal ratio)")
        out.update({"bound": "tensor", "achieved": ach, "peak": tc_peak, "unit": "TFLOP/s", "frac": ach / tc_peak,
                    "peak_note": note})
        if passes > 1:
            out.update({"tensor_passes_per_product": passes, "frac_of_split_peak": ach * passes / tc_peak})
    else:
        ach = bytes_per / t_s / 1e9
        out.update({"bound": "hbm", "achieved": ach, "peak": peaks["hbm_gbs"], "unit": "GB/s",
                    "frac": ach / peaks["hbm_gbs"], "peak_note": f"{peaks['src']} HBM copy bandwidth"})
    out["algorithmic_bytes_per_launch"] = bytes_per
    out["algorithmic_flops_per_launch"] = flops_per
    out["traffic"] = traffic_for(label, prec)
    return out


def e2e_run(F, ctx, torch, cases, prec, steps, flops_step, lanes=3):
    """Same step through the C ABI with pinned host buffers: every step copies
    all its inputs host->device and all its results device->host inside the
    timed region.  Steps alternate between `lanes` contexts on their own
    streams (each with its own device and host buffers), so one step's
    uploads overlap the previous step's contractions and downloads -- the
    pipelining a caller streaming many inputs would use."""
    import ctypes as C

    npdt = torch.float64 if prec == "f64" else torch.float32
    lib = F.lib()
    ctxs = [ctx] + [F.Context(stream=torch.cuda.Stream()) for _ in range(max(lanes, 1) - 1)]
    lane = []
    for q, c in enumerate(ctxs):
        ins = make_inputs(F, c, torch, cases, prec, seed=5 + q)
        outs = {}
        one_step(F, c, cases, ins, outs, prec)  # plans and outputs of this context
        torch.cuda.synchronize()
        h_in = {k: torch.empty(t.numel, dtype=npdt, pin_memory=True) for k, t in ins.items()}
        for k, t in ins.items():
            h_in[k].copy_(t.view().cpu())
        h_out = {k: torch.empty(t.numel, dtype=npdt, pin_memory=True) for k, t in outs.items()}
        lane.append((c, ins, outs, h_in, h_out))
    c0, ins0, outs0 = lane[0][0], lane[0][1], lane[0][2]
    h2d = sum(t.numel * (8 if prec == "f64" else 4) for t in ins0.values())
    d2h = sum(t.numel * (8 if prec == "f64" else 4) for t in outs0.values())
    streams = [c.stream for c in ctxs]
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record(streams[0])
    for st in streams[1:]:
        st.wait_event(e0)
    for i in range(steps):
        c, ins, outs, h_in, h_out = lane[i % len(lane)]
        for k, t in ins.items():
            F._check(lib.ftn_tensor_upload(c.handle, t.handle, C.c_void_p(h_in[k].data_ptr())))
        one_step(F, c, cases, ins, outs, prec)
        for k, t in outs.items():
            F._check(lib.ftn_tensor_download(c.handle, t.handle, C.c_void_p(h_out[k].data_ptr())))
    for st in streams[1:]:
        ev = torch.cuda.Event()
        ev.record(st)
        streams[0].wait_event(ev)
    e1.record(streams[0])
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1)
    for c in ctxs[1:]:
        c.synchronize()
        c.close()
    return {"value": flops_step * steps / (ms / 1e3) / 1e12, "unit": "TFLOP/s", "h2d_bytes_per_step": int(h2d),
            "d2h_bytes_per_step": int(d2h), "ms_per_step": ms / steps, "lanes": len(ctxs),
            "note": "pinned host buffers; steps alternate between contexts on their own streams (copies of one "
                    "step overlap another step's contractions)"}


ENERGY_WORKLOAD = ("Hubbard fPEPS energy <H>/<Psi|Psi> on a 4x4 open square lattice, D=4 (2+2), phys 4 (2+2), "
                   "t=1, U=8, N(0,1) site tensors (seed 1), row-sweep double-layer tree, late compression chi=32: "
                   "24 hopping + 16 on-site terms + the norm = 41 contractions per evaluation")


def energy_bench(F, ctx, evals, with_oracle, workers=8, batches=(0, 2, 3, 6)):
    """fPEPS energy evaluations per second, FP64 and mixed (TF32x3 GEMMs with
    FP64 compression), and their errors.  The 41 contractions of an
    evaluation are independent: `workers` contexts on their own streams run
    them concurrently, either one contraction per ftn_contract call (batch 0)
    or in lock-step batches of a few networks (ftn_contract_batch); the
    batch size is picked by timing each candidate once after the warm-up.
    Every configuration gives the same value bit for bit."""
    import torch

    from paper_2410_02215_gb300 import peps

    ctxs = [ctx] + [F.Context(stream=torch.cuda.Stream()) for _ in range(max(workers, 1) - 1)]

    n, edges = W.square_lattice(4, 4)
    lay = W.peps_layout(n, edges, (2, 2), (2, 2))
    blocks = W.random_peps(lay, 1)
    st = W.site_sweep_tree(list(range(n)))
    tf = lambda ops: W.double_layer_tree(n, st, ops)  # noqa: E731
    out = {"workload": ENERGY_WORKLOAD, "streams": len(ctxs)}
    res = {}
    for prec, dt in (("f64", F.F64), ("tf32x3", F.F32), ("f16x3", F.F32)):
        kets = [F.Tensor.from_blocks(ctx, lay["legs"][s_], 0, blocks[s_], dt) for s_ in range(n)]
        ctx.synchronize()
        for c in ctxs:  # warm-up: every context builds its plans
            e, _, _ = peps.energy(c, lay, kets, 1.0, 8.0, tf, policy="late", chi=32, prec=prec)
        e1, _, _ = peps.energy(ctx, lay, kets, 1.0, 8.0, tf, policy="late", chi=32, prec=prec)
        t0 = time.perf_counter()
        e1, _, _ = peps.energy(ctx, lay, kets, 1.0, 8.0, tf, policy="late", chi=32, prec=prec)
        one_s = time.perf_counter() - t0
        trial = {}
        for b in batches:
            peps.energy(ctxs, lay, kets, 1.0, 8.0, tf, policy="late", chi=32, prec=prec, batch=b)
            t0 = time.perf_counter()
            eb, _, _ = peps.energy(ctxs, lay, kets, 1.0, 8.0, tf, policy="late", chi=32, prec=prec, batch=b)
            trial[b] = (time.perf_counter() - t0, eb == e1)
        best = min(trial, key=lambda b: trial[b][0])
        l0 = sum(c.launches() for c in ctxs)
        t0 = time.perf_counter()
        for _ in range(evals):
            e, _, _ = peps.energy(ctxs, lay, kets, 1.0, 8.0, tf, policy="late", chi=32, prec=prec, batch=best)
        dt_s = time.perf_counter() - t0
        res[prec] = e
        out[prec] = {"evals_per_s": evals / dt_s, "s_per_eval": dt_s / evals, "energy": e, "batch": best,
                     "gpu_launches_per_eval": (sum(c.launches() for c in ctxs) - l0) / evals,
                     "one_stream_s_per_eval": one_s, "same_as_one_stream": e == e1 and all(v[1] for v in trial.values()),
                     "trial_s_per_eval_by_batch": {str(b): round(v[0], 4) for b, v in trial.items()}}
    for p in ("tf32x3", "f16x3"):
        out[p]["rel_err_vs_f64"] = abs(res[p] - res["f64"]) / abs(res["f64"])
        out[p]["speedup_vs_f64"] = out[p]["evals_per_s"] / out["f64"]["evals_per_s"]
    out["mixed_vs_f64_rel_err"] = out["tf32x3"]["rel_err_vs_f64"]
    out["speedup_mixed_vs_f64"] = out["tf32x3"]["speedup_vs_f64"]
    if with_oracle:
        import oracle as O

        t0 = time.perf_counter()
        e_ref, *_ = O.energy_terms(lay, O.ket_tensors(lay, blocks), 1.0, 8.0, tf, policy="late", chi=32)
        out["oracle_energy"] = e_ref
        out["oracle_s_per_eval"] = time.perf_counter() - t0
        out["f64_rel_err_vs_oracle"] = abs(res["f64"] - e_ref) / abs(e_ref)
        out["tf32x3_rel_err_vs_oracle"] = abs(res["tf32x3"] - e_ref) / abs(e_ref)
        out["f16x3_rel_err_vs_oracle"] = abs(res["f16x3"] - e_ref) / abs(e_ref)
    for c in ctxs[1:]:
        c.synchronize()
        c.close()
    return out


GRADIENT_WORKLOAD = ("gradient of the norm <Psi|Psi> of an fPEPS on a 6x6 open square lattice, D=4 (2+2), phys 4 "
                     "(2+2), N(0,1) site tensors (seed 5), boundary-MPS row sweep (ket and bra of a site merged; "
                     "one boundary tensor per column absorbs its column's sites row by row, the horizontal bonds "
                     "between column tensors capped by late compression at chi=48; columns merged at the end), "
                     "locally ordered; dv/dT for all 72 tensors (kets and bras as independent inputs), FP64")


def kernel_breakdown(torch, fn, top=12):
    """Device time per kernel of one call of fn, from torch's profiler (CUDA
    activity; a profile, not a timing: the numbers reported as rates come
    from the runs outside it)."""
    import collections

    from torch.profiler import ProfilerActivity, profile

    # the first profiler session of a process records no kernels: one
    # session is spent on a warm-up call
    for _ in range(2):
        with profile(activities=[ProfilerActivity.CUDA]) as prof:
            fn()
            torch.cuda.synchronize()
    with profile(activities=[ProfilerActivity.CUDA]) as prof:
        fn()
        torch.cuda.synchronize()
    agg = collections.defaultdict(lambda: [0, 0.0])
    for ev in prof.events():
        if ev.device_type == torch.autograd.DeviceType.CUDA:
            t = getattr(ev, "device_time_total", None)
            if t is None:
                t = ev.cuda_time_total
            a = agg[ev.name.replace("(anonymous namespace)::", "").split("(")[0]]
            a[0] += 1
            a[1] += t / 1000.0
    tot = sum(v[1] for v in agg.values()) or 1.0
    rows = sorted(agg.items(), key=lambda kv: -kv[1][1])[:top]
    return {"total_ms": tot, "kernels": [{"name": k, "launches": c, "ms": ms, "share": ms / tot} for k, (c, ms) in rows]}


def gradient_bench(F, ctx, evals, samples=20, h=1e-6, kernels=False):
    """Gradient evaluations per second of the compressed norm network (6x6
    open lattice, D=4, boundary-MPS row sweep, chi=48) through
    ftn_contract_grad with checkpointed
    recomputation (the walk's state kept every ceil(sqrt(steps)) steps, each
    segment replayed in the backward) and with every intermediate kept; the
    library's peak device memory of each (its allocations routed through
    torch's allocator); the two gradients compared bit for bit; the value
    against ftn_contract's; central finite differences of ftn_contract on
    `samples` seeded entries (h = 1e-6, FP64)."""
    import math

    import numpy as np
    import torch

    from paper_2410_02215_gb300 import peps

    n, edges = W.square_lattice(6, 6)
    lay = W.peps_layout(n, edges, (2, 2), (2, 2))
    blocks = W.random_peps(lay, 5)
    kets = [F.Tensor.from_blocks(ctx, lay["legs"][s], 0, blocks[s]) for s in range(n)]
    tensors, bonds, _ = peps.norm_network(ctx, lay, kets)
    tree = W.double_layer_tree(n, W.boundary_mps_tree(6, 6))
    ctx.synchronize()
    k_ck = int(math.ceil(math.sqrt(len(tree))))

    def run(k):
        c = F.Context(use_torch_allocator=True)  # same stream as ctx
        try:
            torch.cuda.synchronize()
            base = torch.cuda.memory_allocated()
            torch.cuda.reset_peak_memory_stats()
            v, grads = F.contract_grad(c, tensors, bonds, tree, policy="late", chi=48, checkpoint=k)  # warm-up
            c.synchronize()
            peak = torch.cuda.max_memory_allocated() - base
            host = [dict(g.to_blocks()) for g in grads]
            del grads
            l0 = c.launches()
            t0 = time.perf_counter()
            for _ in range(evals):
                v, grads = F.contract_grad(c, tensors, bonds, tree, policy="late", chi=48, checkpoint=k)
                del grads
            c.synchronize()
            dt = time.perf_counter() - t0
            return v, host, dt / evals, (c.launches() - l0) / evals, peak
        finally:
            c.close()

    breakdown = None
    if kernels:
        c = F.Context()
        try:
            breakdown = kernel_breakdown(torch, lambda: F.contract_grad(c, tensors, bonds, tree, policy="late", chi=48))
        finally:
            c.close()
    v, host, s_ck, launches, peak_ck = run(k_ck)
    v0, host0, s_0, launches0, peak_0 = run(0)
    same = v == v0 and all(np.array_equal(a[key], b[key]) for a, b in zip(host, host0) for key in a)
    m, lg = F.contract(ctx, tensors, bonds, tree, policy="late", chi=48)
    scale = max(float(np.max(np.abs(b))) for d in host for b in d.values())
    rng = np.random.default_rng(0)
    worst = 0.0
    t1 = time.perf_counter()
    for _ in range(samples):
        i = int(rng.integers(len(tensors)))
        tb = dict(tensors[i].to_blocks())
        key = sorted(tb)[int(rng.integers(len(tb)))]
        idx = tuple(int(rng.integers(d)) for d in tb[key].shape)
        vals = []
        for sg in (1.0, -1.0):
            pb = {k: b.copy() for k, b in tb.items()}
            pb[key][idx] += sg * h
            t = F.Tensor.from_blocks(ctx, tensors[i].legs, tensors[i].parity, sorted(pb.items()))
            mm, ll = F.contract(ctx, tensors[:i] + [t] + tensors[i + 1:], bonds, tree, policy="late", chi=48)
            vals.append(mm * np.exp(ll))
            del t
        fd = (vals[0] - vals[1]) / (2 * h)
        worst = max(worst, abs(fd - float(host[i][key][idx])) / scale)
    fd_s = time.perf_counter() - t1
    return {"workload": GRADIENT_WORKLOAD, "gradient_evals_per_s": 1.0 / s_ck, "s_per_gradient": s_ck,
            "checkpoint": {"every_steps": k_ck, "steps": len(tree), "peak_bytes": peak_ck,
                           "note": "the walk's state kept every k steps, each segment replayed in the backward"},
            "no_checkpoint": {"gradient_evals_per_s": 1.0 / s_0, "s_per_gradient": s_0, "peak_bytes": peak_0,
                              "gpu_launches_per_gradient": launches0},
            "same_as_no_checkpoint": bool(same),
            **({"kernel_breakdown_no_checkpoint": breakdown} if breakdown else {}),
            "gpu_launches_per_gradient": launches, "value": v,
            "value_rel_err_vs_contract": abs(m * np.exp(lg) - v) / abs(v),
            "fd": {"samples": samples, "h": h, "max_abs_err_over_max_grad": worst, "s": fd_s,
                   "note": "central differences of ftn_contract (normalised forward) on seeded entries of seeded "
                           "tensors, against dv/dT"}}


DIAMOND_WORKLOAD = ("Hubbard fPEPS on the 2x2x2-conventional-cell diamond lattice (64 sites, 86 bonds, open "
                    "boundaries), D=4 (2+2), phys 4 (2+2), t=1, U=8, N(0,1) site tensors (seed 1), stand-in gauges "
                    "0.5^k per sector on dangling bonds; every hopping and on-site term (150) by the cluster "
                    "approximation of radius 1 (cluster network with and without the operator, globally ordered), "
                    "late compression chi=32 (at radius 1 the intermediates' bonds reach 64 states and are compressed "
                    "at chi=32 without truncating anything: the oracle's energies at chi=32, chi=64 and exact agree to "
                    "2e-16, so chi=32 and chi=64 give the same energy)")


def diamond_graph(F, torch, nets, num, den, ge, prec, streams, chunk, evals, energy_ref):
    """The diamond evaluation replayed from CUDA graphs.  A compression reads
    its kept dimensions back to the host, so a graph holds only contractions
    that compress nothing: the networks run with the exact policy here (at
    radius 1 the late compressions at chi = 32 keep every state, so the two
    energies agree to rounding; the deviation is reported).  Every context
    (its own stream) takes a strided share of the networks, contracts it once
    in lock-step batches of `chunk` (ftn_contract_batch_async: the plans),
    captures the same calls into one graph, and each evaluation replays the
    graphs on their streams, reads the values back and reduces them
    (ftn_energy_reduce)."""
    import numpy as np

    nets = [dict(j, policy="exact", chi=0) for j in nets]
    ctxs = [F.Context(stream=torch.cuda.Stream()) for _ in range(max(streams, 1))]
    graphs = []
    try:
        shares = [list(range(i, len(nets), len(ctxs))) for i in range(len(ctxs))]
        d_outs = [torch.zeros(max(2 * len(sh), 2), dtype=torch.float64, device="cuda") for sh in shares]
        t0 = time.perf_counter()
        for c, sh, d in zip(ctxs, shares, d_outs):
            sub = [nets[i] for i in sh]
            chunks = [(k, sub[k:k + chunk]) for k in range(0, len(sub), chunk)]
            for k, ch in chunks:  # plans on this context
                F.contract_batch_async(c, ch, d[2 * k:], prec)
            c.synchronize()
            g = torch.cuda.CUDAGraph()
            with torch.cuda.graph(g, stream=c.stream):
                for k, ch in chunks:
                    F.contract_batch_async(c, ch, d[2 * k:], prec)
            graphs.append(g)
        capture_s = time.perf_counter() - t0
        vals = np.zeros((len(nets), 2))

        def evaluate():
            for c, g in zip(ctxs, graphs):
                with torch.cuda.stream(c.stream):
                    g.replay()
            torch.cuda.synchronize()
            for sh, d in zip(shares, d_outs):
                if sh:
                    vals[sh] = d[:2 * len(sh)].cpu().numpy().reshape(-1, 2)
            return F.energy_reduce([tuple(v) for v in vals], num, den, ge)

        evaluate()
        t0 = time.perf_counter()
        for _ in range(evals):
            en, rat = evaluate()
        dt_s = time.perf_counter() - t0
        return {"evals_per_s": evals / dt_s, "s_per_eval": dt_s / evals, "chunk": chunk, "graphs": len(graphs),
                "capture_s": capture_s, "policy": "exact", "energy": en[0],
                "rel_dev_from_late_chi32": abs(en[0] - energy_ref) / abs(energy_ref),
                "note": "one CUDA graph per context (its strided share of the networks in lock-step batches, exact "
                        "policy), replayed per evaluation; values read back and reduced by ftn_energy_reduce"}
    finally:
        graphs.clear()
        torch.cuda.synchronize()
        for c in ctxs:
            c.close()


def diamond_bench(F, ctx, torch, evals, streams, with_oracle, rank=0, world=1, batches=(0, 8, 32), graphs=True,
                  kernels=False):
    """Energy evaluations per second of the 64-site diamond (radius-1 cluster
    approximation of all 150 terms), FP64 and mixed, with their errors; the
    term networks are split across ranks when world > 1 (dist.energy_sharded:
    one all-reduce of the network values, the same reduction on every rank).
    The oracle is timed on one representative term per cluster size and its
    time for all terms extrapolated from the counts (labelled so)."""
    import numpy as np

    from paper_2410_02215_gb300 import dist as D
    from paper_2410_02215_gb300 import peps

    n, edges, _ = W.diamond_lattice(2, 2, 2)
    lay = W.peps_layout(n, edges, (2, 2), (2, 2))
    blocks = W.random_peps(lay, 1)
    gs = W.bond_gauges(lay)

    def cfn(targets):
        sites = W.cluster_sites(lay, targets, 1)
        return (sites, W.dangling_bonds(lay, sites), W.cluster_tree(lay, sites, targets, True),
                W.cluster_tree(lay, sites, targets, False))

    ctxs = [ctx] + [F.Context(stream=torch.cuda.Stream()) for _ in range(max(streams, 1) - 1)]
    out = {"workload": DIAMOND_WORKLOAD, "streams": len(ctxs), "ranks": world,
           "terms": len(lay["edges"]) + n, "networks_per_eval": 2 * (len(lay["edges"]) + n)}
    res = {}
    for prec, dt in (("f64", F.F64), ("tf32x3", F.F32), ("f16x3", F.F32)):
        kets = [F.Tensor.from_blocks(ctx, lay["legs"][s], 0, blocks[s], dt) for s in range(n)]
        ctx.synchronize()
        nets, num, den, ge, keep = peps.cluster_networks(ctx, [(lay, kets, cfn, gs)], 1.0, 8.0, "late", 32, dt)

        def evaluate(batch):
            if world == 1:
                return F.energy(ctxs, nets, num, den, ge, prec, batch)[:2]
            return D.energy_sharded(nets, num, den, ge, rank, world,
                                    lambda sub: F.energy(ctxs, sub, [], [], [], prec, batch)[2])

        for c in ctxs:  # warm-up: every context builds its plans
            F.energy(c, nets, num, den, ge, prec, 0)
        trial = {}
        for b in batches:
            evaluate(b)
            barrier(world)
            t0 = time.perf_counter()
            en, rat = evaluate(b)
            trial[b] = time.perf_counter() - t0
        best = min(trial, key=lambda b: trial[b])
        l0 = sum(c.launches() for c in ctxs)
        barrier(world)
        t0 = time.perf_counter()
        for _ in range(evals):
            en, rat = evaluate(best)
        barrier(world)
        dt_s = max_over_ranks(time.perf_counter() - t0, world)
        res[prec] = (en[0], rat)
        out[prec] = {"evals_per_s": evals / dt_s, "s_per_eval": dt_s / evals, "terms_per_s": evals * len(rat) / dt_s,
                     "energy": en[0], "energy_per_site": en[0] / n, "batch": best,
                     "gpu_launches_per_eval": (sum(c.launches() for c in ctxs) - l0) / evals,
                     "trial_s_per_eval_by_batch": {str(b): round(v, 4) for b, v in trial.items()}}
        if kernels and prec in ("f64", "f16x3"):
            out[prec]["kernel_breakdown_one_stream"] = kernel_breakdown(
                torch, lambda: F.energy(ctx, nets, num, den, ge, prec, best), top=14)
        if world == 1 and graphs:
            try:
                out[prec]["graph"] = diamond_graph(F, torch, nets, num, den, ge, prec, len(ctxs), max(best, 1),
                                                   evals, en[0])
            except Exception as exc:  # reported, not fatal: the eager numbers above stand
                out[prec]["graph"] = {"error": f"{type(exc).__name__}: {exc}"}
        del keep
    e64, r64 = res["f64"]
    for p in ("tf32x3", "f16x3"):
        out[p]["rel_err_vs_f64"] = abs(res[p][0] - e64) / abs(e64)
        out[p]["max_term_err_vs_f64"] = max(abs(x - y) for x, y in zip(res[p][1], r64)) / max(abs(y) for y in r64)
        out[p]["speedup_vs_f64"] = out[p]["evals_per_s"] / out["f64"]["evals_per_s"]
    out["mixed_vs_f64_rel_err"] = out["tf32x3"]["rel_err_vs_f64"]
    out["speedup_mixed_vs_f64"] = out["f16x3"]["speedup_vs_f64"]
    if with_oracle:
        import oracle as O

        okets = O.ket_tensors(lay, blocks)
        terms = [tuple(e) for e in lay["edges"]] + [(s,) for s in range(n)]
        by_size = {}
        for q, tg in enumerate(terms):
            by_size.setdefault((len(tg), len(W.cluster_sites(lay, list(tg), 1))), []).append(q)
        est, errs, sample_s = 0.0, [], 0.0
        for key in sorted(by_size):
            q = by_size[key][0]
            tg = terms[q]
            op = O.hop_gate(1.0) if len(tg) == 2 else O.onsite_gate(8.0)
            sites, dang, tr_op, tr_norm = cfn(list(tg))
            t0 = time.perf_counter()
            rn, ln, _ = O.contract_tree(O.cluster_network(lay, okets, sites, dang, gs, op, list(tg)), tr_op,
                                        mode="global", policy="late", chi=32, normalize=True)
            rd, ld, _ = O.contract_tree(O.cluster_network(lay, okets, sites, dang, gs), tr_norm, mode="global",
                                        policy="late", chi=32, normalize=True)
            dt_t = time.perf_counter() - t0
            ref = float(rn.data) / float(rd.data) * np.exp(ln - ld)
            errs.append(abs(r64[q] - ref))
            sample_s += dt_t
            est += dt_t * len(by_size[key])
        scale = max(abs(y) for y in r64)
        out["oracle"] = {"s_per_eval_extrapolated": est, "evals_per_s_extrapolated": 1.0 / est,
                         "cores": len(os.sched_getaffinity(0)),
                         "sample": f"one term per (term kind, cluster size) class, {len(by_size)} terms in "
                                   f"{sample_s:.1f} s; the full evaluation's time extrapolated from the class counts",
                         "f64_gpu_max_term_err_on_sample": max(errs) / scale}
    for c in ctxs[1:]:
        c.synchronize()
        c.close()
    return out


def run_ours(args, rank, world, local):
    import torch

    from paper_2410_02215_gb300 import ftn as F

    torch.cuda.set_device(local)
    F.lib()
    ctx = F.Context()
    if args.no_tune:
        ctx.set_tuning(False)
    peaks = load_peaks()
    cases = [W.tensordot_case(n, seed=0) for n in args.cases]
    flops_step = sum(sector_flops(c) for c in cases)
    flush = torch.empty(512 * 1024 * 1024, dtype=torch.uint8, device="cuda")  # > 129 MB L2
    clk = ClockSampler(local)
    clk.start()
    ms_eager, launches, prof, ins, outs, ginfo = time_steps(F, ctx, torch, cases, args.prec, args.steps, args.warmup,
                                                            flush, world, profile=True, graph=not args.no_graph)
    clocks = clk.stop()
    use_graph = bool(ginfo and ginfo.get("identical"))
    ms = ginfo["ms"] if use_graph else ms_eager
    back = None
    if not args.no_backward:
        back = backward_bench(F, ctx, torch, cases, args.prec, max(2, args.steps // 2), args.warmup, flush, ins, outs,
                              flops_step)
    del ins, outs
    ms_max = max_over_ranks(ms, world)
    value = flops_step * args.steps * world / (ms_max / 1e3) / 1e12
    result = {
        "metric": "sector-GEMM TFLOP/s", "value": value, "unit": "TFLOP/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_max / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": PREC_DTYPE[args.prec], "data": "synthetic",
        "config": {"workload": WORKLOAD, "precision": args.prec, "sector_gflop_per_step": flops_step / 1e9,
                   "l2": "flushed between steps (512 MB write, outside the timed events)",
                   "parallelism": f"replicas x{world} (independent problems, no collective)"},
        "gpu_launches": launches * args.steps,
    }
    result["config"]["launch"] = ("CUDA graph of the step, captured once and replayed (outputs bit-identical to the "
                                  "eager step)" if use_graph else "eager: one library call per contraction")
    result["eager_ms_per_step"] = max_over_ranks(ms_eager, world) / args.steps
    if ginfo is not None:
        result["graph"] = ginfo
    result["roofline"] = roofline(prof, peaks, args.prec)
    if back is not None:
        result["backward"] = back
    result["kernels"] = [{"label": r["label"], "launches": r["launches"], "ms": r["ms"],
                          "gbs": r["bytes"] / (r["ms"] / 1e3) / 1e9 if r["ms"] else None,
                          "tflops": r["flops"] / (r["ms"] / 1e3) / 1e12 if r["ms"] and r["flops"] else None}
                         for r in prof]
    # each sign-permute beside a plain copy of the same bytes (cold L2)
    copy_ms = {}
    for k, r in zip(result["kernels"], prof):
        if r["label"].endswith("/permute") and r["bytes"] and r["launches"]:
            b = int(r["bytes"] / r["launches"])
            if b not in copy_ms:
                copy_ms[b] = copy_reference_ms(torch, b, flush)
            k["copy_ms_per_launch_same_bytes"] = copy_ms[b]
    if clocks:
        result["clocks"] = clocks
    # the other precisions of the same step, and their errors
    precs = {}
    for p in args.compare:
        if p == args.prec:
            continue
        pms, _, _, pin, pout, _ = time_steps(F, ctx, torch, cases, p, max(2, args.steps // 4), 2, flush, 1)
        del pin, pout
        precs[p] = {"tflops": flops_step * max(2, args.steps // 4) / (pms / 1e3) / 1e12,
                    "ms_per_step": pms / max(2, args.steps // 4)}
    precs[args.prec] = {"tflops": flops_step * args.steps / (ms / 1e3) / 1e12, "ms_per_step": ms / args.steps}
    if rank == 0 and not args.no_accuracy:
        for p in precs:
            precs[p].update(accuracy(F, ctx, p))
    result["precisions"] = precs
    if "f64" in precs:
        result["speedup_vs_f64_gpu"] = precs[args.prec]["tflops"] / precs["f64"]["tflops"]
    if not args.no_e2e:
        result["e2e"] = e2e_run(F, ctx, torch, cases, args.prec, max(4, min(args.steps, 10)), flops_step)
    if not args.no_cluster:
        result["cluster"] = cluster_bench(F, ctx, torch, args.cluster_graphs, args.cluster_streams,
                                          rank == 0 and world == 1 and not args.no_cpu)
    if not args.no_energy:
        result["energy"] = energy_bench(F, ctx, args.energy_evals, rank == 0 and world == 1 and not args.no_cpu,
                                        args.energy_streams)
    if not args.no_gradient:
        result["gradient"] = gradient_bench(F, ctx, args.gradient_evals, kernels=args.gradient_kernels)
    if not args.no_diamond:
        result["energy_diamond"] = diamond_bench(F, ctx, torch, args.diamond_evals, args.cluster_streams,
                                                 rank == 0 and world == 1 and not args.no_cpu, rank, world,
                                                 kernels=args.diamond_kernels)
    if rank == 0 and world == 1 and not args.no_cpu:
        result["cpu_baseline"] = cpu_baseline(cases)
    ctx.synchronize()
    ctx.close()
    if rank == 0:
        print(json.dumps(result), flush=True)
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--prec", default="f16x3", choices=list(PREC_DTYPE))
    ap.add_argument("--compare", default="f64,tf32,bf16x3,tf32x3", type=lambda s: [x for x in s.split(",") if x])
    ap.add_argument("--cases", default=",".join(CASES), type=lambda s: [x for x in s.split(",") if x])
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-energy", action="store_true")
    ap.add_argument("--no-backward", action="store_true")
    ap.add_argument("--no-cluster", action="store_true")
    ap.add_argument("--no-graph", action="store_true", help="time the step eagerly only (no CUDA-graph replay)")
    ap.add_argument("--no-tune", action="store_true",
                    help="keep every plan's default GEMM tile width (for profiler runs, whose timings mislead the tuner)")
    ap.add_argument("--cluster-graphs", type=int, default=64)
    ap.add_argument("--cluster-streams", type=int, default=16,
                    help="contexts (one stream and host thread each) of the cluster-approximation workloads")
    ap.add_argument("--energy-evals", type=int, default=3)
    ap.add_argument("--energy-streams", type=int, default=8,
                    help="contexts (CUDA streams) that run an evaluation's contractions concurrently")
    ap.add_argument("--no-accuracy", action="store_true")
    ap.add_argument("--no-diamond", action="store_true")
    ap.add_argument("--no-gradient", action="store_true")
    ap.add_argument("--gradient-evals", type=int, default=3)
    ap.add_argument("--gradient-kernels", action="store_true",
                    help="add a per-kernel device-time breakdown of one gradient (torch profiler)")
    ap.add_argument("--diamond-evals", type=int, default=2)
    ap.add_argument("--diamond-kernels", action="store_true",
                    help="add a per-kernel device-time breakdown of one diamond evaluation on one stream "
                         "(torch profiler)")
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    rank, world, local = dist_init()
    if args.impl == "reference":
        rc = run_reference(args, rank, world)
    else:
        rc = run_ours(args, rank, world, local)
    if world > 1:
        import torch.distributed as dist

        dist.destroy_process_group()
    return rc


if __name__ == "__main__":
    sys.exit(main())
