"""Benchmark of the quaternion Dirac-Coulomb(-Breit) AO->MO transformation.

One step = one qdt_transform() over the whole hot path (density, screening,
AO integral tiles, first and second half-transforms, packing) of the
workload, with the basis and coefficients already resident on the GPU.

Default workload: the 40-centre s+p chain (nL = 160, nS = 480, 40 Kramers
pairs, Schwarz threshold 1e-12, seeded synthetic inputs standing in for the
paper's Hg/Pu chains).  Prints one JSON line (rank 0).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                  [--workload chain40-sp] [--blocks coulomb[,gaunt,gauge]]
                  [--precision split|fp64]
Multi-GPU (torchrun): every rank transforms its own copy of the workload
(independent problems, weak scaling, no data-path collective).
"""
from __future__ import annotations

import argparse
import json
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from paper_2606_04316_gb300 import synth  # noqa: E402

PEAKS_FILE = os.path.join(ROOT, "MEASURED_PEAKS.json")
NOMINAL = {"bf16": 2250.0, "fp64": 1.25}     # dense TF/s, for dtype ratios
SMS = 152                 # streaming multiprocessors of a GB300
DFMA_PER_CLK_SM = 2       # FP64 FMA lanes per clock per SM (ncu: dfma peak_sustained 2 inst/cycle/SM)
FP32_PER_CLK_SM = 128     # FP32 lanes per clock per SM
DF_OPS_PER_MADD = 12      # FP32 operations of one compensated FP32-pair multiply-add (split-form integrals)


def fp64_alu_peak(clocks):
    """FP64 FMA peak in TFLOP/s from the unit counts and the SM clock sampled under load."""
    mhz = (clocks or {}).get("sm_mhz") or 2070.0
    return SMS * DFMA_PER_CLK_SM * 2 * mhz * 1e6 / 1e12, mhz


def workload(name):
    if name == "chain40-sp":
        return synth.medium_dc()
    if name == "tiny-6s":
        return synth.tiny_dc()
    if name == "cluster64-sp":
        return synth.dcb_cluster()
    if name.startswith("cluster") and "x" in name:       # clusterAxBxC-nK: the same recipe, smaller
        dims, nk = name[7:].split("-")
        return synth.dcb_cluster(dims=tuple(int(d) for d in dims.split("x")), nK=int(nk))
    if name.startswith("chain"):
        n = int(name[5:].split("-")[0])
        return synth.medium_dc(n_centers=n, nK=n)
    raise SystemExit("unknown workload " + name)


def peaks():
    try:
        with open(PEAKS_FILE) as f:
            p = json.load(f)
        return p, "measured"
    except Exception:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0}, "fallback"


class ClockSampler:
    """nvidia-smi clocks and throttle reasons during the timed region."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.lines = []
        self.proc = None

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.Q,
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if not self.proc:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx = float(f[2])
            except ValueError:
                continue
            for n, v in zip(names, f[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(n)
        return {"sm_mhz": float(np.median(sm)) if sm else None, "sm_max_mhz": mx,
                "samples": len(sm), "reasons": sorted(reasons)}


def mo_integrals(nK, nblocks):
    return float((2 * nK) ** 4) * nblocks


def mo_count(problem, nblocks):
    """(pq|rs) over all spinors of the active range: 2 nK spinors for Kramers
    pairs, nK spinors for Kramers-unrestricted input."""
    n = problem.nK if not problem.kramers else 2 * problem.nK
    return float(n) ** 4 * nblocks


def as_unrestricted(problem):
    """The same basis with seeded Kramers-unrestricted coefficients for as many
    spinors (2 nK) as the Kramers-restricted workload has."""
    rng = np.random.Generator(np.random.PCG64(synth.SEED_BASE + 100))
    CL, CS = synth.ku_coefficients(rng, problem.basis.nL, 2 * problem.nK)
    return synth.Problem(problem.name + "-ku", problem.basis, CL, CS, problem.blocks, problem.tau, kramers=False)


def max_over_ranks(ms, world, device):
    """The step time of the job: the slowest rank's (every rank calls this)."""
    if world <= 1:
        return ms
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(ms)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_value(n_mo, world, ms):
    """Whole-job throughput: every rank transforms its own replica of the
    workload (weak scaling), all within the slowest rank's step time."""
    return n_mo * world / (ms / 1e3)


def run_reference(args, problem, blocks, rank):
    """CPU oracle on a bounded sample of the workload (rank 0 only)."""
    if rank != 0:
        return
    res = cpu_oracle_rate(problem, blocks, budget_s=args.ref_budget)
    line = {"metric": METRIC, "value": res["value"], "unit": "MO-integrals/s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": res["ms"],
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "impl": "reference",
            "config": config_dict(args, problem, blocks),
            "cpu_baseline": {"value": res["value"], "unit": "MO-integrals/s", "cores": res["cores"],
                             "kind": "oracle", "sample": res["sample"]},
            "e2e": {"value": res["value"], "unit": "MO-integrals/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def cpu_oracle_rate(problem, blocks, budget_s=20.0):
    """Time the oracle on a reduced chain of the same recipe, grown until one
    full transformation takes about budget_s / 2 seconds."""
    from oracle import oracle as O
    O.build()
    cores = os.cpu_count()
    n, last = 2, None
    while True:
        p = synth.chain_problem(n, n, seed=synth.SEED_BASE + 1, shells=(0, 1), nprim=3,
                                blocks=blocks, tau=problem.tau, name="sample")
        if not problem.kramers:
            p = as_unrestricted(p)
        t0 = time.perf_counter()
        tr = O.Transform(p) if problem.kramers else O.TransformKU(p)
        for b in blocks:
            tr.packed(b)
        dt = time.perf_counter() - t0
        last = (n, dt)
        if dt > budget_s / 2 or n >= 12:
            break
        n += 2
    n, dt = last
    rate = mo_integrals(n, len(blocks)) / dt
    kind = "nK=%d" % n if problem.kramers else "%d unrestricted spinors" % (2 * n)
    return {"value": rate, "ms": dt * 1e3, "cores": cores,
            "sample": "oracle, full transform of a %d-centre s+p chain (same recipe, %s, blocks=%s) "
                      "on %d host threads; %.1f s" % (n, kind, "+".join(blocks), cores, dt)}


METRIC = "DCB AO->MO transform MO-integrals/s (split vs FP64 @1e-10 Eh)"


def config_dict(args, problem, blocks):
    d = {"workload": args.workload, "nL": problem.basis.nL, "nS": problem.basis.nS,
         "n_kramers": problem.nK, "blocks": "+".join(blocks), "schwarz_tau": problem.tau,
         "precision": args.precision, "l2": "inputs larger than L2 (densities, integral rows)"}
    if getattr(args, "route", "density") != "density":
        d["route"] = args.route
        if args.route == "mo":
            d["mo_block"] = args.mo_block
    if not problem.kramers:
        del d["n_kramers"]
        d["n_spinors"] = problem.nK
        d["input"] = "kramers-unrestricted"
    return d


def run_serving(args):
    """Request stream through the continuous-batching server (qdt_server_*):
    seeded chain/cluster requests of different sizes, half Dirac-Coulomb and half
    Dirac-Coulomb-Breit, Poisson arrivals at 0.8 x the capacity measured by a
    sequential calibration pass; p50/p99 latency and MO-integrals/s."""
    import torch
    from paper_2606_04316_gb300 import qdt
    torch.cuda.set_device(0)
    prec = qdt.SPLIT if args.precision == "split" else qdt.FP64
    reqs = synth.serving_requests(args.requests, nl_range=(24, args.max_nl), nk_range=(8, args.max_nk))
    outs = []
    ctx = qdt.Context(0)
    t0 = time.perf_counter()
    for p in reqs:                                  # calibration: one at a time
        ctx.set_basis(p.basis)
        ctx.set_coefficients(p.CL, p.CS)
        o = np.zeros(ctx.packed_size(list(p.blocks), 0, p.nK) // 8)
        ctx.transform(list(p.blocks), 0, p.nK, p.tau, prec, o)
        outs.append(o)
    t_seq = time.perf_counter() - t0
    ctx.close()
    rate = 0.8 * len(reqs) / t_seq
    rng = np.random.Generator(np.random.PCG64(synth.SEED_BASE + 3))
    arrivals = np.cumsum(rng.exponential(1.0 / rate, size=len(reqs)))
    srv = qdt.Server(0, n_slots=args.slots)
    handles, res = [], []
    start = time.perf_counter()
    for p, ta in zip(reqs, arrivals):
        dt = start + ta - time.perf_counter()
        if dt > 0:
            time.sleep(dt)
        o = np.zeros_like(outs[len(res)])
        r, keep = srv.make_request(p, list(p.blocks), 0, p.nK, p.tau, prec, o)
        handles.append(srv.submit(r, keep))
        res.append(o)
    lat = [srv.wait(h)[0] for h in handles]
    makespan = time.perf_counter() - start
    srv.close()
    same = all(np.array_equal(a, b) for a, b in zip(outs, res))
    n_mo = sum(mo_integrals(p.nK, len(p.blocks)) for p in reqs)
    line = {"metric": "serving: p50/p99 request latency and MO-integrals/s (continuous batching)",
            "value": n_mo / makespan, "unit": "MO-integrals/s", "n_gpus": 1, "higher_is_better": True,
            "latency_s": {"p50": float(np.percentile(lat, 50)), "p99": float(np.percentile(lat, 99)),
                          "mean": float(np.mean(lat))},
            "arrival_rate_per_s": rate, "calibration_sequential_s": t_seq, "makespan_s": makespan,
            "requests": len(reqs), "slots": args.slots, "precision": args.precision,
            "results_same_alone_and_in_mix": same, "data": "synthetic",
            "config": {"workload": "serving", "nL": [24, args.max_nl], "nK": [8, args.max_nk],
                       "blocks": "half coulomb, half coulomb+gaunt+gauge", "schwarz_tau": 1e-11}}
    print(json.dumps(line), flush=True)


def run_batch(args):
    """The same seeded request stream as the serving workload, run three ways on
    one GPU: one qdt_transform after another, one qdt_transform_batch (integral
    tiles of all requests fused into one persistent launch per kernel kind), and
    the batch replayed from its captured CUDA graph.  Device-resident outputs;
    host wall-clock time of each synchronised pass, median over --steps passes
    after --warmup."""
    import torch
    from paper_2606_04316_gb300 import qdt
    torch.cuda.set_device(0)
    prec = qdt.SPLIT if args.precision == "split" else qdt.FP64
    reqs = synth.serving_requests(args.requests, nl_range=(24, args.max_nl), nk_range=(8, args.max_nk))
    # graph replay needs a fixed screening outcome across passes: same inputs every pass
    ctxs, outs, jobs = [], [], []
    for p in reqs:
        c = qdt.Context(0)
        c.set_basis(p.basis)
        c.set_coefficients(p.CL, p.CS)
        o = torch.zeros(c.packed_size(list(p.blocks), 0, p.nK) // 8, dtype=torch.float64, device="cuda")
        ctxs.append(c)
        outs.append(o)
        jobs.append((c, list(p.blocks), 0, p.nK, p.tau, prec, o))
    n_mo = sum(mo_integrals(p.nK, len(p.blocks)) for p in reqs)

    def timed(fn):
        ms = []
        for i in range(args.warmup + args.steps):
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            fn()
            torch.cuda.synchronize()
            if i >= args.warmup:
                ms.append((time.perf_counter() - t0) * 1e3)
        return float(np.median(ms))

    phases = {}

    def sequential():
        phases.clear()
        for (c, b, k0, k1, tau, pr, o) in jobs:
            st = c.transform(b, k0, k1, tau, pr, o)
            for k in ("ms_total", "ms_density", "ms_screen", "ms_eri", "ms_half1", "ms_half2", "ms_pack"):
                phases[k] = phases.get(k, 0.0) + st[k]

    ms_seq = timed(sequential)
    ref = [o.clone() for o in outs]
    ms_batch = timed(lambda: qdt.transform_batch(jobs))
    diff_batch = max(float((o - r).abs().max().item()) for o, r in zip(outs, ref))
    ms_graph = timed(lambda: qdt.transform_batch(jobs, graph=True))
    diff_graph = max(float((o - r).abs().max().item()) for o, r in zip(outs, ref))
    caps, reps = ctxs[0].graph_counts()
    line = {"metric": "batching: MO-integrals/s of a request batch (fused persistent launches, graph replay)",
            "value": n_mo / (ms_graph / 1e3), "unit": "MO-integrals/s", "n_gpus": 1, "higher_is_better": True,
            "ms_per_pass": {"sequential": ms_seq, "batch": ms_batch, "batch_graph": ms_graph},
            "sequential_phases_ms": phases,
            "steps": args.steps, "warmup": args.warmup,
            "max_abs_diff_vs_sequential": {"batch": diff_batch, "batch_graph": diff_graph},
            "graph_captures": caps, "graph_replays": reps, "requests": len(reqs), "precision": args.precision,
            "data": "synthetic", "timing": "host wall clock around synchronised passes",
            "config": {"workload": "batch", "nL": [24, args.max_nl], "nK": [8, args.max_nk],
                       "blocks": "half coulomb, half coulomb+gaunt+gauge", "schwarz_tau": 1e-11}}
    print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=2)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="chain40-sp")
    ap.add_argument("--blocks", default="coulomb")
    ap.add_argument("--input", default="kramers", choices=["kramers", "ku"],
                    help="coefficients: quaternion (Kramers pairs) or Kramers-unrestricted spinors")
    ap.add_argument("--precision", default="split", choices=["split", "fp64"])
    ap.add_argument("--route", default="density", choices=["density", "quarter", "mo"],
                    help="density (AO-driven), quarter (O(N^5) Coulomb first half) or mo (MO-driven comparator)")
    ap.add_argument("--mo-block", type=int, default=8, help="MO-driven route: outer MO indices per block")
    ap.add_argument("--fp64-steps", type=int, default=1, help="timed steps of the FP64 form (0: skip)")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--ref-budget", type=float, default=20.0)
    ap.add_argument("--stats", action="store_true", help="print per-phase statistics to stderr")
    ap.add_argument("--requests", type=int, default=32, help="serving workload: number of requests")
    ap.add_argument("--slots", type=int, default=4, help="serving workload: concurrent contexts")
    ap.add_argument("--max-nl", type=int, default=64, help="serving workload: largest nL")
    ap.add_argument("--max-nk", type=int, default=16, help="serving workload: largest nK")
    args = ap.parse_args()
    if args.workload == "serving":
        return run_serving(args)
    if args.workload == "batch":
        return run_batch(args)
    blocks = args.blocks.split(",")
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    problem = workload(args.workload)
    if args.input == "ku":
        problem = as_unrestricted(problem)
    if args.impl == "reference":
        return run_reference(args, problem, blocks, rank)

    import torch
    import torch.distributed as dist
    from paper_2606_04316_gb300 import qdt
    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl")
    stream = torch.cuda.Stream()
    ctx = qdt.Context(local, stream=stream)
    ctx.set_basis(problem.basis)
    CLd = torch.from_numpy(problem.CL).cuda()
    CSd = torch.from_numpy(problem.CS).cuda()
    set_coefs = ctx.set_coefficients if problem.kramers else ctx.set_spinor_coefficients
    set_coefs(CLd, CSd)
    ctx.set_route(args.route, args.mo_block if args.route == "mo" else 0)
    nK = problem.nK
    prec = qdt.SPLIT if args.precision == "split" else qdt.FP64
    nout = ctx.packed_size(blocks, 0, nK) // 8
    out = torch.zeros(nout, dtype=torch.float64, device="cuda")
    tau = problem.tau

    def step():
        return ctx.transform(blocks, 0, nK, tau, prec, out)

    for _ in range(args.warmup):
        st = step()
    sampler = ClockSampler(local)
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    sampler.start()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    phase = {k: 0.0 for k in ("ms_eri", "ms_half1", "ms_half2", "ms_density", "ms_screen", "ms_pack")}
    launches = 0
    for _ in range(args.steps):
        st = step()
        for k in phase:
            phase[k] += st[k]
        launches += st["kernel_launches"]
    e1.record(stream)
    torch.cuda.synchronize()
    clocks = sampler.stop()
    ms = e0.elapsed_time(e1) / args.steps
    ms = max_over_ranks(ms, world, "cuda")
    n_mo = mo_count(problem, len(blocks))
    value = job_value(n_mo, world, ms)

    # end to end through the public API with host buffers (pinned)
    e2e = None
    if not args.no_e2e:
        CLh = torch.from_numpy(problem.CL).pin_memory()
        CSh = torch.from_numpy(problem.CS).pin_memory()
        outh = torch.zeros(nout, dtype=torch.float64).pin_memory()
        torch.cuda.synchronize()
        ne = 1
        t0 = time.perf_counter()
        for _ in range(ne):
            set_coefs(CLh, CSh)
            ctx.transform(blocks, 0, nK, tau, prec, outh)
        dt = (time.perf_counter() - t0) / ne
        e2e = {"value": n_mo * world / dt, "unit": "MO-integrals/s",
               "h2d_bytes_per_step": int(CLh.numel() * 8 + CSh.numel() * 8),
               "d2h_bytes_per_step": int(outh.numel() * 8)}

    # the FP64 form on the same workload, and the agreement of the two forms
    other = None
    if prec == qdt.SPLIT and args.fp64_steps > 0:
        out64 = torch.zeros_like(out)
        set_coefs(CLd, CSd)
        ctx.transform(blocks, 0, nK, tau, qdt.FP64, out64)
        ctx.transform(blocks, 0, nK, tau, prec, out)
        torch.cuda.synchronize()
        diff = float((out - out64).abs().max().item())
        f0 = torch.cuda.Event(enable_timing=True)
        f1 = torch.cuda.Event(enable_timing=True)
        f0.record(stream)
        for _ in range(args.fp64_steps):
            st64 = ctx.transform(blocks, 0, nK, tau, qdt.FP64, out64)
        f1.record(stream)
        torch.cuda.synchronize()
        ms64 = f0.elapsed_time(f1) / args.fp64_steps
        other = {"value": n_mo * world / (ms64 / 1e3), "ms_per_step": ms64, "steps": args.fp64_steps,
                 "phases_ms": {k: st64[k] for k in phase}, "max_abs_diff_split_vs_fp64": diff}

    pk, src = peaks()
    avg = {k: v / args.steps for k, v in phase.items()}
    dom = max(("ms_eri", "ms_half1", "ms_half2"), key=lambda k: avg[k])
    fp64_peak, mhz = fp64_alu_peak(clocks)
    fp64_note = "FP64 pipe: %d SMs x %d DFMA/clk x 2 flops x %.0f MHz sampled SM clock" % (SMS, DFMA_PER_CLK_SM, mhz)
    if dom == "ms_eri":
        achieved = st["flops_eri"] / (avg[dom] / 1e3) / 1e12
        if prec == qdt.SPLIT:
            # split form: the contractions run in compensated FP32 pairs (12 FP32 operations per
            # multiply-add) or, for the quartets within the FP32 error budget, in plain FP32 (one
            # FMA); the bound weighs the two by their share of the flops
            f32 = st.get("flops_eri_f32", 0.0) / st["flops_eri"] if st["flops_eri"] else 0.0
            ops = DF_OPS_PER_MADD * (1.0 - f32) + 1.0 * f32
            peak = SMS * FP32_PER_CLK_SM * mhz * 1e6 / ops * 2 / 1e12
            note = ("FP32 pipe: %d SMs x %d lanes x %.0f MHz / %.2f FP32 ops per multiply-add (%d for "
                    "compensated pairs, 1 for the %.1f %% of flops in plain FP32) x 2 flops (FP64-equivalent)"
                    % (SMS, FP32_PER_CLK_SM, mhz, ops, DF_OPS_PER_MADD, 100.0 * f32))
        else:
            peak, note = fp64_peak, fp64_note
        roof = {"kernel": "eri_rows_kernel", "bound": "alu", "achieved": achieved,
                "peak": peak, "unit": "TFLOP/s", "frac": achieved / peak,
                "traffic": None, "peak_note": note,
                "work": "E R E multiply-adds of the kept quartets (qdt_stats.flops_eri)"}
    else:
        fl = st["flops_half1"] if dom == "ms_half1" else st["flops_half2"]
        achieved = fl / (avg[dom] / 1e3) / 1e12
        if prec == qdt.FP64:
            peak, note, bound = fp64_peak, fp64_note, "alu"
        else:
            peak, note, bound = pk["bf16_tflops_sustained"], "%s bf16 sustained" % src, "tensor"
        roof = {"kernel": "half1" if dom == "ms_half1" else "half2", "bound": bound,
                "achieved": achieved, "peak": peak, "unit": "TFLOP/s", "frac": achieved / peak,
                "traffic": None, "peak_note": note}

    cpu = None
    if rank == 0 and not args.no_cpu:
        try:
            r = cpu_oracle_rate(problem, blocks)
            cpu = {"value": r["value"], "unit": "MO-integrals/s", "cores": r["cores"], "kind": "oracle",
                   "sample": r["sample"]}
        except Exception as ex:  # keep the bench line even if the oracle fails
            cpu = {"value": None, "unit": "MO-integrals/s", "cores": os.cpu_count(), "kind": "oracle",
                   "sample": "failed: %s" % ex}

    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": "MO-integrals/s", "n_gpus": world,
                "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": "f64" if prec == qdt.FP64 else "bf16-slices/f64",
                "data": "synthetic", "config": config_dict(args, problem, blocks), "clocks": clocks,
                "e2e": e2e, "gpu_launches": launches, "roofline": roof, "cpu_baseline": cpu,
                "phases_ms": avg, "quartets_kept": st["quartets_kept"], "quartets_total": st["quartets_total"],
                "fp64_form": other}
        print(json.dumps(line), flush=True)
        if args.stats:
            print(json.dumps(st), file=sys.stderr)
    ctx.close()
    if world > 1:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
