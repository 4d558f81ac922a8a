"""Benchmark of the quaternion Dirac-Coulomb(-Breit) AO->MO transformation.

One step = one qdt_transform() over the whole hot path (density, screening,
AO integral tiles, first and second half-transforms, packing) of the
workload, with the basis and coefficients already resident on the GPU.

Default workload: the Dirac-Coulomb-Breit blocks (Coulomb + Gaunt + gauge)
of the 40-centre s+p chain (nL = 160, nS = 480, 40 Kramers pairs, Schwarz
threshold 1e-12, seeded synthetic inputs standing in for the paper's Hg/Pu
chains), split form timed, FP64 form timed beside it.  Prints one JSON line
(rank 0).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                  [--workload chain40-sp] [--blocks coulomb,gaunt,gauge]
                  [--precision split|fp64]

--impl reference times the CPU oracle on a bounded sample of the same
workload per step (OracleSampler).
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


class OracleSampler:
    """The oracle timed on the bench workload itself: its row-streamed
    transform (oracle.Transform.V_rows_streamed, then each bra row's share
    D[rows]^T V[rows] of the second half) over a stratified sample of the bra
    shell pairs of every requested block.  A block's bra shell pairs are sorted
    by a cost proxy (function pairs x primitive pairs) and every k-th one taken
    (k at most the block's pair count), from an offset that rotates from one
    sample to the next.  Each sample records, per block, its time t_b and the
    fraction f_b of the block's bra shell pairs it covered; the time of a whole
    transformation is estimated as t_setup + sum_b (sum of t_b) / (sum of f_b),
    where t_setup is the per-transformation set-up (densities, Schwarz factors,
    density maxima, screening masks), run once."""

    def __init__(self, problem, blocks):
        from oracle import oracle as O
        O.build()
        self.O = O
        self.blocks = blocks
        self.problem = problem
        t0 = time.perf_counter()
        self.tr = O.Transform(problem) if problem.kramers else O.TransformKU(problem)
        for b in blocks:
            self.tr.density(b)
            self.tr.mask(b)
            list(self.tr.V_rows_streamed(b, bra_pairs=[]))      # ket order of the block
        self.t_setup = time.perf_counter() - t0
        self.order = {}
        for b in blocks:
            cls = 0 if b == "coulomb" else 1
            ob = self.tr.ob
            nsp = ob.n_shell_pairs(cls)
            cost = []
            for p in range(nsp):
                sa, sb = ob._shell_pair_shells(cls, p)
                cost.append(ob._nfunc(sa) * ob._nfunc(sb) * int(problem.basis.shell_nprim[sa % ob.nsh]) *
                            int(problem.basis.shell_nprim[sb % ob.nsh]))
            self.order[b] = np.argsort(-np.array(cost), kind="stable")
        self.step = 0
        self.reset()

    def reset(self):
        self.tsum = {b: 0.0 for b in self.blocks}
        self.fsum = {b: 0.0 for b in self.blocks}
        self.times = []

    def sample(self, k):
        """Seconds of one sample at stride k (next offset); accumulates t_b, f_b."""
        total = 0.0
        for b in self.blocks:
            n = len(self.order[b])
            kb = max(1, min(k, n))
            pairs = self.order[b][self.step % kb::kb]
            t0 = time.perf_counter()
            for rows, Vr in self.tr.V_rows_streamed(b, bra_pairs=pairs):
                self.tr.second_half_rows(b, rows, Vr)
            dt = time.perf_counter() - t0
            self.tsum[b] += dt
            self.fsum[b] += len(pairs) / n
            total += dt
        self.step += 1
        self.times.append(total)
        return total

    def calibrate(self, budget_s):
        """Stride k (a power of two, from 4096 down) at which one sample takes
        at least budget_s / 2."""
        k = 4096
        while self.sample(k) < budget_s / 2 and k > 1:
            k //= 2
        self.reset()
        return k

    def full_seconds(self):
        """Estimated seconds of one whole transformation from the samples so far."""
        return self.t_setup + sum(self.tsum[b] / self.fsum[b] for b in self.blocks if self.fsum[b] > 0)

    def describe(self, k, cores):
        fr = ", ".join("%s %.2e" % (b, self.fsum[b] / max(1, len(self.times))) for b in self.blocks)
        return ("oracle (oracle.Transform, row-streamed, screened) on this workload itself: %d samples, each "
                "every %d-th bra shell pair of every block in cost order (rotating offset; mean fraction of a "
                "block's bra pairs per sample: %s) through both half-transforms; whole transformation "
                "estimated as set-up %.1f s (densities, Schwarz factors, masks; run once) + sum over blocks of "
                "sampled time / sampled fraction = %.1f s; %s host threads"
                % (len(self.times), k, fr, self.t_setup, self.full_seconds(), cores))


def oracle_threads():
    """Host threads the oracle's OpenMP integrals use on this machine."""
    return int(os.environ.get("OMP_NUM_THREADS", os.cpu_count() or 1))


def run_reference(args, problem, blocks, rank):
    """The oracle on the bench workload, a bounded sample per step (rank 0
    only; under torchrun the other ranks exit without work)."""
    if rank != 0:
        return
    n_mo = mo_count(problem, len(blocks))
    smp = OracleSampler(problem, blocks)
    k = smp.calibrate(args.ref_budget)
    for _ in range(max(0, args.warmup - 1)):
        smp.sample(k)
    smp.reset()
    for _ in range(args.steps):
        smp.sample(k)
    t_full = smp.full_seconds()
    value = n_mo / t_full
    cores = oracle_threads()
    one = one_core_rate(smp, n_mo, k)
    cpu = {"value": value, "unit": "MO-integrals/s", "cores": cores, "kind": "oracle",
           "sample": smp.describe(k, cores), "value_1core": one}
    line = {"metric": METRIC, "value": value, "unit": "MO-integrals/s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": float(np.mean(smp.times)) * 1e3,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "impl": "reference",
            "config": config_dict(args, problem, blocks),
            "step": ("one bounded sample of the workload (see cpu_baseline.sample); value = MO integrals of one "
                     "whole transformation / its estimated time %.1f s" % t_full),
            "full_transform_s_est": t_full, "setup_s": smp.t_setup,
            "cpu_baseline": cpu,
            "e2e": {"value": value, "unit": "MO-integrals/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def one_core_rate(smp, n_mo, k):
    """One more sample (stride 4k) with the oracle's integrals on one host
    thread (oracle.set_threads) and numpy's BLAS on one thread where its
    library exposes the switch; the whole transformation's time is estimated
    from it as in OracleSampler.full_seconds, with the set-up (timed on all
    threads) scaled by the all-thread/one-thread ratio of the sample."""
    O = smp.O
    saved = (dict(smp.tsum), dict(smp.fsum), list(smp.times))
    t_all = float(np.mean(smp.times)) if smp.times else None
    try:
        O.set_threads(1)
    except Exception:
        return None
    blas = _blas_threads(1)
    try:
        smp.reset()
        smp.sample(4 * k)
        est = sum(smp.tsum[b] / smp.fsum[b] for b in smp.blocks if smp.fsum[b] > 0)
    finally:
        O.set_threads(oracle_threads())
        _blas_threads(os.cpu_count() or 1)
        smp.tsum, smp.fsum, smp.times = saved
    full_all = smp.full_seconds() - smp.t_setup
    ratio = est / full_all if full_all > 0 else 1.0
    return {"value": n_mo / (est + smp.t_setup * ratio), "unit": "MO-integrals/s",
            "sample": "one sample at stride %d, integrals on 1 thread, BLAS threads %s; set-up scaled by %.1f"
                      % (4 * k, "1" if blas else "unchanged", ratio), "all_thread_sample_s": t_all}


def _blas_threads(n):
    """Set numpy's OpenBLAS thread count through the loaded library, if found."""
    import ctypes
    try:
        with open("/proc/self/maps") as f:
            libs = sorted({ln.split()[-1] for ln in f if "openblas" in ln.lower() and ln.strip().endswith(".so")
                           or ("openblas" in ln.lower() and ".so" in ln)})
    except Exception:
        return False
    for path in libs:
        try:
            lib = ctypes.CDLL(path)
        except Exception:
            continue
        for name in ("openblas_set_num_threads", "scipy_openblas_set_num_threads64_",
                     "openblas_set_num_threads64_", "scipy_openblas_set_num_threads"):
            fn = getattr(lib, name, None)
            if fn is not None:
                fn(ctypes.c_int(n))
                return True
    return False


def dtype_of(fp64):
    if fp64:
        return "f64"
    return ("f32/f32-pair integrals, bf16x6-slice contractions (f32 exact chunks), "
            "f64 recombination and accumulation")


TRAFFIC_FILE = os.path.join(ROOT, "profiles", "traffic.txt")
ERI_SOURCE = os.path.join(ROOT, "paper_2606_04316_gb300", "csrc", "eri_kernels.cu")


def source_sha16(path):
    import hashlib
    with open(path, "rb") as f:
        return hashlib.sha256(f.read()).hexdigest()[:16]


def traffic_per_value(kind):
    """DRAM bytes per integral value of the integral kernel from the committed
    ncu capture (profiles/traffic.txt), or None when that file is absent or was
    taken on another version of the kernel source."""
    try:
        sha = source_sha16(ERI_SOURCE)
        with open(TRAFFIC_FILE) as f:
            for ln in f:
                if ln.startswith("#") or not ln.strip():
                    continue
                parts = ln.split()
                if parts[0] == kind and parts[1] == sha:
                    return float(parts[2]), " ".join(parts[3:])
    except Exception:
        pass
    return None, None


def roofline(st, avg, prec, clocks, pk, src, device, blocks):
    """Roofline of the dominant phase's kernel: algorithmic work per step over
    its measured time (CUDA events on the launching stream), against the
    measured peak of the unit it runs on."""
    from paper_2606_04316_gb300 import qdt
    dom = max(("ms_eri", "ms_half1", "ms_half2"), key=lambda k: avg[k])
    fp64_derived, mhz = fp64_alu_peak(clocks)
    try:
        p32, p64 = qdt.alu_peak(device, "fp32"), qdt.alu_peak(device, "fp64")
    except Exception:
        p32, p64 = None, None
    p32_derived = SMS * FP32_PER_CLK_SM * 2 * mhz * 1e6 / 1e12
    measured = {"fp32_fma_tflops": p32, "fp64_fma_tflops": p64, "how": "qdt_alu_peak (own FMA probe)",
                "fp32_derived_tflops": p32_derived, "fp64_derived_tflops": fp64_derived}
    nclass = (1 if "coulomb" in blocks else 0) + (1 if ("gaunt" in blocks or "gauge" in blocks) else 0)
    if dom == "ms_eri":
        achieved = st["flops_eri"] / (avg[dom] / 1e3) / 1e12
        if prec == qdt.SPLIT:
            # compensated FP32-pair multiply-adds cost 12 FP32 operations, the
            # quartets within the FP32 error budget one FMA: the bound weighs
            # the two by their share of the flops
            f32 = st.get("flops_eri_f32", 0.0) / st["flops_eri"] if st["flops_eri"] else 0.0
            ops = DF_OPS_PER_MADD * (1.0 - f32) + 1.0 * f32
            base = p32 if p32 else p32_derived
            peak = base / ops
            note = ("measured FP32 FMA rate %.1f TF/s / %.2f FP32 operations per multiply-add (%d for "
                    "compensated pairs, 1 for the %.1f %% of flops in plain FP32), FP64-equivalent flops"
                    % (base, ops, DF_OPS_PER_MADD, 100.0 * f32))
        else:
            peak = p64 if p64 else fp64_derived
            note = "measured FP64 FMA rate (qdt_alu_peak)"
        per_value, how = traffic_per_value("eri_rows_kernel")
        traffic = per_value * st["eri_values"] if per_value else None
        return {"kernel": "eri_rows_kernel", "bound": "alu", "achieved": achieved, "peak": peak,
                "unit": "TFLOP/s", "frac": achieved / peak, "traffic": traffic,
                "traffic_note": ("DRAM bytes of the step's integral launches: %s" % how) if how else
                "no capture of this kernel version",
                "launches_per_step": nclass, "peak_note": note, "peaks": measured,
                "work": "E R E multiply-adds of the kept quartets (qdt_stats.flops_eri), per step"}
    fl = st["flops_half1"] if dom == "ms_half1" else st["flops_half2"]
    achieved = fl / (avg[dom] / 1e3) / 1e12
    if prec == qdt.FP64:
        peak, note, bound = (p64 or fp64_derived), "measured FP64 FMA rate (qdt_alu_peak)", "alu"
    else:
        peak, note, bound = pk["bf16_tflops_sustained"], "%s bf16 sustained" % src, "tensor"
    return {"kernel": "half1" if dom == "ms_half1" else "half2", "bound": bound, "achieved": achieved,
            "peak": peak, "unit": "TFLOP/s", "frac": achieved / peak, "traffic": None,
            "peak_note": note, "peaks": measured}


METRIC = "DCB AO->MO transform MO-integrals/s (split vs FP64 @1e-10 Eh)"


WORKLOAD_NOTES = {
    "chain40-sp": "the 40-centre s+p chain (nL 160, nS 480, 40 Kramers pairs, Schwarz 1e-12) with the "
                  "Dirac-Coulomb-Breit blocks: the largest DCB workload whose 20 + 5 steps fit the bench's "
                  "minute of timed work; the 64-centre DCB cluster (nL 256, nK 64) takes 211 s per split "
                  "step (row batches; its first half alone is 5.0e15 FP64-equivalent flops) and is measured "
                  "separately (--workload cluster64-sp)",
}


def config_dict(args, problem, blocks):
    d = {"workload": args.workload, "nL": problem.basis.nL, "nS": problem.basis.nS,
         "n_kramers": problem.nK, "blocks": "+".join(blocks), "schwarz_tau": problem.tau,
         "precision": args.precision, "l2": "inputs larger than L2 (densities, integral rows)"}
    if args.workload in WORKLOAD_NOTES and len(blocks) == 3:
        d["why_this_workload"] = WORKLOAD_NOTES[args.workload]
    if getattr(args, "nk_active", 0) > 0 and args.nk_active < problem.nK:
        d["active_range"] = [0, args.nk_active]
    if getattr(args, "route", "density") != "density":
        d["route"] = args.route
        if args.route == "mo":
            d["mo_block"] = args.mo_block
    if not problem.kramers:
        del d["n_kramers"]
        d["n_spinors"] = problem.nK
        d["input"] = "kramers-unrestricted"
    return d


def serve_stream(reqs, prec, slots, seed_offset=3):
    """One request stream through the continuous-batching server: a sequential
    calibration pass (one qdt_transform after another on one context), then the
    same requests submitted on a seeded Poisson process at 0.8 x the calibrated
    capacity.  Latency = completion - submission (= arrival).  Returns the
    metrics and whether every result equals its sequential result."""
    from paper_2606_04316_gb300 import qdt
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
    print("serving: calibration of %d requests (%s) %.1f s" % (len(reqs), "split" if prec else "fp64", t_seq),
          file=sys.stderr, flush=True)
    rate = 0.8 * len(reqs) / t_seq
    rng = np.random.Generator(np.random.PCG64(synth.SEED_BASE + seed_offset))
    arrivals = np.cumsum(rng.exponential(1.0 / rate, size=len(reqs)))
    srv = qdt.Server(0, n_slots=slots)
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
    lat, failed = [], []
    for i, h in enumerate(handles):
        try:
            lat.append(srv.wait(h)[0])
        except qdt.QdtError as ex:          # reported, not fatal: the stream's other requests still count
            failed.append({"request": i, "error": str(ex)})
    makespan = time.perf_counter() - start
    srv.close()
    ok = [i for i in range(len(reqs)) if i not in {f["request"] for f in failed}]
    same = all(np.array_equal(outs[i], res[i]) for i in ok)
    n_mo = sum(mo_integrals(reqs[i].nK, len(reqs[i].blocks)) for i in ok)
    out = {"value": n_mo / makespan, "unit": "MO-integrals/s",
           "latency_s": {"p50": float(np.percentile(lat, 50)), "p99": float(np.percentile(lat, 99)),
                         "mean": float(np.mean(lat)), "max": float(np.max(lat))},
           "arrival_rate_per_s": rate, "calibration_sequential_s": t_seq,
           "sequential_value": sum(mo_integrals(p.nK, len(p.blocks)) for p in reqs) / t_seq,
           "makespan_s": makespan, "requests": len(reqs), "failed": failed,
           "results_same_alone_and_in_mix": same}
    print("serving: %s" % json.dumps(out), file=sys.stderr, flush=True)
    return out


def run_serving(args):
    """Request stream through the continuous-batching server (qdt_server_*):
    seeded chain/cluster requests (nL 24..200, nK 8..48, half Dirac-Coulomb
    and half Dirac-Coulomb-Breit, tau 1e-11), Poisson arrivals at 0.8 x the
    capacity of a sequential calibration pass; p50/p99 latency and
    MO-integrals/s in the split form over the whole stream, and both forms
    side by side over its first --compare-prefix requests."""
    import torch
    from paper_2606_04316_gb300 import qdt
    torch.cuda.set_device(0)
    prec = qdt.SPLIT if args.precision == "split" else qdt.FP64
    reqs = synth.serving_requests(args.requests, nl_range=(24, args.max_nl), nk_range=(8, args.max_nk))
    main = serve_stream(reqs, prec, args.slots)
    both = None
    if args.compare_prefix > 0:
        pre = reqs[:args.compare_prefix]
        both = {"requests": len(pre),
                "split": serve_stream(pre, qdt.SPLIT, args.slots, seed_offset=4),
                "fp64": serve_stream(pre, qdt.FP64, args.slots, seed_offset=4)}
        both["p99_fp64_over_split"] = both["fp64"]["latency_s"]["p99"] / both["split"]["latency_s"]["p99"]
        both["throughput_split_over_fp64"] = both["split"]["value"] / both["fp64"]["value"]
    line = {"metric": "serving: p50/p99 request latency and MO-integrals/s (continuous batching)",
            "value": main["value"], "unit": "MO-integrals/s", "n_gpus": 1, "higher_is_better": True,
            "latency_s": main["latency_s"], "precision": args.precision, "slots": args.slots,
            "stream": main, "both_forms_on_prefix": both, "data": "synthetic",
            "config": {"workload": "serving", "requests": len(reqs), "nL": [24, args.max_nl], "nK": [8, args.max_nk],
                       "blocks": "half coulomb, half coulomb+gaunt+gauge", "schwarz_tau": 1e-11,
                       "arrivals": "Poisson at 0.8 x the sequential capacity of each form"}}
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
    reqs = synth.serving_requests(args.batch_requests, nl_range=(24, args.batch_max_nl),
                                  nk_range=(8, args.batch_max_nk))
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
            "config": {"workload": "batch", "nL": [24, args.batch_max_nl], "nK": [8, args.batch_max_nk],
                       "blocks": "half coulomb, half coulomb+gaunt+gauge", "schwarz_tau": 1e-11}}
    print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=2)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="chain40-sp")
    ap.add_argument("--blocks", default="coulomb,gaunt,gauge",
                    help="the metric is Dirac-Coulomb-Breit: Coulomb + Gaunt + gauge blocks")
    ap.add_argument("--input", default="kramers", choices=["kramers", "ku"],
                    help="coefficients: quaternion (Kramers pairs) or Kramers-unrestricted spinors")
    ap.add_argument("--precision", default="split", choices=["split", "fp64"])
    ap.add_argument("--route", default="density", choices=["density", "quarter", "mo"],
                    help="density (AO-driven), quarter (O(N^5) Coulomb first half) or mo (MO-driven comparator)")
    ap.add_argument("--mo-block", type=int, default=8, help="MO-driven route: outer MO indices per block")
    ap.add_argument("--fp64-steps", type=int, default=3, help="timed steps of the FP64 form (0: skip)")
    ap.add_argument("--fp64-warmup", type=int, default=1, help="untimed steps of the FP64 form before them")
    ap.add_argument("--e2e-calls", type=int, default=5, help="calls of the end-to-end (host buffers) timing")
    ap.add_argument("--nk-active", type=int, default=0,
                    help="transform only the first N units of the active range (0: all); AO work unchanged")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--cpu-samples", type=int, default=2, help="oracle samples of the cpu_baseline leg")
    ap.add_argument("--ref-budget", type=float, default=4.0, help="seconds of one oracle sample")
    ap.add_argument("--stats", action="store_true", help="print per-phase statistics to stderr")
    ap.add_argument("--requests", type=int, default=256, help="serving workload: number of requests")
    ap.add_argument("--slots", type=int, default=4, help="serving workload: concurrent contexts")
    ap.add_argument("--max-nl", type=int, default=200, help="serving workload: largest nL")
    ap.add_argument("--max-nk", type=int, default=48, help="serving workload: largest nK")
    ap.add_argument("--batch-requests", type=int, default=32, help="batch workload: number of requests")
    ap.add_argument("--batch-max-nl", type=int, default=64, help="batch workload: largest nL")
    ap.add_argument("--batch-max-nk", type=int, default=16, help="batch workload: largest nK")
    ap.add_argument("--compare-prefix", type=int, default=32,
                    help="serving workload: requests of the stream's start run in both forms side by side")
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
    nK = problem.nK if args.nk_active <= 0 else min(args.nk_active, problem.nK)
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
    n_mo = mo_count(problem, len(blocks)) * (float(nK) / problem.nK) ** 4
    value = job_value(n_mo, world, ms)

    # end to end through the public API with host buffers (pinned): coefficients
    # in and packed integrals out, copies inside the timed region; median of calls
    e2e = None
    if not args.no_e2e:
        CLh = torch.from_numpy(problem.CL).pin_memory()
        CSh = torch.from_numpy(problem.CS).pin_memory()
        outh = torch.zeros(nout, dtype=torch.float64).pin_memory()
        torch.cuda.synchronize()
        dts = []
        for _ in range(max(1, args.e2e_calls)):
            t0 = time.perf_counter()
            set_coefs(CLh, CSh)
            ctx.transform(blocks, 0, nK, tau, prec, outh)
            dts.append(time.perf_counter() - t0)
        dt = float(np.median(dts))
        e2e = {"value": n_mo * world / dt, "unit": "MO-integrals/s",
               "h2d_bytes_per_step": int(CLh.numel() * 8 + CSh.numel() * 8),
               "d2h_bytes_per_step": int(outh.numel() * 8), "calls": len(dts),
               "timing": "median host wall clock of qdt_set_coefficients + qdt_transform with pinned host buffers"}

    # the FP64 form on the same workload, and the agreement of the two forms
    # (after --fp64-warmup untimed FP64 steps; `out` still holds the last timed
    # split result, compared with the last FP64 one)
    other = None
    if prec == qdt.SPLIT and args.fp64_steps > 0:
        out64 = torch.zeros_like(out)
        set_coefs(CLd, CSd)
        for _ in range(args.fp64_warmup):
            ctx.transform(blocks, 0, nK, tau, qdt.FP64, out64)
        torch.cuda.synchronize()
        f0 = torch.cuda.Event(enable_timing=True)
        f1 = torch.cuda.Event(enable_timing=True)
        f0.record(stream)
        for _ in range(args.fp64_steps):
            st64 = ctx.transform(blocks, 0, nK, tau, qdt.FP64, out64)
        f1.record(stream)
        torch.cuda.synchronize()
        diff = float((out - out64).abs().max().item())
        ms64 = f0.elapsed_time(f1) / args.fp64_steps
        other = {"value": n_mo * world / (ms64 / 1e3), "ms_per_step": ms64, "steps": args.fp64_steps,
                 "warmup": args.fp64_warmup, "phases_ms": {k: st64[k] for k in phase},
                 "max_abs_diff_split_vs_fp64": diff, "split_speedup": ms64 / ms,
                 "quartets_kept": st64["quartets_kept"], "flops_eri": st64["flops_eri"]}

    pk, src = peaks()
    avg = {k: v / args.steps for k, v in phase.items()}
    roof = roofline(st, avg, prec, clocks, pk, src, local, blocks)

    cpu = None
    if rank == 0 and not args.no_cpu:
        try:
            smp = OracleSampler(problem, blocks)
            k = smp.calibrate(args.ref_budget)
            for _ in range(args.cpu_samples):
                smp.sample(k)
            cores = oracle_threads()
            cpu = {"value": n_mo / smp.full_seconds(), "unit": "MO-integrals/s", "cores": cores,
                   "kind": "oracle", "sample": smp.describe(k, cores),
                   "value_1core": one_core_rate(smp, n_mo, k)}
        except Exception as ex:  # keep the bench line even if the oracle fails
            cpu = {"value": None, "unit": "MO-integrals/s", "cores": os.cpu_count(), "kind": "oracle",
                   "sample": "failed: %s" % ex}

    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": "MO-integrals/s", "n_gpus": world,
                "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": dtype_of(prec == qdt.FP64),
                "data": "synthetic", "config": config_dict(args, problem, blocks), "clocks": clocks,
                "e2e": e2e, "gpu_launches": launches, "roofline": roof, "cpu_baseline": cpu,
                "phases_ms": avg, "quartets_kept": st["quartets_kept"], "quartets_total": st["quartets_total"],
                "quartets_f32": st["quartets_f32"],
                "eri_values_per_s": st["eri_values"] / (avg["ms_eri"] / 1e3) if avg["ms_eri"] > 0 else None,
                "fp64_form": other}
        print(json.dumps(line), flush=True)
        if args.stats:
            print(json.dumps(st), file=sys.stderr)
    ctx.close()
    if world > 1:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
