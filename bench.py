#!/usr/bin/env python
"""Benchmark: FETI solves/s at relative nodal error 1e-8, with p50/p99 latency, on one GB300.

Headline workload (the largest single-GPU one): 2-D bond-based peridynamics, micromodulus
3/delta^3 xi xi^T/|xi|^3 on the l2 ball (nocaps polygon), delta = 3h, structured P1 triangles
h = 1/256 (130 050 unknowns, 2 per node), 8 x 8 subdomains with seeded jittered cuts, 36 of
them floating with 3 rigid modes each, 16 right-hand sides of seeded i.i.d. N(0,1) loads.
A step is one FETI solve request of the 16 right-hand sides with the subdomain operators
resident (setup and factorization excluded, the protocol of the paper's timings; both are
reported under "cold"): reduced forcing, projected PCG with the scaled Dirichlet
preconditioner, FP64 refinement of the FP32 operators until the relative nodal correction (or
the remaining error it predicts) is below 1e-9, back substitution and nodal output.  "value"
is right-hand-side solves per second with the loads resident in HBM; "e2e" is the same
through the C ABI with pinned host buffers (host<->device copies inside the timed region).
The 2-D fractional (64 RHS) and constant-kernel (8 RHS) workloads are reported beside it
("other_workloads"); --workload selects another headline.

--impl reference times the FP64 CPU oracle (one-level FETI in numpy, Algorithm 1) on the
host cores on a bounded sample of the same workload (its per-iteration subdomain work on a
few subdomains, scaled to a whole solve).  Under torchrun (N > 1) every rank solves its own
replica (no collective in the data path).

--serving runs the serving scenario instead: requests drawn from a pool of factored problems
(kernels, mesh sizes, horizons and decompositions sampled from a grid) arrive as a Poisson
process at the server; it reports solves/s, arrival -> result latency p50/p99 and a sweep of
the arrival rate.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import workloads as W  # noqa: E402

METRIC = "FETI solves/sec at rel. error 1e-8 + p50/p99 latency: batched mixed vs plain FP64, 1 GB300"

# The workloads (synthetic stand-ins for the paper's manufactured problems, Sec. 6.2): the
# headline is the largest single-GPU one, the peridynamic problem; the others are reported
# beside it.
WORKLOADS = {
    "peridynamic_2d": (
        lambda **kw: W.peridynamic_2d(**kw),
        "2-D bond-based peridynamics, micromodulus 3/delta^3 xi xi^T/|xi|^3 on the l2 ball (nocaps), "
        "delta=3h, h=1/256 (130050 dofs, 2 per node), 8x8 subdomains with seeded jittered cuts "
        "(+-20%, seed 4), 16 RHS N(0,1) loads per dof (seed 5)"),
    "fractional_2d": (
        lambda **kw: W.fractional_2d(**kw),
        "2-D fractional kernel (2-2s)/(pi delta^(2-2s)) |x-y|^-(2+2s), s=0.5, truncated at delta=0.2, "
        "h=1/96 (9025 dofs), 6x6 subdomains (Omega_k empty on the interior ones), 64 RHS N(0,1) loads (seed 3)"),
    "const_l2_2d": (
        lambda **kw: W.const_l2_2d(**kw),
        "2-D nonlocal diffusion, constant kernel 4/(pi delta^4) on the l2 ball (nocaps), delta=0.1, "
        "h=1/128 (16129 dofs), 4x4 subdomains, 8 RHS N(0,1) loads (seed 2)"),
}
HEADLINE = "peridynamic_2d"


def config_dict(name, w, n_lambda, n_u, world):
    """The workload's config, identical for both arms (built from the inputs and the
    decomposition sizes only)."""
    free = int((w.mesh.node_is_dirichlet == 0).sum()) * w.kernel.ncomp
    return {"workload": WORKLOADS[name][1], "name": name, "global_batch": w.nrhs * world,
            "rhs_per_request": w.nrhs, "n_dofs": free, "subdomains": int(w.K), "n_lambda": int(n_lambda),
            "n_u": int(n_u),
            "step": "one warm solve request of all its right-hand sides (subdomain operators resident; "
                    "setup and factorization excluded)",
            "l2": "subdomain operators exceed the 126 MB L2; no flush between steps"}


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


def dist_env():
    return int(os.environ.get("RANK", 0)), int(os.environ.get("WORLD_SIZE", 1)), int(os.environ.get("LOCAL_RANK", 0))


def max_over_ranks(x, world, device=None):
    """The largest of a per-rank time (every rank gets it); the identity on one rank."""
    if world <= 1:
        return float(x)
    import torch
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
    return float(t.item())


def replica_throughput(units_per_rank, world, slowest_s):
    """Whole-job throughput of independent replicas: the units all ranks processed over the
    time of the slowest rank."""
    return world * units_per_rank / slowest_s


class ClockSampler:
    """nvidia-smi clock and throttle samples during the timed region."""

    def __init__(self, gpu_index):
        self.f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
        q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
        try:
            self.p = subprocess.Popen(["nvidia-smi", "-i", str(gpu_index), f"--query-gpu={q}", "--format=csv,noheader,nounits",
                                       "-lms", "200"], stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.p = None

    def stop(self):
        if self.p is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        time.sleep(0.25)
        self.p.terminate()
        try:
            self.p.wait(timeout=5)
        except Exception:
            self.p.kill()
        self.f.flush()
        self.f.seek(0)
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in self.f.read().splitlines():
            parts = [x.strip() for x in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for n, v in zip(names, parts[5:9]):
                if v.lower() in ("active", "1"):
                    reasons.add(n)
        os.unlink(self.f.name)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "samples": len(sm), "reasons": sorted(reasons)}


def percentile(xs, q):
    xs = sorted(xs)
    if not xs:
        return None
    k = (len(xs) - 1) * q
    lo, hi = int(np.floor(k)), int(np.ceil(k))
    return xs[lo] + (xs[hi] - xs[lo]) * (k - lo)


def profile_traffic(kernel_src_hash, name="k_apply_tma_peridynamic_2d.md"):
    """DRAM bytes per launch of an apply kernel from the committed ncu summary, if it matches
    the current kernel source (else None)."""
    path = os.path.join(ROOT, "profiles", name)
    try:
        txt = open(path).read()
    except OSError:
        return None
    val, h = None, None
    for line in txt.splitlines():
        if line.startswith("traffic_bytes_per_launch:"):
            val = float(line.split(":", 1)[1])
        if line.startswith("kernel_source_sha256:"):
            h = line.split(":", 1)[1].strip()
    return val if (val is not None and h == kernel_src_hash) else None


def kernel_source_hash(name="apply_tma.cuh"):
    with open(os.path.join(ROOT, "paper_2306_00094_gb300", "csrc", name), "rb") as f:
        return hashlib.sha256(f.read()).hexdigest()[:16]


# ------------------------------------------------------------------------------------------ ours

def timed_solves(torch, prob, opt, d_rhs, kind, d_out, R, steps):
    """CUDA-event times of `steps` warm solve requests with the given options (one untimed
    solve first): solves/s, mean / p50 / p99 ms, PCG iterations and refinement sweeps."""
    prob.set_options(opt)
    prob.solve_device(d_rhs, kind, d_out, nrhs=R)
    torch.cuda.synchronize()
    ts = []
    s = None
    for _ in range(steps):
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        a.record()
        s = prob.solve_device(d_rhs, kind, d_out, nrhs=R)
        b.record()
        torch.cuda.synchronize()
        ts.append(a.elapsed_time(b))
    return {"value": R * len(ts) / (sum(ts) / 1e3), "unit": "solves/s", "ms_per_step": statistics.mean(ts),
            "p50_ms": percentile(ts, 0.5), "p99_ms": percentile(ts, 0.99), "iterations": s["iterations"],
            "refine_sweeps": s["refine_sweeps"]}


def apply_rooflines(torch, prob, step, steps, hbm, peak_kind):
    """The dense interface applies' achieved bandwidth: the same steps again with CUDA events
    around every apply launch on the library stream (the PCG loops then run in event-timed
    graph chunks, since a device-side WHILE graph cannot hold event nodes).  Returns the
    S_k^+ apply (FP32 operator) and the preconditioner's S_k apply (FP16 copy), each with its
    share of the profiled steps' time."""
    prob.profile()
    prob.set_profiling(True)
    pa = torch.cuda.Event(enable_timing=True)
    pb = torch.cuda.Event(enable_timing=True)
    pa.record()
    for _ in range(steps):
        step()
    pb.record()
    torch.cuda.synchronize()
    prof_ms = pa.elapsed_time(pb)
    prob.set_profiling(False)
    prof = prob.profile()
    out = {}
    for key in ("apply", "half_apply"):
        n, ms, b = prof[key + "_launches"], prof[key + "_ms"], prof[key + "_bytes"]
        if n > 0 and ms > 0:
            bpl, avg = b / n, ms / n / 1e3
            out[key] = {"bound": "hbm", "achieved": bpl / avg / 1e9, "peak": hbm, "unit": "GB/s",
                        "frac": bpl / avg / 1e9 / hbm, "peak_source": peak_kind, "bytes_per_launch": bpl,
                        "avg_launch_us": avg * 1e6, "launches": n, "share_of_step_time": ms / prof_ms}
        else:
            out[key] = None
    return out


def run_ours(args):
    import torch
    from paper_2306_00094_gb300 import binding

    rank, world, local = dist_env()
    if world > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    dev = torch.device("cuda", torch.cuda.current_device())
    name = args.workload
    w = WORKLOADS[name][0](**({"N": args.cells} if args.cells else {}))
    R = w.nrhs
    ctx = binding.Context()
    t0 = time.perf_counter()
    prob = binding.Problem.from_workload(ctx, w)
    t_setup = time.perf_counter() - t0
    t0 = time.perf_counter()
    prob.factor(2)
    t_factor32 = time.perf_counter() - t0
    t0 = time.perf_counter()
    prob.factor(1)
    t_factor64 = time.perf_counter() - t0
    info = prob.info()
    ndof = prob.n_dofs
    # the apply shapes for R right-hand sides, tuned on this GPU (choices cached per device and
    # subdomain shapes in the build folder)
    t0 = time.perf_counter()
    tuned = prob.autotune(R, os.path.join(ROOT, "paper_2306_00094_gb300", "_build", "apply_tune.json"))
    t_tune = time.perf_counter() - t0
    # inputs resident in HBM: column-major n_dofs x R  ==  contiguous (R, n_dofs)
    d_rhs = torch.from_numpy(np.ascontiguousarray(w.rhs.T)).to(dev)
    d_out = torch.empty_like(d_rhs)
    mixed = binding.default_options(precision=1, batched=1, graph_loop=0 if args.host_loop else 1,
                                    precond_fp16=2 if args.tensor_core_precond else 1)
    plain = binding.default_options(precision=0, batched=0)
    plain_batched = binding.default_options(precision=0, batched=1)

    def step():
        return prob.solve_device(d_rhs, w.rhs_kind, d_out, nrhs=R)

    prob.set_options(mixed)
    # the clock sampler (nvidia-smi) starts before the warm-up: its start-up initialises NVML,
    # which stalled a timed step by about 140 ms when it started right before the timed region
    sampler = ClockSampler(local) if not (args.profile_range or args.only_timed or args.cells) else None
    time.sleep(0.5)
    for _ in range(args.warmup):
        st = step()
    torch.cuda.synchronize()
    if args.profile_range == "factor":
        # one FP32 factorization inside a CUDA profiler range (ncu --profile-from-start off)
        torch.cuda.profiler.start()
        prob.factor(2)
        torch.cuda.synchronize()
        torch.cuda.profiler.stop()
        if rank == 0:
            print(json.dumps({"note": "one FP32 factorization in the profiler range", "workload": name,
                              "cells": args.cells}), flush=True)
        return
    prob.profile()                       # reset counters
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps + 1)]
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    if args.profile_range == "solve":
        torch.cuda.profiler.start()
    ev[0].record()
    stats = []
    for k in range(args.steps):
        stats.append(step())
        ev[k + 1].record()
    torch.cuda.synchronize()
    if args.profile_range == "solve":
        torch.cuda.profiler.stop()
    if world > 1:
        torch.distributed.barrier()
    clocks = sampler.stop() if sampler else {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["not sampled (profiling run)"]}
    launches = prob.profile()["kernel_launches"]
    lat = [ev[k].elapsed_time(ev[k + 1]) for k in range(args.steps)]
    total_ms = max_over_ranks(ev[0].elapsed_time(ev[-1]), world, dev)
    value = replica_throughput(R * args.steps, world, total_ms / 1e3)
    u_gpu = d_out.cpu().numpy().T.copy()

    if args.only_timed or args.cells:
        if rank == 0:
            print(json.dumps({"metric": METRIC, "value": value, "unit": "solves/s", "ms_per_step": total_ms / args.steps,
                              "gpu_launches": launches, "workload": name, "cells": args.cells,
                              "note": "timed steps only (a profiling run, not a bench line)"}), flush=True)
        return

    # roofline of the dominant kernels (dense interface applies) over a second timed region
    hbm, peak_kind = peaks()
    roof = apply_rooflines(torch, prob, step, args.steps, hbm, peak_kind)
    ap, hp = roof["apply"], roof["half_apply"]
    if ap:
        ap.update({"kernel": "k_apply_tma<float> (dense S_k^+ apply, FP32, tensor-copy pipeline)",
                   "timing": "CUDA events around each apply launch over a second timed region of the same "
                             f"{args.steps} steps",
                   "traffic": profile_traffic(kernel_source_hash(), f"k_apply_tma_{name}.md")})
    if hp:
        tc_pre = any(e["kind"] == 1 and e["rc"] == -1 for e in tuned) or args.tensor_core_precond
        if tc_pre:
            hp.update({"kernel": "k_apply_mma (preconditioner S_k apply on the tensor cores: tcgen05 kind::f16, "
                                 "FP16 copy, FP32 accumulators in tensor memory)",
                       "traffic": profile_traffic(kernel_source_hash("apply_mma.cuh"), f"k_apply_mma_{name}.md")})
        else:
            hp.update({"kernel": "k_apply_tma<float, .., __half> (preconditioner S_k apply, FP16 copy)",
                       "traffic": profile_traffic(kernel_source_hash(), f"k_apply_tma_fp16_{name}.md")})

    # end to end through the C ABI with pinned host buffers
    h_rhs = torch.empty((R, ndof), dtype=torch.float64, pin_memory=True)
    h_rhs.copy_(torch.from_numpy(np.ascontiguousarray(w.rhs.T)))
    h_out = torch.empty((R, ndof), dtype=torch.float64, pin_memory=True)
    for _ in range(max(1, args.warmup // 2)):
        prob.solve_host_ptr(h_rhs.data_ptr(), w.rhs_kind, h_out.data_ptr(), R)
    if world > 1:
        torch.distributed.barrier()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        prob.solve_host_ptr(h_rhs.data_ptr(), w.rhs_kind, h_out.data_ptr(), R)
    e2e_s = max_over_ranks(time.perf_counter() - t0, world, dev)
    e2e = {"value": replica_throughput(R * args.steps, world, e2e_s), "unit": "solves/s",
           "h2d_bytes_per_step": 8 * R * ndof,
           "d2h_bytes_per_step": 8 * R * ndof}

    # baselines on the GPU: plain FP64 one subdomain at a time (no graphs), and FP64 batched
    ksteps = max(3, min(args.steps, 5))
    plain_res = timed_solves(torch, prob, plain, d_rhs, w.rhs_kind, d_out, R, 2)
    u_plain = d_out.cpu().numpy().T.copy()
    plain_b_res = timed_solves(torch, prob, plain_batched, d_rhs, w.rhs_kind, d_out, R, ksteps)
    # the mixed solve with the preconditioner's S_k apply on the tensor cores (tcgen05 MMAs on
    # the FP16 copy and FP16 x, FP32 accumulators in tensor memory)
    tc_res = timed_solves(torch, prob, binding.default_options(precision=1, batched=1, precond_fp16=2),
                          d_rhs, w.rhs_kind, d_out, R, ksteps)

    # the paper's baseline solver on the same GPU and inputs: diagonally preconditioned CG on
    # the single-domain system (FP64-accurate products), tol 1e-10
    t0 = time.perf_counter()
    prob.cg_prepare()
    cg_prep_s = time.perf_counter() - t0
    d_cg = torch.empty_like(d_rhs)
    prob.set_options(binding.default_options(tol=1e-10, max_it=20000))

    def cg_all():
        # the CG entry point takes at most 32 right-hand sides per call
        st = None
        for c0 in range(0, R, 32):
            c1 = min(R, c0 + 32)
            st = prob.solve_cg_device(d_rhs[c0:c1], w.rhs_kind, d_cg[c0:c1], nrhs=c1 - c0)
        return st

    cg_all()
    torch.cuda.synchronize()
    ts = []
    for _ in range(2):
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        a.record()
        s_cg = cg_all()
        b.record()
        torch.cuda.synchronize()
        ts.append(a.elapsed_time(b))
    u_cg = d_cg.cpu().numpy().T.copy()
    cg_res = {"value": R * len(ts) / (sum(ts) / 1e3), "unit": "solves/s", "ms_per_step": statistics.mean(ts),
              "iterations": s_cg["iterations"], "tol": 1e-10, "prepare_s": cg_prep_s,
              "rel_diff_vs_fp64_feti": rel_diff(u_cg, u_plain, w)}
    prob.set_options(mixed)

    # cold: setup + assembly + FP32 factorization + one solve
    torch.cuda.synchronize()
    prob.close()
    t0 = time.perf_counter()
    prob2 = binding.Problem.from_workload(ctx, w)
    prob2.factor(2)
    prob2.set_options(mixed)
    prob2.solve_device(d_rhs, w.rhs_kind, d_out, nrhs=R)
    torch.cuda.synchronize()
    cold_s = time.perf_counter() - t0
    prob2.close()
    del d_cg

    # the other workloads, warm: mixed (with the apply rooflines) and the two FP64 baselines
    others = {}
    for oname in WORKLOADS:
        if oname == name or args.headline_only:
            continue
        ow = WORKLOADS[oname][0]()
        op = binding.Problem.from_workload(ctx, ow)
        op.factor(3)
        op.autotune(ow.nrhs, os.path.join(ROOT, "paper_2306_00094_gb300", "_build", "apply_tune.json"))
        od_rhs = torch.from_numpy(np.ascontiguousarray(ow.rhs.T)).to(dev)
        od_out = torch.empty_like(od_rhs)
        res = {"workload": WORKLOADS[oname][1]}
        res["mixed"] = timed_solves(torch, op, mixed, od_rhs, ow.rhs_kind, od_out, ow.nrhs, ksteps)
        oroof = apply_rooflines(torch, op, lambda: op.solve_device(od_rhs, ow.rhs_kind, od_out, nrhs=ow.nrhs),
                                ksteps, hbm, peak_kind)
        res["roofline_apply"] = oroof["apply"]
        res["roofline_precond"] = oroof["half_apply"]
        res["plain_fp64_per_subdomain"] = timed_solves(torch, op, plain, od_rhs, ow.rhs_kind, od_out, ow.nrhs, 2)
        res["fp64_batched"] = timed_solves(torch, op, plain_batched, od_rhs, ow.rhs_kind, od_out, ow.nrhs, 3)
        others[oname] = res
        op.close()
        del od_rhs, od_out

    # the same size as the 2-D constant-kernel workload on an unstructured mesh (irregular
    # nodes and diagonals) with 16 graph-grown local parts: warm mixed solves
    unstr_res = None
    if not args.headline_only:
        wu = W.unstructured_l2(N=128, K=16, nrhs=8, delta=0.1, seed=11)
        pu = binding.Problem.from_workload(ctx, wu)
        pu.factor(2)
        du_rhs = torch.from_numpy(np.ascontiguousarray(wu.rhs.T)).to(dev)
        du_out = torch.empty_like(du_rhs)
        unstr_res = timed_solves(torch, pu, mixed, du_rhs, wu.rhs_kind, du_out, wu.nrhs, ksteps)
        inf_u = pu.info()
        unstr_res.update({"n_dofs": int((wu.mesh.node_is_dirichlet == 0).sum()), "subdomains": inf_u["K"],
                          "n_lambda": inf_u["n_lambda"],
                          "workload": "constant l2 kernel, delta=0.1, 128 x 128 cells with irregular nodes "
                                      "(+-0.15 h) and diagonals, 16 graph-grown local parts, 8 RHS N(0,1)"})
        pu.close()

    # the serving stream through the server: batched mixed vs plain FP64 one subdomain at a time
    serving = None
    if not args.headline_only and world == 1:
        serving = serving_compare(ctx, binding, args)

    line = {
        "metric": METRIC, "value": value, "unit": "solves/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": total_ms / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32 operators and PCG iterations + f64 refinement", "data": "synthetic",
        "config": config_dict(name, w, info["n_lambda"], info["n_u"], world),
        "parallelism": f"replicas x{world}",
        "latency_ms": {"p50": percentile(lat, 0.5), "p99": percentile(lat, 0.99)},
        "iterations": stats[-1]["iterations"], "refine_sweeps": stats[-1]["refine_sweeps"],
        "roofline": ap,
        "roofline_precond": hp,
        "gpu_launches": launches,
        "e2e": e2e,
        "plain_fp64_per_subdomain": plain_res,
        "fp64_batched": plain_b_res,
        "precond_tensor_cores": tc_res,
        "cg_single_domain": cg_res,
        "cold": {"setup_assembly_s": t_setup, "factor_fp32_s": t_factor32, "factor_fp64_s": t_factor64,
                 "setup_factor_solve_s": cold_s},
        "autotune": {"seconds": t_tune, "choices": [
            {"operator": ["FP32 S_k^+ / S_k", "FP16 copy of S_k", "FP64 S_k^+ / S_k"][e["kind"]],
             "rhs_per_pass": e["rc"], "ctas_per_sm": e["ctas_per_sm"], "rows_per_warp": e["rows_per_warp"],
             "us_per_launch": e["us"],
             "from_cache": bool(e["from_cache"])} for e in tuned]},
        "other_workloads": others,
        "unstructured": unstr_res,
        "serving": serving,
        "clocks": clocks,
    }
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"], line["rel_err_vs_oracle"] = cpu_baseline(name, w, args, {
            "mixed": u_gpu, "plain_fp64": u_plain, "cg_single_domain": u_cg})
    if rank == 0:
        print(json.dumps(line), flush=True)
    if world > 1:
        torch.distributed.destroy_process_group()


# ------------------------------------------------------------------------------------- oracle

def rel_diff(u, v, w):
    """max over right-hand sides of max |u - v| / max |v| on the non-Dirichlet dofs"""
    free = np.repeat(w.mesh.node_is_dirichlet == 0, w.kernel.ncomp)
    d = np.abs(u[free] - v[free]).max(axis=0)
    s = np.abs(v[free]).max(axis=0)
    return float((d / np.where(s > 0, s, 1.0)).max())


# PCG iterations of the oracle's FETI (Algorithm 1, FP64, tolerance 1e-10) on each workload,
# from `python -m oracle.feti_iterations <workload>` (the oracle alone): they scale the
# oracle's sampled per-iteration time to a whole solve.
ORACLE_ITERATIONS = {"peridynamic_2d": 58, "fractional_2d": 32, "const_l2_2d": 26}
ORACLE_SAMPLE_SUBDOMAINS = 4


class OracleSample:
    """The FP64 oracle's solve-phase work on a fixed sample of subdomains, for timing on the
    host cores: a full oracle FETI solve of the large workloads takes many minutes (its setup
    alone assembles and factors every subdomain), so a step times the oracle's per-iteration
    subdomain work -- S_k^+ (pinned Neumann solve, Sec. 5.3) and S_k (Dirichlet solve,
    eq. subSchurComplement) applied to all right-hand sides -- on m evenly spaced subdomains,
    and a whole solve is estimated as (K / m) x (PCG iterations + 2) such steps (the forcing
    and the back substitution cost about one iteration each; the Lambda-space work is not
    counted, which favours the oracle)."""

    def __init__(self, name, w, m=ORACLE_SAMPLE_SUBDOMAINS):
        from oracle import assembly, feti
        from oracle.decomposition import build_decomposition
        self.w, self.name = w, name
        dec = build_decomposition(w.mesh, w.kernel, w.labels, w.K)
        self.K = dec.K
        self.ks = sorted({int(round(i * (dec.K - 1) / max(1, m - 1))) for i in range(m)})
        nc = w.kernel.ncomp
        self.ops, self.x = [], []
        rng = np.random.default_rng(0)
        for k in self.ks:
            dofs = dec.dofs(k)
            dof_of = np.full(w.mesh.n_nodes * nc, -1, dtype=np.int32)
            dof_of[dofs] = np.arange(dofs.size, dtype=np.int32)
            Ak, _ = assembly.assemble(w.mesh, w.kernel, w.kernel.scale, dof_of, dofs.size, elem_mask=dec.elem_mask, k=k)
            Zk = dec.Z[dec.u_offset[k]:dec.u_offset[k + 1], dec.coarse_offset[k]:dec.coarse_offset[k + 1]]
            op = feti.SubdomainOps(Ak, dec.n_omega(k), dec.subs[k].pinned, Zk if Zk.shape[1] else None)
            self.ops.append(op)
            self.x.append(rng.standard_normal((op.nG, w.nrhs)))
        self.n_lambda, self.n_u = dec.n_lambda, dec.n_u

    def step(self):
        for op, x in zip(self.ops, self.x):
            op.S_plus(x)
            op.S(x)

    def solves_per_s(self, step_s):
        its = ORACLE_ITERATIONS[self.name]
        return self.w.nrhs / (step_s * (self.K / len(self.ks)) * (its + 2))

    def describe(self, nsteps):
        return (f"{nsteps} steps of the oracle's per-iteration subdomain work (S_k^+ and S_k applied to the "
                f"{self.w.nrhs} right-hand sides) on subdomains {self.ks} of {self.K}, scaled by K/m = "
                f"{self.K / len(self.ks):g} and by the oracle's {ORACLE_ITERATIONS[self.name]} PCG iterations + 2 "
                f"(forcing, back substitution); oracle setup excluded, Lambda-space work not counted")


def cpu_baseline(name, w, args, results):
    """The FP64 oracle as it stands, on the host cores (a bounded sample, ~10-20 s), and the
    GPU results' relative nodal error against the oracle's single-domain solve."""
    from oracle import problem as oprob
    samp = OracleSample(name, w)
    samp.step()
    t0 = time.perf_counter()
    n = 0
    while n < 3 or (time.perf_counter() - t0 < 10.0 and n < 50):
        samp.step()
        n += 1
    dt = (time.perf_counter() - t0) / n
    cores = os.cpu_count()
    base = {"value": samp.solves_per_s(dt), "unit": "solves/s", "cores": cores, "kind": "oracle",
            "sample": samp.describe(n) + f"; numpy/LAPACK FP64 on {cores} host threads"}
    ref = oprob.Monolithic(w.mesh, w.kernel).solve(w.rhs, w.rhs_kind)
    acc = {k: float(oprob.rel_nodal_error(u, ref, w.mesh, w.kernel.ncomp).max()) for k, u in results.items()}
    acc["reference"] = "oracle single-domain FP64 solve (banded LAPACK Cholesky), every right-hand side"
    return base, acc


def run_reference(args):
    rank, world, _ = dist_env()
    if rank != 0:
        return
    name = args.workload
    w = WORKLOADS[name][0]()
    samp = OracleSample(name, w)
    for _ in range(min(args.warmup, 1)):
        samp.step()
    ts = []
    for _ in range(args.steps):
        t0 = time.perf_counter()
        samp.step()
        ts.append(time.perf_counter() - t0)
    step_s = sum(ts) / len(ts)
    value = samp.solves_per_s(step_s)
    scale = value * step_s / w.nrhs                     # whole-solve time = step time / scale
    cores = os.cpu_count()
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "solves/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * step_s,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": config_dict(name, w, samp.n_lambda, samp.n_u, world),
            "parallelism": "host cores",
            "latency_ms": {"p50": 1e3 * percentile(ts, 0.5) / scale, "p99": 1e3 * percentile(ts, 0.99) / scale,
                           "note": "estimated whole-solve latency from the sampled steps"},
            "cpu_baseline": {"value": value, "unit": "solves/s", "cores": cores, "kind": "oracle",
                             "sample": samp.describe(len(ts))},
            "e2e": {"value": value, "unit": "solves/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# ------------------------------------------------------------------------------------------ serving

def serving_pool(rng, size, budget_bytes, cost_cap):
    """Problem configurations of the serving scenario, sampled uniformly from the grid
    kernel x h x delta x K, rejecting those whose subdomains exceed 8k dofs, whose footprint
    exceeds the budget or whose assembly would cost more than cost_cap (element pairs)."""
    kinds = ["1d_const", "2d_const_l2", "2d_fractional"]
    pool, seen, tried, rejected = [], set(), 0, 0
    while len(pool) < size and tried < 5000:
        tried += 1
        kind = kinds[rng.integers(3)]
        N = [64, 128, 256][rng.integers(3)]
        di, ki = int(rng.integers(3)), int(rng.integers(5))
        if kind == "1d_const":
            N *= 10
            K = [4, 8, 16, 32, 64][ki]
            h = 1.0 / N
            delta = [2 * h, 3 * h, 0.1][di]
            e = int(np.ceil(delta / (2 * h) - 1e-9))
            nk = N // K + 2 * e + 1
            foot = K * nk * nk * 28
            cost = N * 2 * delta / h
        else:
            k = [2, 3, 4, 6, 8][ki]
            K = k * k
            h = 1.0 / N
            delta = [2 * h, 3 * h, 0.1][di]
            e = int(np.ceil(delta / (2 * h) - 1e-9))
            nk = (N // k + 2 * e + 1) ** 2
            foot = K * nk * nk * 28
            cost = 2 * (N + 2 * W.collar_cells(delta, N)) ** 2 * np.pi * (delta / h) ** 2
        key = (kind, N, di, K)
        if nk > 8000 or foot > budget_bytes or cost > cost_cap:
            rejected += 1
            continue
        if key in seen:
            continue
        seen.add(key)
        pool.append({"kernel": kind, "N": N, "delta": delta, "K": K, "n_k_est": int(nk)})
    return pool, rejected / max(1, tried)


def serving_workload(cfg, nrhs):
    if cfg["kernel"] == "1d_const":
        return W.const_1d(N=cfg["N"], K=cfg["K"], delta=cfg["delta"], nrhs=nrhs)
    k = int(round(np.sqrt(cfg["K"])))
    if cfg["kernel"] == "2d_const_l2":
        return W.const_l2_2d(N=cfg["N"], k=k, nrhs=nrhs, delta=cfg["delta"])
    return W.fractional_2d(N=cfg["N"], k=k, nrhs=nrhs, delta=cfg["delta"])


class ServingStream:
    """The serving scenario: a pool of problems sampled from the grid kernel x h x delta x K
    (seed 6), Poisson arrivals of requests with R in [1, 32] right-hand sides on a random
    problem of the pool, sent to the continuous-batching server by their inputs (the server's
    factorization cache creates and factors each problem on its first request; the stream is
    measured after every problem has been requested once, i.e. with the factorizations cached
    on the device).  Latency is arrival -> result on the host (submission lag + queue wait +
    solve with copies)."""

    def __init__(self, ctx, binding, n_pool, budget, slots, opt):
        rng = np.random.default_rng(6)
        self.pool_cfg, self.rejected = serving_pool(rng, n_pool, budget, cost_cap=2.0e7)
        self.binding, self.opt = binding, opt
        self.server = binding.Server(ctx, hbm_budget=budget, max_slots=slots)
        self.work = []
        t0 = time.perf_counter()
        for cfg in self.pool_cfg:
            w = serving_workload(cfg, 32)
            cfg["dofs"] = int(w.rhs.shape[0])
            self.work.append(w)
            self.server.wait(self.server.submit_workload(w, rhs=w.rhs[:, :1], opt=opt))    # cache the factorization
        self.setup_s = time.perf_counter() - t0

    def run(self, rate, n_req, n_warm, seed=7, max_s=None):
        import threading
        rng = np.random.default_rng(seed)
        arr = np.cumsum(rng.exponential(1.0 / rate, n_warm + n_req))
        pick = rng.integers(len(self.work), size=n_warm + n_req)
        nr = rng.integers(1, 33, size=n_warm + n_req)
        n = len(arr)
        if max_s is not None:                       # bound the stream by its arrival span
            n = max(n_warm + 20, int(np.searchsorted(arr, max_s)))
            arr, pick, nr = arr[:n], pick[:n], nr[:n]
        tickets, lags, lat, done_at = [None] * n, [0.0] * n, [None] * n, [0.0] * n
        submitted = threading.Semaphore(0)
        start = time.perf_counter() + 0.05
        srv = self.server

        def collect():
            for i in range(n):
                submitted.acquire()
                _, st = srv.wait(tickets[i])
                done_at[i] = time.perf_counter()
                lat[i] = lags[i] + 1e-3 * (st["ms_queue"] + st["ms_solve"])
        th = threading.Thread(target=collect)
        th.start()
        for i in range(n):
            tgt = start + arr[i]
            now = time.perf_counter()
            if tgt > now:
                time.sleep(tgt - now)
            w = self.work[pick[i]]
            tickets[i] = srv.submit_workload(w, rhs=w.rhs[:, :nr[i]], opt=self.opt)
            lags[i] = time.perf_counter() - tgt
            submitted.release()
        th.join()
        meas = range(n_warm, n)
        t_first, t_last = start + arr[n_warm], max(done_at[i] for i in meas)
        span = t_last - t_first
        ls = [1e3 * lat[i] for i in meas]
        return {"offered_rate": rate, "requests": len(meas), "requests_per_s": len(meas) / span,
                "solves_per_s": float(sum(nr[i] for i in meas)) / span,
                "p50_ms": percentile(ls, 0.5), "p99_ms": percentile(ls, 0.99),
                "mean_submit_lag_ms": 1e3 * float(np.mean([lags[i] for i in meas]))}

    def close(self):
        info = self.server.info()
        self.server.close()
        return info


def serving_compare(ctx, binding, args):
    """The serving stream at the offered rate (200 requests/s) through the batched mixed path
    and through the plain FP64 one-subdomain-at-a-time path, same arrivals and problems."""
    budget = 16 << 30
    out = {"workload": "Poisson arrivals (seed 7) at %g requests/s of requests with 1-32 RHS on a pool of %d "
                       "problems sampled from the grid kernel {1-D constant, 2-D constant l2, 2-D fractional} x "
                       "h {1/64, 1/128, 1/256} (1-D: 10x finer) x delta {2h, 3h, 0.1} x K (seed 6), "
                       "factorizations cached on the device" % (args.rate, args.pool),
           "slots": args.slots, "hbm_budget_bytes": budget}
    arms = (("mixed_batched", binding.default_options(precision=1, batched=1), args.requests, None),
            ("plain_fp64_per_subdomain", binding.default_options(precision=0, batched=0), args.requests,
             args.serving_plain_s))
    for name, opt, n_req, max_s in arms:
        ss = ServingStream(ctx, binding, args.pool, budget, args.slots, opt)
        res = ss.run(args.rate, n_req, n_req // 10, max_s=max_s)
        inf = ss.close()
        res.update({"setup_and_factor_s": ss.setup_s, "server": inf})
        out[name] = res
        out["pool"] = ss.pool_cfg
        out["rejected_fraction_of_grid_draws"] = ss.rejected
    return out


def run_serving(args):
    """--serving: the serving stream of the mixed batched path with a sweep of the offered
    rate, one JSON line."""
    import torch  # noqa: F401  (device memory and the caller stream of the context)
    from paper_2306_00094_gb300 import binding
    rank, world, _ = dist_env()
    if rank != 0:
        return
    ctx = binding.Context()
    budget = 16 << 30
    ss = ServingStream(ctx, binding, args.pool, budget, args.slots, binding.default_options(precision=1, batched=1))
    main_run = ss.run(args.rate, args.requests, args.requests // 10)
    sweep = [ss.run(r, 300, 30, seed=8 + j) for j, r in enumerate((50, 100, 200, 400, 800))]
    sustainable = max([s["offered_rate"] for s in sweep if s["requests_per_s"] >= 0.9 * s["offered_rate"]], default=None)
    info = ss.close()
    line = {"metric": "serving: FETI requests (mixed kernels, h, delta, K; R in [1, 32]) under Poisson arrivals, "
                      "arrival -> host result latency, 1 GB300",
            "mode": "serving", "value": main_run["solves_per_s"], "unit": "solves/s", "n_gpus": 1,
            "higher_is_better": True, "data": "synthetic", "dtype": "f32 operators and PCG iterations + f64 refinement",
            "config": {"workload": "serving pool of problems sampled from the grid (seed 6)",
                       "pool": ss.pool_cfg, "slots": args.slots, "hbm_budget_bytes": budget,
                       "rejected_fraction_of_grid_draws": ss.rejected},
            "setup_and_factor_s": ss.setup_s, "run": main_run, "rate_sweep": sweep,
            "max_sustained_rate": sustainable, "server": info}
    print(json.dumps(line), flush=True)


PAPER_ROWS = [
    # (table, kernel, N, delta, k): the rows of the paper's Tables fixedHorizon and fixedRatio
    # that fit one GPU with dense subdomain matrices (the fixed-ratio rows at 12 x 12 hold about
    # 170 GB of subdomain matrices, the larger rows more than the device holds)
    ("fixedHorizon", "constant", 250, 0.008, 6),
    ("fixedHorizon", "fractional", 250, 0.008, 6),
    ("fixedHorizon", "peridynamic", 250, 0.008, 6),
    ("fixedRatio", "constant", 500, 0.008, 6),
    ("fixedRatio", "fractional", 500, 0.008, 6),
    ("fixedHorizon", "constant", 500, 0.008, 12),
    ("fixedHorizon", "fractional", 500, 0.008, 12),
    ("fixedHorizon", "peridynamic", 500, 0.008, 12),
]


def run_paper_rows(args):
    """The paper's table rows that fit one GB300 with dense subdomain matrices (6 x 6
    subdomains): its manufactured problem (u = x1^2 x2 + x2^2, g = u on the collar,
    f = -2 (1 + x2) for every kernel; the peridynamic u = (u, u)), FETI in FP64 at the
    paper's tolerance 1e-10 and in the mixed mode, and the diagonally preconditioned CG;
    iteration counts beside the paper's.  One JSON line."""
    import torch
    from paper_2306_00094_gb300 import binding
    rank, world, _ = dist_env()
    if rank != 0:
        return
    golden = {}
    for line in open(os.path.join(ROOT, "tests", "golden", "paper_table_fixed_horizon.txt")):
        f = line.split()
        if f and not f[0].startswith("#"):
            golden[("fixedHorizon", f[0], f[1])] = {"cg_its": int(f[3]), "feti_its": int(f[5]), "l2": float(f[7])}
    for line in open(os.path.join(ROOT, "tests", "golden", "paper_table_fixed_ratio.txt")):
        f = line.split()
        if f and not f[0].startswith("#"):
            golden[("fixedRatio", f[0], f[1])] = {"cg_its": int(f[4]), "feti_its": int(f[6])}
    kinds = {"constant": W.KERNEL_CONST_LINF, "fractional": W.KERNEL_FRACTIONAL, "peridynamic": W.KERNEL_PERIDYNAMIC}
    ctx = binding.Context()
    rows = []
    for table, kname, N, delta, k in PAPER_ROWS:
        mesh = W.make_mesh(2, N, W.collar_cells(delta, N))
        kern = W.Kernel(kinds[kname], delta, s=0.4 if kname == "fractional" else 0.0)
        kern.scale = W.default_scale(kern, 2)
        nc = kern.ncomp
        x, y = mesh.xy[:, 0], mesh.xy[:, 1]
        uex = x * x * y + y * y
        fval = -2.0 * (1.0 + y)
        u = np.repeat(uex, nc).reshape(-1, 1)
        f = np.repeat(fval, nc).reshape(-1, 1)
        w = W.Workload(f"{table}_{kname}", mesh, kern, W.rect_labels(mesh, k, k), k * k, np.asfortranarray(f), 0,
                       g=np.asfortranarray(u))
        t0 = time.perf_counter()
        p = binding.Problem.from_workload(ctx, w)
        t_setup = time.perf_counter() - t0
        t0 = time.perf_counter()
        p.factor(3)
        t_factor = time.perf_counter() - t0
        free = np.repeat(mesh.node_is_dirichlet == 0, nc)
        res = {"table": table, "kernel": kname, "K": f"{k}x{k}", "h": 1.0 / N, "delta": delta,
               "dofs": int(free.sum()), "setup_s": t_setup, "factor_fp64_fp32_s": t_factor}
        for mode, opt in (("feti_fp64", binding.default_options(precision=0, tol=1e-10)),
                          ("feti_mixed", binding.default_options(precision=1)),
                          ("cg", binding.default_options(tol=1e-10, max_it=20000))):
            p.set_options(opt)
            solve = p.solve_cg if mode == "cg" else p.solve
            uh, st = solve(w.rhs, 0, w.g)
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            uh, st = solve(w.rhs, 0, w.g)
            dt = time.perf_counter() - t0
            res[mode] = {"iterations": st["iterations"], "refine_sweeps": st["refine_sweeps"], "solve_s": dt,
                         "max_nodal_err_vs_u": float(np.abs(uh[:, 0] - u[:, 0])[free].max())}
        gold = golden.get((table, kname, f"{k}x{k}"))
        if gold:
            res["paper"] = gold
        rows.append(res)
        p.close()
    print(json.dumps({"mode": "paper_rows", "rows": rows}), flush=True)


def main():
    ap = argparse.ArgumentParser(description=__doc__, formatter_class=argparse.RawDescriptionHelpFormatter)
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--workload", choices=list(WORKLOADS), default=HEADLINE,
                    help="the workload of the timed steps (default: the largest single-GPU one)")
    ap.add_argument("--headline-only", action="store_true", help="skip the other workloads")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--only-timed", action="store_true", help="setup, warm-up and the timed steps only (for ncu)")
    ap.add_argument("--cells", type=int, default=0,
                    help="profiling: the workload at h = 1/CELLS (same kernel, subdomains and right-hand "
                         "sides) for ncu captures that must stay small; implies --only-timed")
    ap.add_argument("--profile-range", choices=["solve", "factor"], default=None,
                    help="profiling: wrap the timed steps (solve) or one extra FP32 factorization (factor) "
                         "in a CUDA profiler range, for ncu --profile-from-start off")
    ap.add_argument("--tensor-core-precond", action="store_true",
                    help="the timed mixed solve applies the preconditioner's S_k on the tensor cores "
                         "(precond_fp16 = 2; default: the FP16 copy on the FP32 pipes)")
    ap.add_argument("--host-loop", action="store_true",
                    help="PCG loops as host-checked graph chunks instead of device-side WHILE graphs "
                         "(ncu cannot profile kernels inside conditional graphs)")
    ap.add_argument("--serving", action="store_true",
                    help="serving scenario: Poisson arrivals of mixed requests to the server (one JSON line)")
    ap.add_argument("--rate", type=float, default=200.0, help="serving: offered requests per second")
    ap.add_argument("--requests", type=int, default=1000, help="serving: measured requests")
    ap.add_argument("--serving-plain-s", type=float, default=2.0,
                    help="serving comparison: arrival span of the plain FP64 arm's stream (s)")
    ap.add_argument("--pool", type=int, default=6, help="serving: distinct factored problems")
    ap.add_argument("--slots", type=int, default=4, help="serving: server slots")
    ap.add_argument("--paper-rows", action="store_true",
                    help="the paper's table rows that fit one GPU (6 x 6 subdomains, 62.5k / 250k dofs)")
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    if args.serving:
        run_serving(args)
    elif args.paper_rows:
        run_paper_rows(args)
    elif args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
