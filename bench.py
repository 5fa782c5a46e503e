#!/usr/bin/env python
"""Benchmark of the particle-particle ladder term R_ijab = sum_cd (ac|bd) t_ijcd
with (ac|bd) = sum_P L_Pac L_Pbd built on the fly in blocks of `a` (Eq. 5, 6).

One step = one full ladder evaluation (integral blocks + ladder GEMM + pair
symmetry scatter) on the o=40, v=400, n_chol=2000 workload in emulated FP64
(Ozaki BF16 slices on tcgen05 tensor cores), inputs resident in HBM (L 2.56 GB
and t2 2.05 GB, both larger than the 129 MB L2).  Prints one JSON line.

  python bench.py [--gpus N --steps K --warmup W] [--impl reference]

N > 1 (torchrun): every rank evaluates its own independent problem (seed = rank),
no data-path collective; value = all ranks' flops / the slowest rank's time.
--impl reference times the FP64 CPU oracle on the host cores, one sampled `a`
column block per step.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

WORKLOADS = {"o40_v400_n2000": (40, 400, 2000), "o20_v200_n1000": (20, 200, 1000),
             "o60_v600_n3000": (60, 600, 3000), "o16_v160_n800": (16, 160, 800), "o4_v24_n60": (4, 24, 60),
             # the paper's synthetic shapes of Table 1: n = 5K, v = 3K/4, o = K - v for K = 300, 400, 500
             "o75_v225_n1500": (75, 225, 1500), "o100_v300_n2000": (100, 300, 2000),
             "o125_v375_n2500": (125, 375, 2500)}
METRIC = "ladder-term TFLOP/s (emulated FP64)"
UNIT = "TFLOP/s"


def algorithmic_flops(o, v, n):
    """2 (o^2 + n) v^4: integral build n v^4 plus ladder GEMM o^2 v^4 multiply-adds."""
    return 2.0 * (o * o + n) * float(v) ** 4


def peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        return d, "measured"
    return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0, "sm_max_mhz": 2070.0}, "fallback"


class Clocks:
    """nvidia-smi samples of SM clock and throttle reasons during the timed region."""

    def __init__(self, index=0):
        self.index, self.proc, self.lines = index, None, []

    def __enter__(self):
        q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
             "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
             "clocks_event_reasons.sw_power_cap")
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), f"--query-gpu={q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except OSError:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
            self.t.join(timeout=2)

    def summary(self):
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
            for nm, val in zip(names, f[5:9]):
                if val.lower().startswith("active"):
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}
        sm.sort()
        return {"sm_mhz": sm[len(sm) // 2], "sm_max_mhz": mx, "reasons": sorted(reasons), "samples": len(sm)}


def dist_init():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch.distributed as dist
        import torch
        backend = "nccl" if torch.cuda.is_available() else "gloo"
        dist.init_process_group(backend)
    return rank, local, world


def dist_max(x, world, device=None):
    """Max of a float over ranks (identity for one rank)."""
    if world == 1:
        return x
    import torch
    import torch.distributed as dist
    t = torch.tensor([x], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def dist_barrier(world):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def oracle_sample(L, t2, a_list):
    """Time the FP64 CPU oracle on the `a` columns a_list; returns (R_sample, seconds, threads)."""
    from oracle import oracle as O
    O.build()
    t0 = time.perf_counter()
    R = O.ladder(L, t2, a_list=a_list)
    return R, time.perf_counter() - t0, O.max_threads()


def cpu_model() -> str:
    """Host CPU model name (lscpu, else /proc/cpuinfo), for the CPU baseline record."""
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.strip().startswith("Model name:"):
                return line.split(":", 1)[1].strip()
    except (OSError, subprocess.SubprocessError):
        pass
    try:
        for line in open("/proc/cpuinfo"):
            if line.lower().startswith(("model name", "cpu part")):
                return line.split(":", 1)[1].strip()
    except OSError:
        pass
    return "unknown"


def traffic_record():
    """Per-launch DRAM bytes of the tensor-core GEMM from the committed ncu summary, if the
    kernel source is unchanged since it was captured (else None)."""
    import hashlib
    p = os.path.join(ROOT, "profiles", "traffic.json")
    if not os.path.exists(p):
        return None
    rec = json.load(open(p))
    src = os.path.join(ROOT, "paper_2310_04559_gb300", "csrc", "gemm_tc.cu")
    sha = hashlib.sha256(open(src, "rb").read()).hexdigest()[:16]
    return rec if rec.get("gemm_tc_sha") == sha else None


# --------------------------------------------------------------------- ours
def run_ours(a):
    import numpy as np
    import torch

    from paper_2310_04559_gb300 import binding as B
    from paper_2310_04559_gb300 import synth

    rank, local, world = dist_init()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    o, v, n = WORKLOADS[a.workload]
    mode = a.mode
    flops = algorithmic_flops(o, v, n)

    L_np, t2_np = synth.ladder_inputs(o, v, n, seed=rank)
    L_h = torch.from_numpy(L_np).pin_memory()
    t2_h = torch.from_numpy(t2_np).pin_memory()
    Lg, tg = L_h.to(dev), t2_h.to(dev)
    R = torch.empty_like(tg)
    E = torch.empty((), dtype=torch.float64, device=dev)
    # device-memory budget covers everything: inputs, R and the library's workspace
    budget = int(a.budget_gb * 1e9) - L_np.nbytes - 2 * t2_np.nbytes - (2 << 30)
    ws_bytes = B.workspace_size(o, v, n, mode=mode, symmetric=True, budget=budget)
    ws = B.alloc_workspace(ws_bytes, dev)
    plan = B.plan(o, v, n, ws_bytes=ws_bytes, mode=mode, symmetric=True)

    def step():
        B.ladder_forward(Lg, tg, R=R, mode=mode, symmetric=True, workspace=ws, no_sync=True)

    from paper_2310_04559_gb300 import _lib
    lib = _lib.load()
    for _ in range(a.warmup):
        step()
    _lib.check(lib.cc_ladder_device_status(B._ptr(ws), B._stream(dev)), "warm-up")

    stream = torch.cuda.current_stream(dev)
    dist_barrier(world)
    torch.cuda.synchronize(dev)
    B.profile_enable(True)
    n0 = B.launch_count()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with Clocks(local) as clk:
        e0.record(stream)
        for _ in range(a.steps):
            step()
        e1.record(stream)
        torch.cuda.synchronize(dev)
    launches = B.launch_count() - n0
    prof = B.profile_read()
    B.profile_enable(False)
    dist_barrier(world)
    _lib.check(lib.cc_ladder_device_status(B._ptr(ws), B._stream(dev)), "timed steps")
    t_step = e0.elapsed_time(e1) / 1e3 / a.steps
    t_max = dist_max(t_step, world, dev)
    value = flops * world / t_max / 1e12

    # roofline of the dominant kernel (the tcgen05 slice GEMM): issued slice-MMA
    # flops per launch over its average launch time, from the live events
    tc = [k for k in prof if k.endswith("_tc")]
    tc_ms = sum(prof[k]["ms"] for k in tc)
    tc_fl = sum(prof[k]["flops"] for k in tc)
    tc_n = sum(prof[k]["launches"] for k in tc)
    pk, pk_src = peaks()
    peak = pk.get("bf16_tflops_sustained", pk["bf16_tflops"])
    achieved = tc_fl / (tc_ms / 1e3) / 1e12 if tc_ms > 0 else None
    tr = traffic_record()
    roofline = {"kernel": "gemm_tc_kernel<bf16>", "bound": "tensor", "achieved": achieved, "peak": peak,
                "unit": "TFLOP/s", "frac": (achieved / peak) if achieved else None,
                "traffic": tr["bytes_per_launch"] if tr else None,
                "peak_source": f"{pk_src} bf16_tflops_sustained (kernel timed inside a long step)",
                "launches": tc_n, "flops_per_launch": tc_fl / max(tc_n, 1), "ms_per_launch": tc_ms / max(tc_n, 1),
                "share_of_step": tc_ms / (t_step * 1e3 * a.steps)}

    # end to end through the public API: pinned host -> device, forward + energy, R and E -> host
    R_h = torch.empty(R.shape, dtype=torch.float64, pin_memory=True)
    E_h = torch.empty((), dtype=torch.float64, pin_memory=True)

    def e2e_step():
        Lg.copy_(L_h, non_blocking=True)
        tg.copy_(t2_h, non_blocking=True)
        B.ladder_forward(Lg, tg, R=R, mode=mode, symmetric=True, workspace=ws, energy=False, no_sync=True)
        E.copy_(B.pair_energy(R, tg))
        R_h.copy_(R, non_blocking=True)
        E_h.copy_(E, non_blocking=True)

    e2e_step()
    torch.cuda.synchronize(dev)
    dist_barrier(world)
    e2 = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
    e2[0].record(stream)
    for _ in range(a.e2e_steps):
        e2e_step()
    e2[1].record(stream)
    torch.cuda.synchronize(dev)
    t_e2e = dist_max(e2[0].elapsed_time(e2[1]) / 1e3 / a.e2e_steps, world, dev)
    e2e = {"value": flops * world / t_e2e / 1e12, "unit": UNIT,
           "h2d_bytes_per_step": L_h.numel() * 8 + t2_h.numel() * 8, "d2h_bytes_per_step": R_h.numel() * 8 + 8}

    out = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": a.steps, "warmup": a.warmup,
           "ms_per_step": t_max * 1e3, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
           "dtype": "bf16", "precision": "fp64 emulated (Ozaki: 6 bf16 slices x 7 bits, exact fp32 products, "
                                         "fp64 recombination)",
           "data": "synthetic (seeded random Cholesky vectors and amplitudes, shapes of the paper's benchmarks)",
           "config": {"workload": a.workload, "o": o, "v": v, "n_chol": n, "mode": mode, "order": plan["order"],
                      "a_block": plan["a_block"], "n_blocks": plan["n_blocks"], "pairs": plan["pairs"],
                      "symmetric_t": True, "workspace_gb": round(ws_bytes / 1e9, 2),
                      "peak_device_gb": round(torch.cuda.max_memory_allocated(dev) / 1e9, 2),
                      "flops_algorithmic_per_step": flops, "flops_issued_per_step": plan["flops_issued"],
                      "l2": "inputs larger than L2 (L %.2f GB, t2 %.2f GB)" % (L_np.nbytes / 1e9, t2_np.nbytes / 1e9)},
           "e2e": e2e, "roofline": roofline, "clocks": clk.summary(), "gpu_launches": launches,
           "phases_ms_per_step": {k: round(v_["ms"] / a.steps, 3) for k, v_ in sorted(prof.items())}}

    if rank == 0 and not a.quick:
        # accuracy on a sampled `a` block vs the FP64 oracle, FP64-MMA speed-up, other modes,
        # and the oracle itself as the CPU baseline
        a_list = list(range(a.sample_a))
        Rs, t_cpu, threads = oracle_sample(L_np, t2_np, a_list)
        # entries computed for an `a` column under pair symmetry with an a-range: i <= j
        iu = np.triu_indices(o)
        rel = lambda X: float(np.linalg.norm(X[:, :, a_list, :][iu] - Rs[iu]) / np.linalg.norm(Rs[iu]))
        modes = {mode: {"tflops": value / world, "rel_err": rel(R.cpu().numpy())}}
        # plain FP64-MMA on the same sampled columns (its full run takes minutes)
        nb = max(a.fp64_sample, 1)
        R64 = torch.zeros_like(tg)
        B.ladder_forward(Lg, tg, R=R64, mode="fp64", symmetric=True, a_range=(0, 2), workspace=ws)
        f0, f1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        f0.record(stream)
        B.ladder_forward(Lg, tg, R=R64, mode="fp64", symmetric=True, a_range=(0, nb), workspace=ws)
        f1.record(stream)
        torch.cuda.synchronize(dev)
        # the range's share of the work: integrals and ladder columns exist for b >= a only
        full = B.plan(o, v, n, ws_bytes=ws_bytes, mode="fp64", symmetric=True)["flops_issued"]
        part = B.plan(o, v, n, ws_bytes=ws_bytes, mode="fp64", symmetric=True, a_range=(0, nb))["flops_issued"]
        t64 = f0.elapsed_time(f1) / 1e3 * full / part
        modes["fp64"] = {"tflops": flops / t64 / 1e12, "rel_err": rel(R64.cpu().numpy()),
                         "timed_on": f"a in [0,{nb}) of {v}, scaled by the issued-flop ratio {full / part:.2f}"}
        for m in a.other_modes.split(","):
            if not m:
                continue
            Rm = torch.empty_like(tg)
            B.ladder_forward(Lg, tg, R=Rm, mode=m, symmetric=True, workspace=ws)
            g0, g1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            g0.record(stream)
            B.ladder_forward(Lg, tg, R=Rm, mode=m, symmetric=True, workspace=ws)
            g1.record(stream)
            torch.cuda.synchronize(dev)
            modes[m] = {"tflops": flops / (g0.elapsed_time(g1) / 1e3) / 1e12, "rel_err": rel(Rm.cpu().numpy())}
        out["modes"] = modes
        out["speedup_vs_fp64_mma"] = modes[mode]["tflops"] / modes["fp64"]["tflops"]
        # the two further Cholesky terms with the ladder's contraction (Eq. 8, Eq. 9), same workload
        del ws, R64
        torch.cuda.empty_cache()
        Lov = torch.from_numpy(synth.cholesky_ov(n, o, v, seed=rank + 7)).to(dev)
        terms = {}
        for name, fl in (("tijbk", 2.0 * (n + o * o) * o * float(v) ** 3),
                         ("tijkl", 2.0 * (n + o * o) * o * o * float(v) ** 2)):
            call = (lambda: B.tijbk(Lov, Lg, tg, mode=mode, budget=40 << 30)) if name == "tijbk" else \
                   (lambda: B.tijkl(Lov, tg, mode=mode, budget=40 << 30))
            call()
            h0, h1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            h0.record(stream)
            call()
            h1.record(stream)
            torch.cuda.synchronize(dev)
            ms = h0.elapsed_time(h1)
            terms[name] = {"tflops": fl / (ms / 1e3) / 1e12, "ms": ms, "flops_algorithmic": fl}
        out["terms"] = terms
        # both contraction orders (Section 3.2), each timed after a warm-up call and counted
        # against its own algorithmic flops (2(o^2+n)v^4 integral-first, 4 n o^2 v^3
        # Cholesky-first), next to the order the autotuner picks for the shape
        orders = {}
        for (oo, vo, no), bud in (((4, 96, 480), 8 << 30), ((20, 200, 1000), 24 << 30)):
            key = f"o{oo}_v{vo}_n{no}"
            try:
                Lo_np, to_np = synth.ladder_inputs(oo, vo, no, seed=21)
                Lo, to = torch.from_numpy(Lo_np).to(dev), torch.from_numpy(to_np).to(dev)
                Ro = torch.empty_like(to)
                rec = {}
                for od, fl in (("integral_first", 2.0 * (oo * oo + no) * float(vo) ** 4),
                               ("cholesky_first", 4.0 * no * oo * oo * float(vo) ** 3)):
                    wso = B.alloc_workspace(B.workspace_size(oo, vo, no, mode=mode, order=od, symmetric=True,
                                                             budget=bud), dev)
                    B.ladder_forward(Lo, to, R=Ro, mode=mode, order=od, symmetric=True, workspace=wso)
                    q0, q1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                    q0.record(stream)
                    B.ladder_forward(Lo, to, R=Ro, mode=mode, order=od, symmetric=True, workspace=wso)
                    q1.record(stream)
                    torch.cuda.synchronize(dev)
                    ms = q0.elapsed_time(q1)
                    rec[od] = {"ms": ms, "tflops": fl / (ms / 1e3) / 1e12, "flops_algorithmic": fl}
                    del wso
                rec["autotuner_choice"] = B.autotune(Lo, to, R=Ro, mode=mode, symmetric=True, budget=bud)["order"]
                orders[key] = rec
                del Lo, to, Ro
            except Exception as e:  # noqa: BLE001 - reported in the JSON line, the main figures stand
                orders[key] = {"error": f"{type(e).__name__}: {e}"}
        out["orders"] = orders
        # adjoint (dt2, dL of loss = <W, R>) on the o=16, v=160, n_chol=800 workload: forward and
        # backward times, sampled gradient entries against the FP64 oracle
        oa, va, na = 16, 160, 800
        La_np, ta_np = synth.ladder_inputs(oa, va, na, seed=4)
        Wa_np = synth.cotangent(oa, va, seed=5)
        La, ta, Wa = (torch.from_numpy(x).to(dev) for x in (La_np, ta_np, Wa_np))
        from oracle import oracle as O
        gi = np.random.default_rng(6)
        i1, i2 = gi.integers(0, ta_np.size, 16), gi.integers(0, La_np.size, 16)
        e1, e2 = O.ladder_grad_entries(La_np, ta_np, Wa_np, i1, i2)
        fwd_fl = algorithmic_flops(oa, va, na)
        adj = {"workload": "o16_v160_n800", "flops_forward": fwd_fl, "flops_backward": 2 * fwd_fl}
        for m in ("fp64", mode):
            B.ladder_forward(La, ta, mode=m, symmetric=True)
            dLa, dta = B.ladder_backward(La, ta, Wa, mode=m, symmetric=True)
            torch.cuda.synchronize(dev)
            a0_, a1_, a2_ = (torch.cuda.Event(enable_timing=True) for _ in range(3))
            a0_.record(stream)
            B.ladder_forward(La, ta, mode=m, symmetric=True)
            a1_.record(stream)
            dLa, dta = B.ladder_backward(La, ta, Wa, mode=m, symmetric=True)
            a2_.record(stream)
            torch.cuda.synchronize(dev)
            tf, tb = a0_.elapsed_time(a1_) / 1e3, a1_.elapsed_time(a2_) / 1e3
            g1 = dta.cpu().numpy().ravel()[i1]
            g2 = dLa.cpu().numpy().ravel()[i2]
            adj[m] = {"forward_tflops": fwd_fl / tf / 1e12, "backward_tflops": 2 * fwd_fl / tb / 1e12,
                      "backward_ms": tb * 1e3, "dt2_rel_err": float(np.linalg.norm(g1 - e1) / np.linalg.norm(e1)),
                      "dL_rel_err": float(np.linalg.norm(g2 - e2) / np.linalg.norm(e2))}
        out["adjoint"] = adj
        del La, ta, Wa, dLa, dta
        # host-resident amplitudes: t2 and R in page-locked host memory, read and written over the
        # host link, the device holding L, one block of pairs and the integral blocks (40 GB budget)
        Rh = torch.empty(t2_h.shape, dtype=torch.float64).pin_memory()
        hb = 40 << 30
        B.ladder_forward(Lg, t2_h, R=Rh, mode=mode, symmetric=True, host_t2r=True, budget=hb)
        torch.cuda.synchronize(dev)
        k0, k1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        k0.record(stream)
        B.ladder_forward(Lg, t2_h, R=Rh, mode=mode, symmetric=True, host_t2r=True, budget=hb)
        k1.record(stream)
        torch.cuda.synchronize(dev)
        hp = B.plan(o, v, n, mode=mode, symmetric=True, host_t2r=True, budget=hb)
        out["host_resident"] = {"tflops": flops / (k0.elapsed_time(k1) / 1e3) / 1e12,
                                "rel_err": rel(Rh.numpy()), "device_budget_gb": round(hb / 1e9, 1),
                                "a_blocks": hp["n_blocks"], "ws_gb": round(hp["ws_bytes"] / 1e9, 2)}
        sample_flops = 2.0 * (o * o + n) * float(v) ** 3 * len(a_list)
        out["cpu_baseline"] = {"value": sample_flops / t_cpu / 1e12, "unit": UNIT, "cores": threads, "kind": "oracle",
                               "cpu_model": cpu_model(),
                               "sample": f"R[:, :, a, :] for a in {a_list} of the same workload "
                                         f"({len(a_list)}/{v} of the work, {t_cpu:.1f} s)"}
    if rank == 0:
        print(json.dumps(out), flush=True)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


# ---------------------------------------------------------------- reference
def run_reference(a):
    """The FP64 CPU oracle as it stands, timed on the host cores, one sampled `a`
    column per step of the same workload."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    from paper_2310_04559_gb300 import synth
    o, v, n = WORKLOADS[a.workload]
    L, t2 = synth.ladder_inputs(o, v, n, seed=0)
    per_step = 2.0 * (o * o + n) * float(v) ** 3  # one `a` column
    for w in range(a.warmup):
        oracle_sample(L, t2, [w % v])
    times, threads = [], 1
    for s in range(a.steps):
        _, t, threads = oracle_sample(L, t2, [(a.warmup + s) % v])
        times.append(t)
    t_step = sum(times) / len(times)
    value = per_step / t_step / 1e12
    sample = f"one `a` column block R[:, :, a, :] of the {a.workload} workload per step ({per_step:.3e} flops)"
    out = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": int(os.environ.get(
        "WORLD_SIZE", "1")), "steps": a.steps, "warmup": a.warmup, "ms_per_step": t_step * 1e3,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic", "config": {"workload": a.workload, "o": o, "v": v, "n_chol": n},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": threads, "kind": "oracle", "sample": sample,
                         "cpu_model": cpu_model()},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(out), flush=True)


def main(argv=None):
    p = argparse.ArgumentParser(description=__doc__, formatter_class=argparse.RawDescriptionHelpFormatter)
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=5)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", choices=["ours", "reference"], default="ours")
    p.add_argument("--workload", choices=sorted(WORKLOADS), default="o40_v400_n2000")
    p.add_argument("--mode", default="ozaki_bf16")
    p.add_argument("--budget-gb", type=float, default=150.0, help="peak device memory (GB, 1e9 bytes)")
    p.add_argument("--e2e-steps", type=int, default=2)
    p.add_argument("--sample-a", type=int, default=1, help="oracle `a` columns for accuracy / CPU baseline")
    p.add_argument("--fp64-sample", type=int, default=20, help="`a` columns timed in plain FP64")
    p.add_argument("--other-modes", default="tf32,bf16")
    p.add_argument("--quick", action="store_true", help="skip accuracy, FP64 and CPU-baseline legs")
    a = p.parse_args(argv)
    if a.warmup < 3:
        p.error("--warmup must be >= 3")
    if a.impl == "reference":
        run_reference(a)
    else:
        run_ours(a)


if __name__ == "__main__":
    main()
