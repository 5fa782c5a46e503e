#!/usr/bin/env python
"""Benchmark of the particle-particle ladder term R_ijab = sum_cd (ac|bd) t_ijcd
with (ac|bd) = sum_P L_Pac L_Pbd built on the fly in blocks of `a` (Eq. 5, 6).

One step = one full ladder evaluation (integral blocks + ladder GEMMs + pair
symmetry write) on the o=40, v=400, n_chol=2000 workload in emulated FP64
(Ozaki BF16 slices on tcgen05 tensor cores), inputs resident in HBM (L 2.56 GB
and t2 2.05 GB, both larger than the 129 MB L2).  Prints one JSON line.

  python bench.py [--gpus N --steps K --warmup W] [--impl reference]

N > 1 (torchrun): ONE problem, its `a` range split over the ranks by work
(cc_ladder_partition); every rank computes its share of R with no exchange, the
pair energy is one all-reduce of the ranks' shares (end-to-end leg), R is summed
onto rank 0 there.  value = the problem's flops / the slowest rank's time
(strong scaling).
--impl reference times the FP64 CPU oracle on the host cores, one sampled `a`
column per step, on the same workload and config.
"""
from __future__ import annotations

import argparse
import json
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
DTYPE = "f64 (emulated: bf16 Ozaki slices, exact fp32 level sums, int64/fp64 recombination)"


def algorithmic_flops(o, v, n):
    """2 (o^2 + n) v^4: integral build n v^4 plus ladder GEMM o^2 v^4 multiply-adds."""
    return 2.0 * (o * o + n) * float(v) ** 4


def workload_config(name):
    """The `config` object of both arms' JSON lines (identical for the same workload)."""
    o, v, n = WORKLOADS[name]
    L_gb, t_gb = n * v * v * 8 / 1e9, o * o * v * v * 8 / 1e9
    return {"workload": name, "o": o, "v": v, "n_chol": n, "symmetric_t": True,
            "l2": "inputs larger than L2 (L %.2f GB, t2 %.2f GB)" % (L_gb, t_gb) if min(L_gb, t_gb) > 0.129
            else "inputs smaller than L2"}


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


def shard_range(o, v, n, rank, world, mode):
    """This rank's `a` range of the one problem (the library's work-balanced partition)."""
    if world == 1:
        return None
    from paper_2310_04559_gb300 import binding as B
    b = B.partition(o, v, n, world, mode=mode, symmetric=True)
    return (b[rank], b[rank + 1])


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
    """DRAM bytes over algorithmic bytes of the tensor-core GEMM, from the committed summary of an
    ncu capture (profiles/gemm_tc_traffic.json), if the kernel source is unchanged since it was
    captured (else None)."""
    import hashlib
    p = os.path.join(ROOT, "profiles", "gemm_tc_traffic.json")
    if not os.path.exists(p):
        return None
    rec = json.load(open(p))
    src = os.path.join(ROOT, "paper_2310_04559_gb300", "csrc", "gemm_tc.cu")
    sha = hashlib.sha256(open(src, "rb").read()).hexdigest()[:16]
    return rec if rec.get("gemm_tc_sha") == sha else None


def timed(stream, fn, reps=1):
    """Milliseconds per call of fn() on `stream` (CUDA events; one untimed call first)."""
    import torch
    fn()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record(stream)
    for _ in range(reps):
        fn()
    e1.record(stream)
    torch.cuda.synchronize()
    return e0.elapsed_time(e1) / reps


def mode_peak(mode, probed, pk):
    """Peak (TFLOP/s) of the unit a mode's GEMMs run on, and where it comes from."""
    if mode == "fp64":
        return probed.get("dmma"), "probed dmma (mma.sync.m8n8k4.f64)"
    if mode == "tf32":
        return probed.get("tc_tf32"), "probed tcgen05 kind::tf32"
    return pk.get("bf16_tflops_sustained", pk["bf16_tflops"]), "MEASURED_PEAKS bf16_tflops_sustained"


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
    rng_a = shard_range(o, v, n, rank, world, mode)

    # one problem for every rank (seed 0); the ranks split its `a` range
    L_np, t2_np = synth.ladder_inputs(o, v, n, seed=0)
    L_h = torch.from_numpy(L_np).pin_memory()
    t2_h = torch.from_numpy(t2_np).pin_memory()
    Lg, tg = L_h.to(dev), t2_h.to(dev)
    R = torch.zeros_like(tg)
    # device-memory budget covers everything: inputs, R and the library's workspace
    budget = int(a.budget_gb * 1e9) - L_np.nbytes - 2 * t2_np.nbytes - (2 << 30)
    ws_bytes = B.workspace_size(o, v, n, mode=mode, symmetric=True, budget=budget, a_range=rng_a)
    ws = B.alloc_workspace(ws_bytes, dev)
    plan = B.plan(o, v, n, ws_bytes=ws_bytes, mode=mode, symmetric=True, a_range=rng_a)

    def step():
        B.ladder_forward(Lg, tg, R=R, mode=mode, symmetric=True, workspace=ws, no_sync=True, a_range=rng_a)

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
    value = flops / t_max / 1e12  # one problem, all ranks

    # roofline of the dominant kernel (the tcgen05 slice GEMM): issued slice-MMA
    # flops per launch over its average launch time, from the live events
    tc = [k for k in prof if k.endswith("_tc")]
    tc_ms = sum(prof[k]["ms"] for k in tc)
    tc_fl = sum(prof[k]["flops"] for k in tc)
    tc_by = sum(prof[k]["bytes"] for k in tc)
    tc_n = sum(prof[k]["launches"] for k in tc)
    pk, pk_src = peaks()
    peak = pk.get("bf16_tflops_sustained", pk["bf16_tflops"])
    achieved = tc_fl / (tc_ms / 1e3) / 1e12 if tc_ms > 0 else None
    tr = traffic_record()
    alg_bytes = tc_by / max(tc_n, 1)
    roofline = {"kernel": "gemm_tc_kernel<bf16>", "bound": "tensor", "achieved": achieved, "peak": peak,
                "unit": "TFLOP/s", "frac": (achieved / peak) if achieved else None,
                "traffic": tr["ratio"] * alg_bytes if tr else None,
                "algorithmic_bytes_per_launch": alg_bytes,
                "traffic_source": (f"ncu dram__bytes_read+write ({tr['launch']}, {tr['workload']}): "
                                   f"{tr['ratio']:.2f} x their algorithmic bytes, applied to this run's "
                                   "algorithmic bytes per launch") if tr else None,
                "peak_source": f"{pk_src} bf16_tflops_sustained (kernel timed inside a long step), of measured"
                               if pk_src == "measured" else "fallback 1.7 PFLOP/s sustained, of fallback",
                "launches": tc_n, "flops_per_launch": tc_fl / max(tc_n, 1), "ms_per_launch": tc_ms / max(tc_n, 1),
                "share_of_step": tc_ms / (t_step * 1e3 * a.steps)}

    # end to end through the public API: pinned host -> device, forward + energy, R and E -> host.
    # With N ranks each one computes its share of R and of the energy; the energy is all-reduced
    # and R summed onto rank 0, which reads it back.
    R_h = torch.empty(R.shape, dtype=torch.float64, pin_memory=True) if rank == 0 else None
    E_h = torch.empty((), dtype=torch.float64, pin_memory=True)

    def e2e_step():
        Lg.copy_(L_h, non_blocking=True)
        tg.copy_(t2_h, non_blocking=True)
        if world > 1:
            R.zero_()
        _, E = B.ladder_forward(Lg, tg, R=R, mode=mode, symmetric=True, workspace=ws, energy=True, no_sync=True,
                                a_range=rng_a)
        if world > 1:
            import torch.distributed as dist
            dist.all_reduce(E)
            dist.reduce(R, dst=0)
        if rank == 0:
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
    e2e = {"value": flops / t_e2e / 1e12, "unit": UNIT,
           "h2d_bytes_per_step": (L_h.numel() * 8 + t2_h.numel() * 8) * world,
           "d2h_bytes_per_step": R.numel() * 8 + 8 * world}
    E_e2e = float(E_h)

    out = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": a.steps, "warmup": a.warmup,
           "ms_per_step": t_max * 1e3, "higher_is_better": True, "scaling": "strong" if world > 1 else "weak",
           "vs_baseline": None, "dtype": DTYPE,
           "precision": "fp64 emulated (Ozaki: 6 bf16 slices x 7 bits, exact fp32 products, fp64 recombination)",
           "data": "synthetic (seeded random Cholesky vectors and amplitudes, shapes of the paper's benchmarks)",
           "config": workload_config(a.workload),
           "plan": {"mode": mode, "order": plan["order"], "a_block": plan["a_block"], "n_blocks": plan["n_blocks"],
                    "pairs": plan["pairs"], "a_range": list(rng_a) if rng_a else [0, v],
                    "parallelism": f"a-range partition over {world} ranks" if world > 1 else "single GPU",
                    "workspace_gb": round(ws_bytes / 1e9, 2),
                    "peak_device_gb": round(torch.cuda.max_memory_allocated(dev) / 1e9, 2),
                    "flops_algorithmic_per_step": flops, "flops_issued_per_step_this_rank": plan["flops_issued"]},
           "e2e": e2e, "roofline": roofline, "clocks": clk.summary(), "gpu_launches": launches,
           "phases_ms_per_step": {k: round(v_["ms"] / a.steps, 3) for k, v_ in sorted(prof.items())}}

    if rank == 0 and not a.quick:
        extras(a, out, o, v, n, mode, L_np, t2_np, Lg, tg, R, ws, E_e2e, value, dev, stream, world)
        if a.large:
            del ws, Lg, tg, R, R_h
            torch.cuda.empty_cache()
            try:
                out["large"] = large_leg(a, dev, stream, mode)
            except Exception as e:  # noqa: BLE001 - reported in the JSON line, the main figures stand
                out["large"] = {"error": f"{type(e).__name__}: {e}"}
    if rank == 0:
        print(json.dumps(out), flush=True)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


def extras(a, out, o, v, n, mode, L_np, t2_np, Lg, tg, R, ws, E_e2e, value, dev, stream, world):
    """Rank 0's side legs: accuracy against the oracle, the other precision modes with their
    rooflines, the measured plain-FP64 speed-up, both contraction orders, the further terms,
    the adjoint, host-resident amplitudes, the large workload and the CPU baseline."""
    import numpy as np
    import torch

    from oracle import oracle as O
    from paper_2310_04559_gb300 import binding as B
    from paper_2310_04559_gb300 import synth

    pk, _ = peaks()
    probed = {}
    for name in ("dmma", "dfma", "tc_bf16", "tc_tf32", "imma"):
        try:
            probed[name] = B.peak_probe(name, device=dev)
        except Exception as e:  # noqa: BLE001 - reported, the main figures stand
            probed[name] = None
            out.setdefault("errors", []).append(f"probe {name}: {e}")
    out["peaks_probed_tflops"] = probed

    # accuracy on three `a` columns (all i, j, b) vs the FP64 oracle; the oracle's time on them
    # is the CPU baseline
    a_list = sorted({0, v // 2, v - 1})
    Rs, t_cpu, threads = oracle_sample(L_np, t2_np, a_list)
    rel = lambda X: float(np.linalg.norm(X[:, :, a_list, :] - Rs) / np.linalg.norm(Rs))
    full_R = R if world == 1 else None
    plan_of = lambda m: B.plan(o, v, n, ws_bytes=ws.numel(), mode=m, symmetric=True)

    def mode_entry(m, ms, Rm):
        issued = plan_of(m)["flops_issued"]
        peak, src = mode_peak(m, probed, pk)
        ach = issued / (ms / 1e3) / 1e12
        return {"tflops": algorithmic_flops(o, v, n) / (ms / 1e3) / 1e12, "ms": ms,
                "rel_err": rel(Rm.cpu().numpy()) if Rm is not None else None,
                "issued_tflops": ach, "peak": peak, "frac": ach / peak if peak else None, "peak_source": src}

    modes = {}
    if full_R is not None:
        modes[mode] = mode_entry(mode, out["ms_per_step"], full_R)
        modes[mode]["rel_err_columns"] = a_list
    for m in [x for x in a.other_modes.split(",") if x]:
        Rm = torch.empty_like(tg)
        ms = timed(stream, lambda: B.ladder_forward(Lg, tg, R=Rm, mode=m, symmetric=True, workspace=ws))
        modes[m] = mode_entry(m, ms, Rm)
        del Rm
    if a.fp64_full:
        R64 = torch.empty_like(tg)
        f0, f1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        f0.record(stream)
        B.ladder_forward(Lg, tg, R=R64, mode="fp64", symmetric=True, workspace=ws)
        f1.record(stream)
        torch.cuda.synchronize(dev)
        modes["fp64"] = mode_entry("fp64", f0.elapsed_time(f1), R64)
        modes["fp64"]["timed_on"] = "the full workload, one call"
        del R64
    out["modes"] = modes
    if mode in modes and "fp64" in modes:
        out["speedup_vs_fp64_mma"] = modes[mode]["tflops"] / modes["fp64"]["tflops"]
    if E_e2e is not None:
        out["energy_e2e"] = E_e2e

    # the two further Cholesky terms with the ladder's contraction (Eq. 8, Eq. 9), same workload
    Lov = torch.from_numpy(synth.cholesky_ov(n, o, v, seed=7)).to(dev)
    terms = {}
    for name, fl in (("tijbk", 2.0 * (n + o * o) * o * float(v) ** 3),
                     ("tijkl", 2.0 * (n + o * o) * o * o * float(v) ** 2)):
        call = (lambda: B.tijbk(Lov, Lg, tg, mode=mode, budget=40 << 30)) if name == "tijbk" else \
               (lambda: B.tijkl(Lov, tg, mode=mode, budget=40 << 30))
        ms = timed(stream, call)
        terms[name] = {"tflops": fl / (ms / 1e3) / 1e12, "ms": ms, "flops_algorithmic": fl}
    out["terms"] = terms
    del Lov

    # host-resident amplitudes: t2 and R in page-locked host memory, read and written over the
    # host link, the device holding L, one block of pairs and the integral blocks (40 GB budget)
    t2_h = torch.from_numpy(t2_np).pin_memory()
    Rh = torch.empty(t2_h.shape, dtype=torch.float64).pin_memory()
    hb = 40 << 30
    ms = timed(stream, lambda: B.ladder_forward(Lg, t2_h, R=Rh, mode=mode, symmetric=True, host_t2r=True, budget=hb))
    hp = B.plan(o, v, n, mode=mode, symmetric=True, host_t2r=True, budget=hb)
    out["host_resident"] = {"tflops": algorithmic_flops(o, v, n) / (ms / 1e3) / 1e12, "rel_err": rel(Rh.numpy()),
                            "device_budget_gb": round(hb / 1e9, 1), "a_blocks": hp["n_blocks"],
                            "ws_gb": round(hp["ws_bytes"] / 1e9, 2)}
    del t2_h, Rh
    sample_flops = 2.0 * (o * o + n) * float(v) ** 3 * len(a_list)
    out["cpu_baseline"] = {"value": sample_flops / t_cpu / 1e12, "unit": UNIT, "cores": threads, "kind": "oracle",
                           "cpu_model": cpu_model(),
                           "sample": f"R[:, :, a, :] for a in {a_list} of the same workload "
                                     f"({len(a_list)}/{v} of the work, {t_cpu:.1f} s)"}
    torch.cuda.empty_cache()

    # both contraction orders (Section 3.2) at the crossover shape and at o20/v200/n1000, each
    # timed after a warm-up call and counted against its own algorithmic flops (2(o^2+n)v^4
    # integral-first, 4 n o^2 v^3 Cholesky-first); o20/v200/n1000 in plain FP64 as well, which
    # gives the measured speed-up of emulated over plain FP64 at that workload
    orders = {}
    for (oo, vo, no), bud, ms_modes in (((4, 96, 480), 8 << 30, (mode,)),
                                        ((20, 200, 1000), 24 << 30, (mode, "fp64"))):
        key = f"o{oo}_v{vo}_n{no}"
        try:
            Lo_np, to_np = synth.ladder_inputs(oo, vo, no, seed=21)
            Lo, to = torch.from_numpy(Lo_np).to(dev), torch.from_numpy(to_np).to(dev)
            Ro = torch.empty_like(to)
            R_or = O.ladder(Lo_np, to_np, a_list=[0, vo - 1])
            rec = {}
            for m in ms_modes:
                for od, fl in (("integral_first", 2.0 * (oo * oo + no) * float(vo) ** 4),
                               ("cholesky_first", 4.0 * no * oo * oo * float(vo) ** 3)):
                    wso = B.alloc_workspace(B.workspace_size(oo, vo, no, mode=m, order=od, symmetric=True,
                                                             budget=bud), dev)
                    ms = timed(stream, lambda: B.ladder_forward(Lo, to, R=Ro, mode=m, order=od, symmetric=True,
                                                                workspace=wso))
                    err = float(np.linalg.norm(Ro.cpu().numpy()[:, :, [0, vo - 1], :] - R_or) / np.linalg.norm(R_or))
                    rec[f"{m}/{od}"] = {"ms": ms, "tflops": fl / (ms / 1e3) / 1e12, "flops_algorithmic": fl,
                                        "rel_err": err}
                    del wso
                rec[f"{m}/autotuner_choice"] = B.autotune(Lo, to, R=Ro, mode=m, symmetric=True, budget=bud)["order"]
            if "fp64" in ms_modes:
                best = lambda m: min(rec[f"{m}/integral_first"]["ms"], rec[f"{m}/cholesky_first"]["ms"])
                rec["speedup_vs_fp64_mma"] = best("fp64") / best(mode)
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
    gi = np.random.default_rng(6)
    i1, i2 = gi.integers(0, ta_np.size, 16), gi.integers(0, La_np.size, 16)
    g1_ref, g2_ref = O.ladder_grad_entries(La_np, ta_np, Wa_np, i1, i2)
    fwd_fl = algorithmic_flops(oa, va, na)
    adj = {"workload": "o16_v160_n800", "flops_forward": fwd_fl, "flops_backward": 2 * fwd_fl}
    for m in ("fp64", mode):
        tf = timed(stream, lambda: B.ladder_forward(La, ta, mode=m, symmetric=True))
        res = {}
        tb = timed(stream, lambda: res.update(g=B.ladder_backward(La, ta, Wa, mode=m, symmetric=True)))
        dLa, dta = res["g"]
        g1 = dta.cpu().numpy().ravel()[i1]
        g2 = dLa.cpu().numpy().ravel()[i2]
        adj[m] = {"forward_tflops": fwd_fl / (tf / 1e3) / 1e12, "backward_tflops": 2 * fwd_fl / (tb / 1e3) / 1e12,
                  "backward_ms": tb, "dt2_rel_err": float(np.linalg.norm(g1 - g1_ref) / np.linalg.norm(g1_ref)),
                  "dL_rel_err": float(np.linalg.norm(g2 - g2_ref) / np.linalg.norm(g2_ref))}
    out["adjoint"] = adj
    del La, ta, Wa


def large_leg(a, dev, stream, mode):
    """The largest workload (o=60, v=600, n_chol=3000, pCCD-LCCSD-sized): emulated FP64 under a
    150 GB device budget with the autotuned order, timed over two steps after a warm-up, and 24
    entries checked against the oracle's entries computed one by one."""
    import numpy as np
    import torch

    from oracle import oracle as O
    from paper_2310_04559_gb300 import binding as B
    from paper_2310_04559_gb300 import synth

    o, v, n = WORKLOADS["o60_v600_n3000"]
    torch.cuda.empty_cache()
    torch.cuda.reset_peak_memory_stats(dev)
    t0 = time.perf_counter()
    L, t2 = synth.ladder_inputs_torch(o, v, n, seed=0, device=dev)
    t_gen = time.perf_counter() - t0
    R = torch.empty_like(t2)
    budget = int(a.budget_gb * 1e9) - L.numel() * 8 - 2 * t2.numel() * 8 - (2 << 30)
    tune = B.autotune(L, t2, R=R, mode=mode, symmetric=True, budget=budget)
    ws_bytes = B.workspace_size(o, v, n, mode=mode, symmetric=True, budget=budget)
    ws = B.alloc_workspace(ws_bytes, dev)
    plan = B.plan(o, v, n, ws_bytes=ws_bytes, mode=mode, symmetric=True)
    B.profile_enable(True)
    ms = timed(stream, lambda: B.ladder_forward(L, t2, R=R, mode=mode, symmetric=True, workspace=ws), reps=2)
    prof = B.profile_read()
    B.profile_enable(False)
    tc = [k for k in prof if k.endswith("_tc")]
    tc_ms = sum(prof[k]["ms"] for k in tc)
    tc_fl = sum(prof[k]["flops"] for k in tc)
    pk, _ = peaks()
    peak = pk.get("bf16_tflops_sustained", pk["bf16_tflops"])
    ach = tc_fl / (tc_ms / 1e3) / 1e12 if tc_ms else None
    gi = np.random.default_rng(8)
    idx = gi.integers(0, R.numel(), 24)
    idx[:4] = [0, R.numel() - 1, ((1 * o + 1) * v + 3) * v + 3, ((5 * o + 2) * v + 599) * v]
    got = R.view(-1)[torch.from_numpy(idx).to(dev)].cpu().numpy()
    ref = O.ladder_entries(L.cpu().numpy(), t2.cpu().numpy(), idx)
    return {"workload": "o60_v600_n3000", "tflops": algorithmic_flops(o, v, n) / (ms / 1e3) / 1e12, "ms": ms,
            "order": tune["order"], "n_blocks": plan["n_blocks"], "peak_device_gb":
            round(torch.cuda.max_memory_allocated(dev) / 1e9, 2),
            "roofline": {"achieved": ach, "peak": peak, "frac": ach / peak if ach else None,
                         "unit": "TFLOP/s", "flops_issued_per_step": plan["flops_issued"]},
            "rel_err_sampled_entries": float(np.linalg.norm(got - ref) / np.linalg.norm(ref)),
            "inputs": f"drawn on the device with torch's generator, same recipe ({t_gen:.1f} s)"}


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
        "data": "synthetic", "config": workload_config(a.workload),
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
    p.add_argument("--other-modes", default="tf32,bf16")
    p.add_argument("--no-fp64-full", dest="fp64_full", action="store_false",
                   help="skip the plain-FP64 run of the whole workload")
    p.add_argument("--no-large", dest="large", action="store_false", help="skip the o60/v600/n3000 leg")
    p.add_argument("--quick", action="store_true", help="skip every side leg (accuracy, modes, CPU baseline, ...)")
    a = p.parse_args(argv)
    if a.warmup < 3:
        p.error("--warmup must be >= 3")
    if a.impl == "reference":
        run_reference(a)
    else:
        run_ours(a)


if __name__ == "__main__":
    main()
