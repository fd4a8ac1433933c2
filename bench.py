"""Benchmark: FTLM H.v throughput in states x vectors per second.

One step = one whole FTLM run (all rows of the hot path): start block of R
random vectors, M Lanczos steps (matvec with fused reductions, recurrence
update), tridiagonal eigensolves and the Boltzmann sums of Eqs. (4)-(5), on
the open 4x5 s=1/2 lattice with all-pairs dipolar coupling (N = 20,
d = 1,048,576, R = 64, M = 200, complex64 vectors with FP32 matvec and FP64
scalars).  value = d * R * M * steps * n_gpus / time, time from CUDA events
on the run's stream (max over ranks).

--impl reference times the FP64 CPU oracle instead, on bounded samples of
the same workload (R = number of oracle threads, a few Lanczos steps).

Multi-GPU (torchrun): every rank runs its own R vectors (vec_offset =
rank * R); no collective touches the data path (weak scaling).
"""
from __future__ import annotations

import argparse
import json
import os
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import ftlm_workloads as W  # noqa: E402

METRIC = "FTLM H·v states×vectors/s, batched FP32 vs plain FP64 at N=20; %HBM roof"
UNIT = "states*vectors/s"
WORKLOAD = "lattice4x5"
SM_COUNT = 152
FP32_LANES_PER_SM = 128


def load_peaks():
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except Exception:
        return {}


def algorithmic_flops_per_sv(two_s, epilogue=True):
    """Flops one state x vector needs per Lanczos step in the matvec, averaged
    over the product basis (site i has q_i = 2 s_i + 1 levels; a raising flip
    is possible from q_i - 1 of them, a double flip from q_i - 2): a pair's
    s+ s- / s- s+ terms have a real coefficient (4 flops each), its s+ s+ /
    s- s- terms a complex one (8 flops); every single-site flip by one or two
    levels is complex (8 flops); the diagonal is real (2 flops); the fused
    epilogue (the beta term, alpha and p reductions) adds 14.  For s = 1/2
    every pair has exactly one possible flip: 6 flops on average."""
    q = np.asarray(two_s, dtype=np.float64) + 1.0
    up = (q - 1.0) / q            # P(a site can be raised) = P(it can be lowered)
    up2 = np.maximum(q - 2.0, 0.0) / q
    flops = 2.0 + (14.0 if epilogue else 0.0)
    n = len(q)
    for i in range(n):
        flops += 8.0 * 2.0 * up[i] + 8.0 * 2.0 * up2[i]
        for j in range(i + 1, n):
            flops += 4.0 * 2.0 * up[i] * up[j] + 8.0 * 2.0 * up[i] * up[j]
    return float(flops)


def gather_kernel_name(shp):
    """The H.v kernel a launch shape names."""
    if shp.get("vector_major") and shp.get("cube_bits", 0) > 0:
        return f"vm_kernel<float,{shp['cube_bits']}> (vector-major spin-1/2 gather)"
    if shp.get("vector_major") and shp.get("site_cube", 0) > 0:
        return (f"cube_gather_kernel<float,{shp['site_cube']},{shp['group_vectors']}> (vector-major general gather, "
                f"register cube of the top site's {shp['site_cube']} rows, the step's w' in its epilogue)")
    if shp.get("vector_major"):
        return f"rows_vm_kernel<float,{shp['group_vectors']}> (vector-major general gather)"
    if shp.get("cube_bits", 0) > 0:
        return f"half_kernel<float,{shp['cube_bits']}> (row-major spin-1/2 register-cube gather)"
    return "rows_kernel (row-major general gather)"


def batch_roofline(systems_two_s, dims, R, hv_ms, sm_max_mhz, kernel, epilogue):
    """FP32 roofline of one H.v launch over a batch (epilogue: the launch also
    forms the Lanczos step's w' and its alpha and p sums, as the register-cube
    gather does; the one-row gathers leave them to the next launch)."""
    flops = sum(algorithmic_flops_per_sv(t, epilogue=epilogue) * d * R for t, d in zip(systems_two_s, dims))
    achieved = flops / (hv_ms / 1e3) / 1e12
    peak = SM_COUNT * FP32_LANES_PER_SM * 2 * sm_max_mhz * 1e6 / 1e12
    return {"bound": "alu", "kernel": kernel, "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
            "frac": achieved / peak, "flops_per_launch": flops, "hv_ms_per_launch": hv_ms,
            "peak_note": "FP32 FMA peak = 152 SMs x 128 lanes x 2 flop x max SM clock (derived)"}


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index=0):
        self.f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
        self.proc = None
        self.gpu = gpu_index

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.f.flush()
        rows = [ln.split(",") for ln in open(self.f.name).read().strip().splitlines() if ln.strip()]
        os.unlink(self.f.name)
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in rows:
            try:
                sm.append(float(r[1]))
                mx = float(r[2])
                for k, nm in enumerate(names):
                    if r[5 + k].strip().lower().startswith("active"):
                        reasons.add(nm)
            except (ValueError, IndexError):
                continue
        return {"sm_mhz": float(np.median(sm)) if sm else None, "sm_max_mhz": mx, "reasons": sorted(reasons),
                "samples": len(sm)}


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def run_ours(args):
    import torch
    import torch.distributed as dist

    import paper_2607_25585_gb300 as F

    ws, rank, local = dist_env()
    torch.cuda.set_device(local)
    if ws > 1:
        dist.init_process_group("nccl", init_method="env://")
    F.build()
    spec = W.WORKLOADS[WORKLOAD]
    w = spec["system"]()
    R, M = spec["R"], args.M or spec["M"]
    T = W.temperatures()
    s = F.System.from_dict(w)
    d = s.dim
    stream = torch.cuda.Stream()
    kw = dict(R=R, M=M, T=T, seed=spec["seed"], vec_offset=rank * R, dtype="c64", stream=stream,
              time_kernels=True)
    if args.shape:
        F.tune_shape(s, R, "c64", *[int(v) for v in args.shape.split(",")])
        F.run(s, **kw)                     # captures the graph
    else:
        F.run(s, autotune=args.autotune, **kw)  # (tunes launch shapes,) captures the graph
    for _ in range(args.warmup):
        F.run(s, **kw)
    sampler = ClockSampler(local)
    if ws > 1:
        dist.barrier()
    torch.cuda.synchronize()
    sampler.start()
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    ev0.record(stream)
    hv_ms, launches, hv_launches, results = 0.0, 0, 0, None
    for _ in range(args.steps):
        results = F.run(s, **kw)
        hv_ms += results["hv_ms"]
        launches += results["kernel_launches"]
        hv_launches += results["hv_launches"]
    ev1.record(stream)
    torch.cuda.synchronize()
    clocks = sampler.stop()
    ms = ev0.elapsed_time(ev1)
    if ws > 1:
        t = torch.tensor([ms], device="cuda")
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        ms = float(t.item())
        dist.barrier()
    sv_per_step = d * R * M
    value = sv_per_step * args.steps * ws / (ms / 1e3)

    # end to end through the C ABI from host inputs: create the system from
    # host arrays, run, read the results back, destroy -- every step
    e2e = None
    if not args.no_e2e:
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        h2d = d2h = 0
        for _ in range(max(1, min(args.steps, 3))):
            s2 = F.System.from_dict(w)
            r2 = F.run(s2, R=R, M=M, T=T, seed=spec["seed"], vec_offset=rank * R, dtype="c64")
            h2d += s2.table_bytes + r2["h2d_bytes"]
            d2h += r2["d2h_bytes"]
            s2.close()
        n_e2e = max(1, min(args.steps, 3))
        torch.cuda.synchronize()
        e2e_s = time.perf_counter() - t0
        e2e = {"value": sv_per_step * n_e2e * ws / e2e_s, "unit": UNIT, "h2d_bytes_per_step": int(h2d / n_e2e),
               "d2h_bytes_per_step": int(d2h / n_e2e), "steps": n_e2e}

    peaks = load_peaks()
    hbm = peaks.get("hbm_gbs", 6778.0)
    line = None
    if rank == 0:
        # dominant kernel: the fused H.v + Lanczos epilogue
        hv_per_launch_ms = hv_ms / max(1, hv_launches)
        flops_sv = algorithmic_flops_per_sv(w["two_s"])
        achieved = flops_sv * d * R / (hv_per_launch_ms / 1e3) / 1e12
        sm_max = clocks.get("sm_max_mhz") or peaks.get("sm_max_mhz", 2070.0)
        fp32_peak = SM_COUNT * FP32_LANES_PER_SM * 2 * sm_max * 1e6 / 1e12
        shp = results["shape"]
        if shp.get("vector_major"):
            kname = (f"vm_kernel<float,{shp['cube_bits']},{'multi' if shp['passes'] > 1 else 'single'}> "
                     f"(vector-major spin-1/2 gather{', %d passes' % shp['passes'] if shp['passes'] > 1 else ''})")
        elif shp["cube_bits"] > 0:
            kname = (f"half_kernel<float,{shp['cube_bits']},Apply,{64 if R == 64 else 0},"
                     f"{'multi' if shp['passes'] > 1 else 'single'}> (spin-1/2 register-cube gather)")
        else:
            kname = "rows_kernel<float,2,Lanczos> (general gather with the fused step)"
        traffic = measured_traffic(shp)
        precision = None if args.no_precision else precision_legs(F, T, stream, args, s, spec, results)
        plain = None if args.no_plain else plain_fp64(F, s, T, spec, stream, args)
        extra = None if args.no_extra else extra_workloads(F, T, stream, args)
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": f"open 4x5 s=1/2 lattice, all-pairs dipolar, d={d}, R={R} vectors, M={M} "
                                   "Lanczos steps, complex64 vectors, FP32 matvec, FP64 scalars/eigensolve/sums",
                       "d": d, "R": R, "M": M, "global_batch_vectors": R * ws, "parallelism": f"replicas x{ws}",
                       "l2": "inputs larger than L2 (four 512 MB vector blocks: q_j, q_{j-1}, H q_j, u)"},
            "hbm_roof_frac": value / ws * 32 / (hbm * 1e9),
            "roofline": {"bound": "alu", "kernel": kname,
                         "achieved": achieved, "peak": fp32_peak, "unit": "TFLOP/s", "frac": achieved / fp32_peak,
                         "traffic": traffic, "algorithmic_flops_per_sv": flops_sv,
                         "hv_ms_per_launch": hv_per_launch_ms, "launch_shape": results["shape"],
                         "launch_gap_ms_per_step": results["gap_ms"] / max(1, M - 1),
                         "peak_note": "FP32 FMA peak = 152 SMs x 128 lanes x 2 flop x max SM clock (derived)"},
            "hbm": {"bytes_per_sv": 32, "peak_gbs": hbm, "peak_source": "MEASURED_PEAKS.json hbm_gbs (measured)",
                    "frac": value / ws * 32 / (hbm * 1e9)},
            "plain_fp64": plain,
            "fp32_vs_fp64": precision,
            "other_workloads": extra,
            "clocks": clocks, "e2e": e2e, "gpu_launches": launches,
        }
        if plain and plain.get("value"):
            line["speedup_vs_plain_fp64"] = value / ws / plain["value"]
        if precision and precision.get("lattice4x5", {}).get("fp64_value"):
            line["speedup_vs_batched_fp64"] = value / ws / precision["lattice4x5"]["fp64_value"]
        if args.cpu_baseline and ws == 1:
            line["cpu_baseline"] = cpu_baseline(args)
    s.close()
    if ws > 1:
        dist.destroy_process_group()
    return line


def measured_traffic(shape):
    """DRAM bytes per launch of the dominant kernel from the committed ncu
    capture, or None when the kernel source or its launch shape has changed
    since the counters were taken."""
    import hashlib
    tf = os.path.join(ROOT, "profiles", "traffic_lattice4x5.json")
    try:
        recs = json.load(open(tf))["records"]
    except Exception:
        return None
    for rec in recs:
        try:  # every source file of the kernel as it was when the counters were taken
            same = all(hashlib.sha256(open(os.path.join(ROOT, f), "rb").read()).hexdigest() == h
                       for f, h in rec["sources"].items())
        except (OSError, KeyError):
            continue
        if not same:
            continue
        if any(rec["shape"][k] != shape.get(k) for k in rec["shape"]):
            continue
        return rec["bytes_per_launch"]
    return None


def per_t_errors(a, b, T, floor=1e-3):
    """Relative error of every thermodynamic result of run a against run b at
    each temperature, with a floor of `floor` times the quantity's maximum
    over T (quantities that pass through zero), its maximum over T >= 0.1 K,
    the absolute error over T >= 0.1 K on the scale of the quantity's largest
    value, and run b's values."""
    out = {}
    cold = T >= 0.1
    for k in ("lnZ", "E", "C", "M_B"):
        x, y = np.asarray(a[k]), np.asarray(b[k])
        e = np.abs(x - y) / np.maximum(np.abs(y), floor * np.max(np.abs(y)))
        out[k] = {"max_T_ge_0.1": float(e[cold].max()), "max_all_T": float(e.max()),
                  "per_T": [float(v) for v in e],
                  # the absolute error on the scale of the quantity (its largest |value| over T)
                  "abs_over_max_T_ge_0.1": float((np.abs(x - y)[cold]).max() / np.max(np.abs(y))),
                  "fp64_per_T": [float(v) for v in y]}
    out["max_T_ge_0.1"] = max(out[k]["max_T_ge_0.1"] for k in ("lnZ", "E", "C", "M_B"))
    return out


def timed_run(F, s, stream, **kw):
    """One run timed with CUDA events on its stream (the graph is captured in
    the same call: tens of ms, against runs of seconds here)."""
    import torch
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    res = F.run(s, stream=stream, **kw)
    e1.record(stream)
    torch.cuda.synchronize()
    return res, e0.elapsed_time(e1)


def precision_legs(F, T, stream, args, s_head, spec_head, res_head):
    """FP32 (complex64 vectors, FP32 matvec, FP64 scalars) against FP64
    (complex128, the same kernels in double) on the same random vectors,
    per temperature: the 4x5 lattice at its full R = 64, M = 200 (the c64 run
    is the headline's last timed run; the c128 run of the whole block is also
    the batched-FP64 throughput) and the 2x13 ladder at M = 300 (both timed as
    full runs) with its R = 4 vectors (--ladder-precision-R; the FP64 run
    takes about three minutes, bound by the FP64 pipes)."""
    out = {}
    R, M = spec_head["R"], args.M or spec_head["M"]
    d = s_head.dim
    r128, ms128 = timed_run(F, s_head, stream, R=R, M=M, T=T, seed=spec_head["seed"], dtype="c128")
    out["lattice4x5"] = {"R": R, "M": M, "d": d, "fp64_value": d * R * M / (ms128 / 1e3), "fp64_ms": ms128,
                         "fp64_launch_shape": r128["shape"], "unit": UNIT,
                         "errors_vs_fp64": per_t_errors(res_head, r128, T),
                         "note": "same Philox vectors; FP64 = complex128 block of all 64 vectors (batched FP64)"}
    if not args.no_ladder_precision:
        spec = W.WORKLOADS["ladder2x13"]
        s = F.System.from_dict(spec["system"]())
        R, M = args.ladder_precision_R, spec["M"]
        d = s.dim
        r64, ms64 = timed_run(F, s, stream, R=R, M=M, T=T, seed=spec["seed"], dtype="c64", time_kernels=True)
        r128, ms128 = timed_run(F, s, stream, R=R, M=M, T=T, seed=spec["seed"], dtype="c128")
        out["ladder2x13"] = {"R": R, "M": M, "d": d, "fp32_value": d * R * M / (ms64 / 1e3), "fp32_ms": ms64,
                             "fp64_value": d * R * M / (ms128 / 1e3), "fp64_ms": ms128, "unit": UNIT,
                             "fp32_hv_ms_per_launch": r64["hv_ms"] / max(1, r64["hv_launches"]),
                             "fp32_launch_shape": r64["shape"], "fp64_launch_shape": r128["shape"],
                             "errors_vs_fp64": per_t_errors(r64, r128, T)}
        s.close()
    out["T"] = [float(t) for t in T]
    return out


def plain_fp64(F, s, T, spec, stream, args):
    """The plain FP64 GPU path: complex128, one Lanczos chain at a time (R = 1),
    same gather kernels; timed on a bounded sample of chains."""
    import torch
    d = s.dim
    M = args.M or spec["M"]
    chains = args.plain_chains
    kw = dict(R=1, M=M, T=T, seed=spec["seed"], dtype="c128", stream=stream)
    F.run(s, autotune=args.autotune, **kw)
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    ev0.record(stream)
    for c in range(chains):
        F.run(s, vec_offset=c, **kw)
    ev1.record(stream)
    torch.cuda.synchronize()
    ms = ev0.elapsed_time(ev1)
    return {"value": d * M * chains / (ms / 1e3), "unit": UNIT, "chains": chains, "M": M,
            "sample": f"{chains} complex128 chains (R=1) x {M} steps on the same system"}


def extra_workloads(F, T, stream, args):
    """Bounded measurements of the other workloads (reported beside the
    headline, not part of it): the uneven-size batch of 24 s = 1 chains in
    one graph (one full run), and the N = 26 ladder (a run of --ladder-steps
    Lanczos steps)."""
    import torch
    out = {}
    spec = W.WORKLOADS["chains_s1_x24"]
    ws_ = spec["system"]()
    systems = [F.System.from_dict(w) for w in ws_]
    R, M = spec["R"], spec["M"]
    kw = dict(R=R, M=M, T=T, seed=spec["seed"], dtype="c64", stream=stream, time_kernels=True)
    F.run_batch(systems, autotune=True, **kw)  # the autotuner picks the launch shape (kept for the timed run)
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    res = F.run_batch(systems, **kw)
    e1.record(stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1)
    sv = sum(s.dim for s in systems) * R * M
    out["chains_s1_x24"] = {"value": sv / (ms / 1e3), "unit": UNIT, "ms_per_run": ms, "M": M, "R": R,
                            "instances": len(systems), "hv_ms_per_launch": res[0]["hv_ms"] / max(1, res[0]["hv_launches"]),
                            "launch_gap_ms_per_step": res[0]["gap_ms"] / max(1, M - 1),
                            "launch_gap_share": res[0]["gap_ms"] / max(1e-9, res[0]["device_ms"]),
                            "launch_shape": res[0]["shape"], "autotuned": True,
                            "roofline": batch_roofline([w["two_s"] for w in ws_], [s.dim for s in systems], R,
                                                       res[0]["hv_ms"] / max(1, res[0]["hv_launches"]),
                                                       load_peaks().get("sm_max_mhz", 2070.0),
                                                       gather_kernel_name(res[0]["shape"]),
                                                       res[0]["shape"].get("site_cube", 0) > 0),
                            "note": "one graph for all 24 instances; shape chosen by the autotuner"}
    for s in systems:
        s.close()
    spec = W.WORKLOADS["ladder2x13"]
    s = F.System.from_dict(spec["system"]())
    R, M = spec["R"], args.ladder_steps
    kw = dict(R=R, M=M, T=T, seed=spec["seed"], dtype="c64", stream=stream, time_kernels=True)
    F.run(s, autotune=args.autotune, **kw)
    e0.record(stream)
    res = F.run(s, **kw)
    e1.record(stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1)
    out["ladder2x13"] = {"value": s.dim * R * M / (ms / 1e3), "unit": UNIT, "ms_per_run": ms, "M": M, "R": R,
                         "hv_ms_per_launch": res["hv_ms"] / max(1, res["hv_launches"]), "launch_shape": res["shape"],
                         "note": f"sample of {M} Lanczos steps (the workload runs 300)"}
    s.close()
    out["time_reversed_pairs"] = time_reversal_leg(F, T, stream)
    out["mn9_powder"] = mn9_leg(F, T, stream, args)
    out["mn9_symmetric"] = sftlm_leg(F, T, stream)
    out["stored_matrix"] = stored_matrix_leg(F, stream)
    return out


def stored_matrix_leg(F, stream):
    """The stored-matrix comparison path on the headline system: assembly
    time and memory, and one H.v with the stored matrix against the
    matrix-free ftlm_apply_h on the same row-major block (complex64 with
    R = 64, and complex128 with R = 1 as in the plain FP64 path)."""
    import time
    import torch
    spec = W.WORKLOADS[WORKLOAD]
    s = F.System.from_dict(spec["system"]())
    d = s.dim
    out = {}
    for dtype, R in (("c64", spec["R"]), ("c128", 1)):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        m = F.CsrMatrix(s, dtype)
        build_s = time.perf_counter() - t0
        tdt = torch.complex64 if dtype == "c64" else torch.complex128
        x = torch.randn(d, R, dtype=tdt, device="cuda")
        y = torch.empty_like(x)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        res = {}
        for name, fn in (("stored", lambda: m.apply(x, y, R, stream=stream)),
                         ("matrix_free", lambda: F.apply_h(s, x, y, R, dtype, stream=stream))):
            for _ in range(2):
                fn()
            e0.record(stream)
            for _ in range(5):
                fn()
            e1.record(stream)
            torch.cuda.synchronize()
            res[name] = e0.elapsed_time(e1) / 5
        out[f"{dtype}_R{R}"] = {"stored_ms": res["stored"], "matrix_free_ms": res["matrix_free"],
                                "matrix_free_speedup": res["stored"] / res["matrix_free"], "nnz": m.nnz,
                                "matrix_bytes": m.bytes, "build_s": build_s,
                                "stored_gbs": (m.bytes + 2 * d * R * x.element_size()) / (res["stored"] / 1e3) / 1e9}
        m.close()
        del x, y
    s.close()
    return out


def sftlm_leg(F, T, stream):
    """Symmetric FTLM (Eqs. E-2-G, E-2-H) on the Mn9-like system along one
    dodecahedron direction: the run with its Lanczos vectors kept, then
    O_ij = <v_i|u.S|v_j> on the device; against the plain run of the same
    vectors."""
    import torch
    spec = W.WORKLOADS["mn9_powder"]
    w = spec["system"]()[0]
    s = F.System.from_dict(w)
    R, M = spec["R"], spec["M"]
    kw = dict(R=R, M=M, T=T, seed=spec["seed"], dtype="c64", stream=stream, start="pairs")
    times = {}
    for sym in (False, True):
        F.run(s, symmetric=sym, **kw)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        res = F.run(s, symmetric=sym, **kw)
        e1.record(stream)
        torch.cuda.synchronize()
        times[sym] = (e0.elapsed_time(e1), res)
    ms_sym, res = times[True]
    d = int(s.dim)
    s.close()
    return {"value": d * R * M / (ms_sym / 1e3), "unit": UNIT, "ms_per_run": ms_sym, "plain_ms_per_run": times[False][0],
            "sym_ms": res["sym_ms"], "overhead": ms_sym / times[False][0], "R": R, "M": M, "d": d,
            "stored_vector_bytes": d * R * M * 8,
            "M_B_sym_minus_M_B_at_T": {f"{T[i]:.3g}": float(res["M_B_sym"][i] - res["M_B"][i]) for i in (0, 20, 39)},
            "note": "states x vectors/s of the whole symmetric run; O formed from the stored Lanczos vectors"}


def mn9_leg(F, T, stream, args):
    """The mixed-spin Mn9-like system (d = 2,343,750) at 1 T along the 10
    dodecahedron directions, as one batch (one graph), with time-reversed
    start pairs; the powder average of M_B is over the 10 results."""
    import torch
    spec = W.WORKLOADS["mn9_powder"]
    ws_ = spec["system"]()
    systems = [F.System.from_dict(w) for w in ws_]
    R, M = spec["R"], spec["M"]
    kw = dict(R=R, M=M, T=T, seed=spec["seed"], dtype="c64", stream=stream, time_kernels=True, start="pairs")
    F.run_batch(systems, autotune=args.autotune, **kw)
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    res = F.run_batch(systems, **kw)
    e1.record(stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1)
    sv = sum(s.dim for s in systems) * R * M
    d = int(systems[0].dim)
    mb = np.mean([r["M_B"] for r in res], axis=0)
    hv = res[0]["hv_ms"] / max(1, res[0]["hv_launches"])
    roof = batch_roofline([w["two_s"] for w in ws_], [s.dim for s in systems], R, hv,
                          load_peaks().get("sm_max_mhz", 2070.0), gather_kernel_name(res[0]["shape"]),
                          res[0]["shape"].get("site_cube", 0) > 0)
    for s in systems:
        s.close()
    return {"value": sv / (ms / 1e3), "unit": UNIT, "ms_per_run": ms, "M": M, "R": R, "directions": len(systems),
            "d": d, "hv_ms_per_launch": hv, "roofline": roof,
            "launch_shape": res[0]["shape"], "powder_M_B_at_T": {f"{T[i]:.3g}": float(mb[i]) for i in (0, 20, 39)},
            "note": "one graph for the 10 directions; general mixed-radix gather (launch_shape, roofline.kernel)"}


def time_reversal_leg(F, T, stream):
    """Time-reversed start pairs (tau = 1) on the headline system: one FTLM
    run with pairs (same throughput as random starts: only the start block
    differs), and ftlm_time_reverse on the [d][R] complex64 block, an
    HBM-bound permutation (read 8 B + write 8 B per state x vector)."""
    import torch
    spec = W.WORKLOADS[WORKLOAD]
    s = F.System.from_dict(spec["system"]())
    d, R = s.dim, spec["R"]
    kw = dict(R=R, M=20, T=T, seed=spec["seed"], dtype="c64", stream=stream, start="pairs")
    F.run(s, **kw)
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    F.run(s, **kw)
    e1.record(stream)
    torch.cuda.synchronize()
    run_ms = e0.elapsed_time(e1)
    x = torch.empty(d, R, dtype=torch.complex64, device="cuda")
    F.start_pairs(s, x, R, seed=1, dtype="c64", stream=stream)
    y = torch.empty_like(x)
    for _ in range(3):
        F.time_reverse(s, x, y, R, "c64", stream=stream)
    n = 20
    e0.record(stream)
    for _ in range(n):
        F.time_reverse(s, x, y, R, "c64", stream=stream)
    e1.record(stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / n
    hbm = load_peaks().get("hbm_gbs", 6778.0)
    gbs = 2 * d * R * 8 / (ms / 1e3) / 1e9
    s.close()
    return {"run_value": d * R * 20 / (run_ms / 1e3), "unit": UNIT, "run_M": 20, "R": R,
            "time_reverse_ms": ms, "time_reverse_gbs": gbs, "time_reverse_hbm_frac": gbs / hbm,
            "note": "run: 20 Lanczos steps from 32 pairs; time_reverse: 2 x 8 B per state x vector moved"}


def cpu_baseline(args, steps=None):
    """The oracle as it stands on the host cores: R = #threads vectors x a few
    Lanczos steps of the same workload."""
    import oracle
    oracle.build()
    spec = W.WORKLOADS[WORKLOAD]
    w = spec["system"]()
    s = oracle.System(**{k: v for k, v in w.items() if k != "name"})
    cores = oracle.num_threads()
    M = args.cpu_steps
    t0 = time.perf_counter()
    oracle.ftlm(s, R=cores, M=M, T=W.temperatures(), seed=spec["seed"])
    dt = time.perf_counter() - t0
    # the same on one host thread (one vector: the oracle threads over vectors)
    t0 = time.perf_counter()
    oracle.ftlm(s, R=1, M=M, T=W.temperatures(), seed=spec["seed"])
    dt1 = time.perf_counter() - t0
    return {"value": s.dim * cores * M / dt, "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": f"{cores} vectors x {M} Lanczos steps of the full d={s.dim} system "
                      f"(plain C++ FP64 oracle, OpenMP over vectors), {dt:.1f} s",
            "single_thread": {"value": s.dim * M / dt1, "unit": UNIT, "cores": 1,
                              "sample": f"1 vector x {M} Lanczos steps of the same system, {dt1:.1f} s"}}


def run_reference(args):
    ws, rank, _ = dist_env()
    if rank != 0:
        return None
    import oracle
    oracle.build()
    spec = W.WORKLOADS[WORKLOAD]
    w = spec["system"]()
    s = oracle.System(**{k: v for k, v in w.items() if k != "name"})
    cores = oracle.num_threads()
    M = args.cpu_steps
    T = W.temperatures()
    for _ in range(args.warmup):
        oracle.ftlm(s, R=cores, M=1, T=T, seed=spec["seed"])
    t0 = time.perf_counter()
    for _ in range(args.steps):
        oracle.ftlm(s, R=cores, M=M, T=T, seed=spec["seed"])
    dt = time.perf_counter() - t0
    value = s.dim * cores * M * args.steps / dt
    sample = (f"each step: {cores} vectors x {M} Lanczos steps of the full d={s.dim} system "
              "(plain C++ FP64 oracle, OpenMP over vectors)")
    return {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": dt * 1e3 / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": "open 4x5 s=1/2 lattice, all-pairs dipolar, d=1048576 (oracle sample)",
                       "R": cores, "M": M},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": sample},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}


def run_profile(args):
    """One short Lanczos run (R vectors, M steps, complex64) of the workload
    through ftlm_run, with the default plan or --shape: the launches a profiler
    captures are those of the timed runs, on a case small enough to capture."""
    import paper_2607_25585_gb300 as F

    F.build()
    R, M = (int(v) for v in args.profile_run.split(","))
    spec = W.WORKLOADS[args.hv_workload]
    w = spec["system"]()
    if isinstance(w, list):  # a batch: the largest instance
        w = max(w, key=lambda v: int(np.prod(v["two_s"].astype(np.int64) + 1)))
    s = F.System.from_dict(w)
    if args.shape:
        F.tune_shape(s, R, "c64", *[int(v) for v in args.shape.split(",")])
    out = F.run(s, R=R, M=M, T=W.temperatures(), seed=spec["seed"], dtype="c64", time_kernels=True)
    return {"mode": "profile_run", "workload": args.hv_workload, "d": s.dim, "R": R, "M": M,
            "hv_ms_per_launch": out["hv_ms"] / max(1, out["hv_launches"]),
            "device_ms_per_step": out["device_ms"] / M, "launch_shape": out["shape"]}


def run_profile_batch(args):
    """One run of a batch workload (--batch-workload: the 24 s = 1 chains x
    field directions, R = 16, M = 120, or the 10-direction Mn9-like powder
    batch, R = 8, M = 40; complex64, one graph) with the library's default
    launch shape or --shape (cube_bits,group_vectors,tile_cubes,multipass as
    in ftlm_tune_shape, set for the largest system): device time of the whole
    graph from CUDA events, for comparison with the summed kernel durations
    of an ncu launch list of the same command (the difference is the launch
    gaps)."""
    import torch

    import paper_2607_25585_gb300 as F

    F.build()
    spec = W.WORKLOADS[args.batch_workload]
    systems = [F.System.from_dict(w) for w in spec["system"]()]
    R, M = spec["R"], spec["M"]
    if args.shape:
        F.tune_shape(max(systems, key=lambda s: s.dim), R, "c64", *[int(v) for v in args.shape.split(",")])
    T = W.temperatures()
    stream = torch.cuda.Stream()
    kw = dict(R=R, M=M, T=T, seed=spec["seed"], dtype="c64", stream=stream,
              start="pairs" if args.batch_workload == "mn9_powder" else "random")
    F.run_batch(systems, **kw)  # captures the graph
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    res = F.run_batch(systems, **kw)
    e1.record(stream)
    torch.cuda.synchronize()
    return {"mode": "profile_batch", "workload": args.batch_workload, "instances": len(systems), "R": R, "M": M,
            "graph_ms": e0.elapsed_time(e1), "kernel_launches": res[0]["kernel_launches"],
            "launch_shape": res[0]["shape"]}


def run_hv_only(args):
    """ftlm_apply_h alone: args.hv_only launches of H.v on the workload's
    row-major [d][R] complex64 block (the row-major kernels, as a caller of
    ftlm_apply_h gets them), timed with CUDA events."""
    import torch

    import paper_2607_25585_gb300 as F

    F.build()
    spec = W.WORKLOADS[args.hv_workload]
    w = spec["system"]()
    if isinstance(w, list):  # a batch: the largest instance
        w = max(w, key=lambda v: int(np.prod(v["two_s"].astype(np.int64) + 1)))
    s = F.System.from_dict(w)
    d, R = s.dim, spec["R"]
    g = torch.Generator(device="cuda").manual_seed(1)
    x = torch.randn(d, R, dtype=torch.complex64, device="cuda", generator=g)
    y = torch.empty_like(x)
    for _ in range(2):
        F.apply_h(s, x, y, R, "c64")
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(args.hv_only):
        F.apply_h(s, x, y, R, "c64")
    e1.record()
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / args.hv_only
    return {"mode": "hv_only", "workload": args.hv_workload, "d": d, "R": R, "launches": args.hv_only,
            "ms_per_launch": ms, "states_vectors_per_s": d * R / (ms / 1e3)}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--M", type=int, default=0, help="Lanczos steps per run (default: the workload's 200)")
    ap.add_argument("--cpu-steps", type=int, default=2, help="Lanczos steps of the oracle sample")
    ap.add_argument("--plain-chains", type=int, default=2)
    ap.add_argument("--no-plain", action="store_true")
    ap.add_argument("--no-precision", action="store_true", help="skip the FP32-vs-FP64 legs")
    ap.add_argument("--no-ladder-precision", action="store_true", help="skip the 2x13 ladder in the FP32-vs-FP64 legs")
    ap.add_argument("--ladder-precision-R", type=int, default=4,
                    help="vectors of the 2x13 ladder's FP32-vs-FP64 comparison (the workload's R, 4, by default)")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-extra", action="store_true", help="skip the batch and ladder measurements")
    ap.add_argument("--ladder-steps", type=int, default=20)
    ap.add_argument("--no-cpu-baseline", dest="cpu_baseline", action="store_false")
    ap.add_argument("--hv-only", type=int, default=0, help="time N launches of the H.v kernel alone")
    ap.add_argument("--hv-workload", default=WORKLOAD, choices=sorted(W.WORKLOADS),
                    help="workload of --hv-only (a batch uses its largest instance)")
    ap.add_argument("--shape", default="", help="cube_bits,group_vectors,tile_cubes[,multipass] for the main run")
    ap.add_argument("--profile-run", default="", help="R,M: one short run of --hv-workload (for profilers)")
    ap.add_argument("--profile-batch", action="store_true", help="one run of a batch workload (for profilers)")
    ap.add_argument("--batch-workload", default="chains_s1_x24", choices=["chains_s1_x24", "mn9_powder"],
                    help="the batch --profile-batch runs")
    ap.add_argument("--profile-sym", action="store_true",
                    help="the symmetric-estimator leg alone: Mn9-like system, one direction (for profilers)")
    ap.add_argument("--autotune", action="store_true",
                    help="time candidate launch shapes first (default: the library's default plan, which "
                         "keeps the command's kernels the same under a profiler)")
    args = ap.parse_args()
    if args.profile_run:
        print(json.dumps(run_profile(args)))
        return
    if args.profile_batch:
        print(json.dumps(run_profile_batch(args)))
        return
    if args.profile_sym:
        import torch

        import paper_2607_25585_gb300 as F

        F.build()
        print(json.dumps(sftlm_leg(F, W.temperatures(), torch.cuda.Stream())))
        return
    if args.hv_only:
        print(json.dumps(run_hv_only(args)), flush=True)
        return
    if args.warmup < 3:
        args.warmup = 3
    line = run_reference(args) if args.impl == "reference" else run_ours(args)
    if line is not None:
        print(json.dumps(line), flush=True)


if __name__ == "__main__":
    main()
