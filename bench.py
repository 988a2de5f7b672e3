"""Benchmark: the batched 1D laser workload of the ECS split-operator method.

Workload: 4096 independent 1D instances, N drawn from {2048, 4096, 8192,
16384}, box [-8N/1024, 8N/1024] (h = 1/64), smooth (SECS) ECS from 75% of
the half-width to theta = 0.5 at the edge, soft-Coulomb a^2 = 2, laser pulse
E0 sin^2 sin with omega = 0.057, 4 cycles, E0 ~ U[0.01, 0.1]; dt = 0.02.
One benchmark step advances every instance by STEPS_PER_CALL time steps in
one library call (one persistent kernel over all instances).

The headline line is complex128 (FP64 arithmetic, the oracle's precision);
complex64 is reported beside it with its error after the whole pulse.

Metric: grid-point-steps per second = sum_j N_j * time steps / seconds.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--prec c128|c64]
  python bench.py --impl reference      # the FP64 CPU oracle on a sample

One JSON line is printed by rank 0."""
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

METRIC = "ECS SO-FFT grid-point-steps/s"
UNIT = "grid-point-steps/s"
N_INST = 4096
STEPS_PER_CALL = 256
W2_DT = 0.02
L2_BYTES = 129 * 1024 * 1024


def _peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        try:
            d = json.load(open(p))
            return d, "measured"
        except Exception:
            pass
    return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0}, "fallback"


def _hbm_peak(d):
    for k in ("hbm_gbs", "hbm_GBps", "hbm"):
        if k in d:
            v = d[k]
            return float(v["value"] if isinstance(v, dict) else v)
    return 6800.0


# DRAM bytes (read + write) of one launch of the dominant kernel, from an
# ncu capture of that launch (dram__bytes_read.sum + dram__bytes_write.sum),
# valid only while the kernel sources hash to the same value and the launch
# has the same instances and steps.
TRAFFIC_MEASURED = {
    "c64": {"src_sha1": "017cc908ca484d84bee6e1e40864622eadd99c5a", "n": 16384, "instances": 988,
            "steps": 256, "bytes": 133621504 + 78311936},
}


def _kernel_src_sha1():
    import hashlib
    h = hashlib.sha1()
    for f in ("soft1d.cuh", "device_common.cuh"):
        with open(os.path.join(ROOT, "paper_1505_06707_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()


def _traffic(prec, n, instances, steps):
    t = TRAFFIC_MEASURED.get(prec)
    if not t or t["src_sha1"] != _kernel_src_sha1():
        return None
    if (t["n"], t["instances"], t["steps"]) != (n, instances, steps):
        return None
    return float(t["bytes"])


# FMA lanes per SM and clock: 128 FP32 lanes; FP64 2 DFMA per clock per SM
# (NVIDIA's dense FP64 figure for GB300, 1.25 TFLOP/s at 152 SMs and
# 2.07 GHz, which the FMA probe of this package reproduces within a few %)
FP32_FMA_PER_SM_CLK = 128
FP64_FMA_PER_SM_CLK = 2


def alu_peaks(torch=None, dev=0):
    """ALU peaks derived from unit counts and the maximum SM clock: SM count
    of the device x FMA lanes x 2 flop x clock (TFLOP/s)."""
    nsm = None
    if torch is not None and torch.cuda.is_available():
        nsm = torch.cuda.get_device_properties(dev).multi_processor_count
    peaks, _ = _peaks()
    mhz = float(peaks.get("sm_max_mhz", 2070.0))
    nsm = nsm or 152
    return {"fp32_tflops": nsm * FP32_FMA_PER_SM_CLK * 2 * mhz * 1e6 / 1e12,
            "fp64_tflops": nsm * FP64_FMA_PER_SM_CLK * 2 * mhz * 1e6 / 1e12,
            "sms": nsm, "sm_max_mhz": mhz,
            "how": "SMs x FMA lanes per SM (FP32 128, FP64 2) x 2 flop x max SM clock"}


def alu_probe(iters=4096):
    """The FMA throughput probe (paper_1505_06707_gb300/probe/alu_peak.cu):
    measured FP32 and FP64 rates, TFLOP/s."""
    import ctypes as C
    lib = C.CDLL(os.path.join(ROOT, "paper_1505_06707_gb300", "_lib", "libaluprobe.so"))
    lib.alu_fma_rate.argtypes = [C.c_int, C.c_int, C.POINTER(C.c_double), C.POINTER(C.c_double)]
    out = {}
    for name, f64, it in (("fp32", 0, iters), ("fp64", 1, iters // 32)):
        fl, ms = C.c_double(), C.c_double()
        rc = lib.alu_fma_rate(f64, it, C.byref(fl), C.byref(ms))
        out[name + "_tflops"] = fl.value / 1e12 if rc == 0 else None
        out[name + "_ms_per_launch"] = ms.value if rc == 0 else None
    return out


def flops_per_call(ns, nbs, steps, field=True):
    """Algorithmic FLOPs of one call: per time step and instance, two FFTs
    (5 N log2 N each), the kinetic and potential phase products (6 N each),
    the field phase (6 N) and the strip Crank-Nicolson (32 per strip row:
    two sweeps, the combination 2x - r and the second potential factor)."""
    tot = 0.0
    for n, nb in zip(ns, nbs):
        tot += 10.0 * n * math.log2(n) + 12.0 * n + (6.0 * n if field else 0.0) + 32.0 * nb
    return tot * steps


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled during the timed region."""

    Q = ("clocks.sm,clocks.max.sm,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, dev=0):
        self.dev, self.rows, self.proc = dev, [], None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.dev), "--query-gpu=" + self.Q,
                 "--format=csv,noheader,nounits", "-lms", "100"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.th = threading.Thread(target=self._read, daemon=True)
            self.th.start()
        except Exception:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.rows.append([c.strip() for c in line.split(",")])

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        sm = [float(r[0]) for r in self.rows if r and r[0].replace(".", "").isdigit()]
        mx = [float(r[1]) for r in self.rows if len(r) > 1 and r[1].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = set()
        for r in self.rows:
            for i, nm in enumerate(names):
                if len(r) > 2 + i and r[2 + i].lower() == "active":
                    reasons.add(nm)
        sm.sort()
        return {"sm_mhz": sm[len(sm) // 2] if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def workload(count=N_INST):
    import workloads as W
    return [W.w2_instance(j) for j in range(count)]


def config(prec="c128", instances=N_INST, spc=STEPS_PER_CALL):
    return {"workload": "1D ECS SO-FFT laser batch: %d instances, N in {2048..16384}, h=1/64, "
                        "smooth (SECS) ECS from R0=0.75 half-width to theta=0.5 at the edge, soft-Coulomb a2=2, "
                        "pulse omega=0.057 4 cycles, dt=0.02" % instances,
            "instances": instances, "time_steps_per_step": spc, "precision": prec,
            "l2": "inputs larger than L2 (packed state %s)" % ("252 MB c64" if prec == "c64" else "504 MB c128")}


def max_over_ranks(ms, world, device="cpu"):
    """The slowest rank's time sets the whole-job rate: the maximum of every
    rank's timed region (an all-reduce on the default process group)."""
    if world <= 1:
        return ms
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(ms)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_value(units_per_rank_step, steps, world, ms):
    """Units all ranks processed (each rank runs its own batch: weak
    scaling) over the slowest rank's time."""
    return units_per_rank_step * steps * world / (ms / 1e3)


def run_reference(args):
    """The FP64 CPU oracle on a bounded, stratified sample of the workload."""
    import numpy as np
    from oracle import propagate as P
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    ws = workload(N_INST)
    sample = []
    for n in (2048, 4096, 8192, 16384):
        sample += [w for w in ws if w["n"] == n][:8]
    nst = 16
    probs = [P.Problem1D(w["n"], w["a"], w["b"], w["R0"], theta=w["theta"], kind=w["contour"],
                         a2=w["a2"], dt=w["dt"]) for w in sample]
    psis = [w["psi0"] for w in sample]
    fields = [(w["E0"], w["omega"], w["ncyc"]) for w in sample]
    for _ in range(max(1, args.warmup)):                 # untimed warm-up steps
        P.step_batch(probs, psis, nst, fields=fields)
    times = []
    for _ in range(max(1, args.steps)):
        t = time.perf_counter()
        P.step_batch(probs, psis, nst, fields=fields)
        times.append(time.perf_counter() - t)
    pts = sum(w["n"] for w in sample) * nst
    v = pts / (sum(times) / len(times))
    cores = P.num_threads()
    desc = ("oracle (FP64 C, literal 4-FFT step, full cyclic CN) on %d instances (8 per size) x %d "
            "time steps per step" % (len(sample), nst))
    out = {"impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": args.gpus,
           "steps": args.steps, "warmup": args.warmup,
           "ms_per_step": 1e3 * sum(times) / len(times), "higher_is_better": True,
           "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
           "config": config(args.prec, args.instances, args.steps_per_call),
           "cpu_baseline": {"value": v, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": desc},
           "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(out))


def cpu_baseline_sample():
    """Oracle timed on a bounded sample (about 10-20 s of CPU work)."""
    from oracle import propagate as P
    ws = workload(N_INST)
    sample = []
    for n in (2048, 4096, 8192, 16384):
        sample += [w for w in ws if w["n"] == n][:4]
    nst = 16
    probs = [P.Problem1D(w["n"], w["a"], w["b"], w["R0"], theta=w["theta"], kind=w["contour"],
                         a2=w["a2"], dt=w["dt"]) for w in sample]
    psis = [w["psi0"] for w in sample]
    fields = [(w["E0"], w["omega"], w["ncyc"]) for w in sample]
    P.step_batch(probs, psis, 1, fields=fields)
    t = time.perf_counter()
    P.step_batch(probs, psis, nst, fields=fields)
    dt = time.perf_counter() - t
    pts = sum(w["n"] for w in sample) * nst
    return {"value": pts / dt, "unit": UNIT, "cores": P.num_threads(), "kind": "oracle",
            "sample": "%d instances (4 per size) x %d time steps, FP64 C oracle, OpenMP over "
                      "instances" % (len(sample), nst)}


def bench_2d(S, torch, dev, args):
    """The 2D workload (2048^2, sharp theta = 0.4): throughput of the step in
    both precisions, and its HBM rate counting the minimum traffic of the pass
    structure: the row pass and the column pass each read and write the state
    and read the potential table once (4 S + 2 table bytes per point-step)."""
    import numpy as np
    import workloads as W
    w = W.w3()
    n = w["nx"]
    res = {}
    peaks, src = _peaks()
    hbm = _hbm_peak(peaks)
    for prec, name, nst, reps in ((S.SOFT_C64, "c64", 64, 3), (S.SOFT_C128, "c128", 8, 2)):
        plan = S.soft_create((n, n), w["box"], w["R0"], w["theta"], w["dt"], prec=prec,
                             soft_a2=w["a2"])
        d = torch.tensor(w["psi0"], dtype=torch.complex64 if prec == S.SOFT_C64 else torch.complex128,
                         device=dev)
        st = torch.cuda.current_stream(dev)
        S.soft_step(plan, d, nst, 0.0, stream=st)        # warm-up (captures the graph)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(st)
        for _ in range(reps):
            S.soft_step(plan, d, nst, 0.0, stream=st)
        e1.record(st)
        torch.cuda.synchronize()
        sec = e0.elapsed_time(e1) / 1e3
        steps = nst * reps
        Sb = 8 if prec == S.SOFT_C64 else 16
        tab = 8 if prec == S.SOFT_C64 else 16             # e^{-iU tau/2} per point (c64: minus 1, float2)
        bytes_pt = 4 * Sb + 2 * tab
        gps = n * n * steps / sec
        res[name] = {"grid_point_steps_per_s": gps, "ms_per_step": 1e3 * sec / steps,
                     "hbm_GBps_alg": gps * bytes_pt / 1e9, "hbm_frac_alg": gps * bytes_pt / 1e9 / hbm,
                     "bytes_per_point_step": bytes_pt, "launches_per_call": S.soft_last_launches(plan)}
        S.soft_destroy(plan)
        del d
    res["workload"] = "2048^2 on [-200,200]^2, sharp ECS R0=150 theta=0.4, U=-1/sqrt(r^2+1), dt=0.02"
    res["hbm_peak_GBps"] = hbm
    res["hbm_peak_source"] = src
    return res


def bench_3d(S, torch, dev, args):
    """The 3D workload (256^3, sharp theta = 0.4) in both precisions, and
    512^3 in complex64: throughput of the step and its HBM rate counting the
    minimum traffic of the pass structure: rows, z lines and y lines each read
    and write the state, the row and z passes read the potential table
    (6 S + 2 table bytes per point-step; the y-strip CN pass, which touches
    the strip block only, is not counted)."""
    import workloads as W
    w = W.w6()
    peaks, src = _peaks()
    hbm = _hbm_peak(peaks)
    res = {}
    for prec, name, n, nst, reps in ((S.SOFT_C64, "c64", 256, 24, 3), (S.SOFT_C128, "c128", 256, 8, 2),
                                     (S.SOFT_C64, "c64_512", 512, 8, 2)):
        box = (-w["box"][1] * n / 256, w["box"][1] * n / 256) * 3   # h fixed at 0.3125
        R0 = w["R0"] * n / 256
        t0 = time.perf_counter()
        plan = S.soft_create((n, n, n), box, R0, w["theta"], w["dt"], prec=prec, soft_a2=w["a2"],
                             contour=w["kind"])
        setup = time.perf_counter() - t0
        psi0 = W.w6_state((n, n, n), box, seed=0)
        d = torch.tensor(psi0, dtype=torch.complex64 if prec == S.SOFT_C64 else torch.complex128,
                         device=dev)
        del psi0
        st = torch.cuda.current_stream(dev)
        S.soft_step(plan, d, nst, 0.0, stream=st)        # warm-up (captures the graph)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(st)
        for _ in range(reps):
            S.soft_step(plan, d, nst, 0.0, stream=st)
        e1.record(st)
        torch.cuda.synchronize()
        sec = e0.elapsed_time(e1) / 1e3
        steps = nst * reps
        Sb = 8 if prec == S.SOFT_C64 else 16
        tab = 8 if prec == S.SOFT_C64 else 16             # e^{-iU tau/2} per point (c64: minus 1, float2)
        bytes_pt = 6 * Sb + 2 * tab
        pts = n ** 3
        gps = pts * steps / sec
        res[name] = {"n": n, "grid_point_steps_per_s": gps, "ms_per_step": 1e3 * sec / steps,
                     "hbm_GBps_alg": gps * bytes_pt / 1e9, "hbm_frac_alg": gps * bytes_pt / 1e9 / hbm,
                     "bytes_per_point_step": bytes_pt, "launches_per_call": S.soft_last_launches(plan),
                     "plan_setup_s": setup, "state_MB": pts * Sb / 1e6}
        S.soft_destroy(plan)
        del d
        torch.cuda.empty_cache()
    res["workload"] = ("256^3 on [-40,40]^3 (h = 0.3125; 512^3 on [-80,80]^3), sharp ECS R0 = 0.75 of the "
                       "half-width, theta=0.4, U=-1/sqrt(r^2+1), dt=0.02")
    res["hbm_peak_GBps"] = hbm
    res["hbm_peak_source"] = src
    return res


def oracle_3d_sample(steps=1):
    """The FP64 C oracle's literal 3D step (four 3D FFTs, full cyclic CN on
    every line) on the 256^3 workload, timed on the host cores."""
    import workloads as W
    from oracle import propagate as P
    w = W.w6()
    p = P.Problem3D(w["n"], w["box"], w["R0"], theta=w["theta"], kind=w["kind"], a2=w["a2"], dt=w["dt"])
    psi0 = W.w6_state(w["n"], w["box"], seed=0)
    t0 = time.perf_counter()
    p.step(psi0, steps)
    sec = time.perf_counter() - t0
    pts = w["n"][0] * w["n"][1] * w["n"][2]
    return {"value": pts * steps / sec, "unit": "grid-point-steps/s", "seconds_per_step": sec / steps,
            "cores": P.num_threads(), "kind": "oracle",
            "sample": "%d step of the 256^3 workload, FP64 C oracle, OpenMP over lines" % steps}


def oracle_2d_sample(steps=3):
    """The FP64 C oracle's literal 2D step (four FFTs, full cyclic CN) on the
    2048^2 workload, timed for a few steps on the host cores."""
    import workloads as W
    from oracle import propagate as P
    w = W.w3()
    p = P.Problem2D(w["nx"], w["ny"], w["box"], w["R0"], theta=w["theta"], a2=w["a2"], dt=w["dt"])
    t0 = time.perf_counter()
    p.step(w["psi0"], steps)
    sec = time.perf_counter() - t0
    return {"value": w["nx"] * w["ny"] * steps / sec, "unit": "grid-point-steps/s", "seconds_per_step": sec / steps,
            "cores": P.num_threads(), "kind": "oracle",
            "sample": "%d steps of the 2048^2 workload, FP64 C oracle, OpenMP over rows/columns" % steps}


def oracle_pcg_sample(mean_iterations, iters=6):
    """The oracle's COCG (numpy FP64, banded preconditioner) on one energy of
    the 1024^2 workload: a few iterations timed, scaled to a solve at the
    given mean iteration count."""
    import workloads as W
    from oracle import propagate as P
    from oracle import stationary as ST
    from oracle import tables as T
    w = W.w4()
    n = w["nx"]
    p2 = P.Problem2D(n, n, w["box"], w["R0"], theta=w["theta"], a2=w["a2"], dt=0.02)
    st = ST.Stationary2D(p2, nbw=10, kind=T.SHARP, R0=w["R0"], theta=w["theta"])
    E = float(w["E"][0])
    t0 = time.perf_counter()
    ST.cocg(lambda v: st.apply_A(v, E), lambda r: st.precond_band(r, E), w["f"], tol=1e-30, maxit=iters)
    per_it = (time.perf_counter() - t0) / iters
    per_solve = per_it * mean_iterations
    return {"value": 1.0 / per_solve, "unit": "solves/s", "seconds_per_iteration": per_it,
            "seconds_per_solve": per_solve, "cores": 1, "kind": "oracle",
            "sample": "%d COCG iterations (banded preconditioner) on one 1024^2 energy, numpy FP64 on one "
                      "core, scaled to %.0f iterations per solve (the GPU FP64 COCG's mean)"
                      % (iters, mean_iterations)}


def bench_pcg(S, torch, dev, args):
    """The stationary workload: 64 energies solved as one batch on 1024^2 with
    the banded ECS preconditioner to relative residual 1e-8."""
    import numpy as np
    import workloads as W
    w = W.w4()
    n = w["nx"]
    plan = S.soft_create((n, n), w["box"], w["R0"], w["theta"], 0.02, prec=S.SOFT_C128,
                         soft_a2=w["a2"])
    f = torch.tensor(w["f"], dtype=torch.complex128, device=dev)
    E = [float(e) for e in w["E"]]
    if args.pcg_energies > 0:
        E = E[:args.pcg_energies]
    out = torch.zeros((len(E), n, n), dtype=torch.complex128, device=dev)
    st = torch.cuda.current_stream(dev)
    # warm-up: builds the tables and the workspace for all energies
    S.sse_pcg_solve(plan, E, f, out, tol=w["tol"], maxit=2, precond=1, stream=st)
    torch.cuda.synchronize()
    res = {}
    names = {1: "band_fp64", 4: "band_fp32", 5: "mixed_fp32_reliable"}
    for pc in (int(v) for v in args.pcg_precond.split(",")):
        name = names[pc]
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(st)
        rc, its, rr = S.sse_pcg_solve(plan, E, f, out, tol=w["tol"], maxit=3000, precond=pc, stream=st)
        e1.record(st)
        torch.cuda.synchronize()
        sec = e0.elapsed_time(e1) / 1e3
        res[name] = {"solves_per_s": len(E) / sec, "seconds": sec, "status": rc,
                     "iterations_mean": float(np.mean(its)), "iterations_max": int(np.max(its)),
                     "max_relres": float(np.max(rr))}
        if pc == 5:
            # minimum HBM traffic of one mixed iteration, per grid point (complex64
            # vectors, double-float increment): A row 16 + column 24, P row 16 +
            # column 16 + row 32 (t, z, r, w), x/r update 64, p update 24
            bpp = 192.0
            gbs = float(np.sum(its)) * n * n * bpp / sec / 1e9
            res[name]["hbm_alg"] = {"GBps": gbs, "frac": gbs / _hbm_peak(_peaks()[0]),
                                    "bytes_per_point_iteration": bpp}
    S.soft_destroy(plan)
    del out
    best = max(res.values(), key=lambda r: r["solves_per_s"] if r["status"] == 0 else 0)
    return {"solves_per_s": best["solves_per_s"], "energies": len(E), **res,
            "precond": "banded ECS (N_BW = 10): FP64 (precond 1), FP32 arithmetic (precond 4), "
                       "FP32 A and preconditioner with FP64 reliable updates (precond 5)",
            "precision": "c128 state, FP64 dots; FP64 A and residual (1, 4); FP32 A inside the "
                         "iteration with the FP64 true residual deciding convergence (5)",
            "workload": "1024^2 on [-200,200]^2, sharp ECS R0=150 theta=0.4, 64 energies in [0.05,2]"}


def bench_accuracy(S, torch, dev, args, sizes=(2048,)):
    """Accuracy of the complex64 path: one laser-batch instance per size
    propagated over the whole pulse (22046 steps of dt = 0.02) in complex64
    and in complex128 on the GPU (complex128 matches the FP64 oracle to
    1e-11 in the tests); rel-L2 of the difference at the end."""
    import numpy as np
    import workloads as W
    out = {}
    for n in sizes:
        w = next(v for v in (W.w2_instance(j) for j in range(256)) if v["n"] == n)
        nst = int(round(w["ncyc"] * 2 * math.pi / w["omega"] / w["dt"]))
        res = {}
        for prec, name, ct in ((S.SOFT_C64, "c64", torch.complex64), (S.SOFT_C128, "c128", torch.complex128)):
            pl = S.soft_create(n, (w["a"], w["b"]), w["R0"], w["theta"], w["dt"], prec=prec,
                               contour=w["contour"], soft_a2=w["a2"])
            d = torch.tensor(w["psi0"], dtype=ct, device=dev)
            S.soft_step(pl, d, nst, 0.0, field=(w["E0"], w["omega"], w["ncyc"]))
            res[name] = d.cpu().numpy().astype(np.complex128)
            S.soft_destroy(pl)
        out[str(n)] = {"steps": nst, "rel_l2_c64_vs_c128":
                       float(np.linalg.norm(res["c64"] - res["c128"]) / np.linalg.norm(res["c128"]))}
    return out


def bench_conv(S, torch, dev, args, plan=None):
    """The learned correction's forward pass alone (three 3x3 convolutions,
    2 -> 32 -> 32 -> 2 channels, BF16 operands on the tensor cores, FP32
    accumulate) on 16 fields of the stationary workload's 1024^2 grid,
    against the BF16 tensor peak."""
    import workloads as W
    w = W.w4()
    n = w["nx"]
    own = plan is None
    if own:
        plan = S.soft_create((n, n), w["box"], w["R0"], w["theta"], 0.02, prec=S.SOFT_C128,
                             soft_a2=w["a2"])
    st = torch.cuda.current_stream(dev)
    nf = 16
    xf = torch.randn((nf, n, n), dtype=torch.complex64, device=dev)
    yf = torch.zeros((nf, n, n, 2), dtype=torch.float32, device=dev)
    for _ in range(3):
        S.sse_nn_forward(plan, xf, yf, stream=st)
    torch.cuda.synchronize()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(5)]
    for a_, b_ in ev:
        a_.record(st)
        S.sse_nn_forward(plan, xf, yf, stream=st)
        b_.record(st)
    torch.cuda.synchronize()
    fms = sum(a_.elapsed_time(b_) for a_, b_ in ev) / len(ev)
    if own:
        S.soft_destroy(plan)
    flops = 2.0 * 9 * (2 * 32 + 32 * 32 + 32 * 2) * nf * n * n
    peaks, psrc = _peaks()
    bf16 = float(peaks.get("bf16_tflops", 1900.0))
    return {"fields": nf, "ms": fms, "tflops": flops / (fms / 1e3) / 1e12,
            "peak_bf16_tflops": bf16, "frac": flops / (fms / 1e3) / 1e12 / bf16,
            "peak_source": psrc, "flop_per_point": flops / (nf * n * n),
            "path": "tcgen05.mma kind::f16 (BF16 in shared memory, FP32 accumulators in TMEM) for the 32-input-channel layers; warp mma.sync m16n8k16 for the 2-input-channel layer"}


CROPS_PER_FIELD = 1024        # learned correction: training crops per harvested field


def bench_learned(S, torch, dev, args):
    """The learned correction on the stationary workload: errors of plain
    banded CG runs at 8 training energies after 2 .. 80 iterations are cut
    into 49,152 random 128^2 crops (1024 per field) and the network is
    trained on the GPU for one pass over them; then 8 held-out energies of the workload
    are solved by COCG with the banded preconditioner (the paper's method),
    by flexible GCR with it, and by flexible GCR with the trained correction.
    Everything runs through the library's own calls."""
    import numpy as np
    import workloads as W
    w = W.w4()
    n = w["nx"]
    gamma = 0.1
    plan = S.soft_create((n, n), w["box"], w["R0"], w["theta"], 0.02, prec=S.SOFT_C128,
                         soft_a2=w["a2"])
    f = torch.tensor(w["f"], dtype=torch.complex128, device=dev)
    rng = np.random.default_rng(15055)
    train_E = [float(e) for e in np.sort(rng.uniform(0.05, 2.0, 8))]
    test_E = [float(e) for e in w["E"][4::8]]
    st = torch.cuda.current_stream(dev)
    t0 = time.perf_counter()
    xs = torch.zeros((len(train_E), n, n), dtype=torch.complex128, device=dev)
    S.sse_pcg_solve(plan, train_E, f, xs, tol=1e-11, maxit=4000, precond=1, stream=st)
    ins, tgs = [], []
    Ax = torch.zeros((n, n), dtype=torch.complex128, device=dev)
    z = torch.zeros_like(Ax)
    for k in (2, 5, 10, 20, 40, 80):
        xk = torch.zeros_like(xs)
        S.sse_pcg_solve(plan, train_E, f, xk, tol=1e-14, maxit=k, precond=1, stream=st)
        for e, E in enumerate(train_E):
            S.sse_apply_A(plan, E, xk[e], Ax, stream=st)
            r = f - Ax
            S.sse_apply_precond(plan, E, 1, r, z, stream=st)
            err = xs[e] - xk[e]
            sc = torch.sqrt(torch.mean(torch.abs(z) ** 2) / 2)
            tgt = gamma * (err * (torch.linalg.norm(z) / torch.linalg.norm(err)) - z) / sc
            zin = z / sc
            # CROPS_PER_FIELD random 128^2 windows, gathered on the device
            yx = torch.as_tensor(rng.integers(0, n - 128, (CROPS_PER_FIELD, 2)), device=dev)
            ar = torch.arange(128, device=dev)
            iy = (yx[:, 0, None, None] + ar[None, :, None]).expand(-1, 128, 128)
            ix = (yx[:, 1, None, None] + ar[None, None, :]).expand(-1, 128, 128)
            ins.append(zin[iy, ix].to(torch.complex64))
            tgs.append(tgt[iy, ix].to(torch.complex64))
    ins = torch.cat(ins).contiguous()
    tgs = torch.cat(tgs).contiguous()
    train_steps = int(ins.shape[0]) // 32                 # one pass over the crops at batch 32
    torch.cuda.synchronize()
    t_harvest = time.perf_counter() - t0
    t0 = time.perf_counter()
    losses = S.sse_nn_train(plan, ins, tgs, steps=train_steps, batch=32, lr=2e-3, seed=7, stream=st)
    torch.cuda.synchronize()
    t_train = time.perf_counter() - t0
    del ins, tgs
    torch.cuda.empty_cache()
    res = {"train_energies": len(train_E), "crops": CROPS_PER_FIELD * 6 * len(train_E), "crop": 128,
           "harvest_s": t_harvest, "train_s": t_train, "train_steps": train_steps,
           "loss_first": float(np.mean(losses[:10])), "loss_last": float(np.mean(losses[-10:])),
           "test_energies": len(test_E), "gamma": gamma}
    res["conv_forward"] = bench_conv(S, torch, dev, args, plan)
    out = torch.zeros((len(test_E), n, n), dtype=torch.complex128, device=dev)
    for name, pc in (("cocg_band", 1), ("fgcr_band", 3), ("fgcr_band_learned", 2)):
        out.zero_()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(st)
        rc, its, rr = S.sse_pcg_solve(plan, test_E, f, out, tol=w["tol"], maxit=2000, precond=pc,
                                      stream=st)
        e1.record(st)
        torch.cuda.synchronize()
        res[name] = {"status": rc, "iterations": [int(i) for i in its],
                     "iterations_mean": float(np.mean(its)), "seconds": e0.elapsed_time(e1) / 1e3,
                     "max_relres": float(np.max(rr))}
    S.soft_destroy(plan)
    return res


def bench_w1(S, torch, dev, args):
    """The single 1D instance (N = 1024 on [-200, 200], sharp ECS R0 = 150,
    theta = 0.5, soft-Coulomb a^2 = 2, dt = 0.05): the whole 2000-step run
    as one soft_step call, in both precisions.  One instance is one CTA on
    one SM with its state in shared memory, so this is the latency of the
    step's dependent passes, not a throughput bound (the batch is the
    throughput form)."""
    import workloads as W
    w = W.w1()
    st = torch.cuda.current_stream(dev)
    res = {}
    for prec, name in ((S.SOFT_C128, "c128"), (S.SOFT_C64, "c64")):
        plan = S.soft_create(w["n"], (w["a"], w["b"]), w["R0"], w["theta"], w["dt"], prec=prec,
                             soft_a2=w["a2"])
        ct = torch.complex64 if prec == S.SOFT_C64 else torch.complex128
        d = torch.tensor(w["psi0"], dtype=ct, device=dev)
        S.soft_step(plan, d, w["nsteps"], 0.0, stream=st)          # warm-up
        torch.cuda.synchronize()
        reps = 3
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(st)
        for _ in range(reps):
            d.copy_(torch.tensor(w["psi0"], dtype=ct))
            S.soft_step(plan, d, w["nsteps"], 0.0, stream=st)
        e1.record(st)
        torch.cuda.synchronize()
        sec = e0.elapsed_time(e1) / 1e3 / reps
        res[name] = {"ms_per_run": 1e3 * sec, "us_per_step": 1e6 * sec / w["nsteps"],
                     "grid_point_steps_per_s": w["n"] * w["nsteps"] / sec,
                     "launches_per_call": S.soft_last_launches(plan)}
        S.soft_destroy(plan)
    res["workload"] = ("N = 1024 on [-200,200], sharp ECS R0 = 150 theta = 0.5, U = -1/sqrt(x^2+2), "
                       "dt = 0.05, 2000 steps in one call (the timed region includes a 16 KB "
                       "host-to-device reset of the state per run)")
    return res


def oracle_w1_sample():
    """The FP64 oracle on the whole single-instance 1D run (2000 steps)."""
    from oracle import propagate as P
    import workloads as W
    w = W.w1()
    prob = P.Problem1D(w["n"], w["a"], w["b"], w["R0"], theta=w["theta"], a2=w["a2"], dt=w["dt"])
    prob.step(w["psi0"], 10)
    t = time.perf_counter()
    prob.step(w["psi0"], w["nsteps"])
    sec = time.perf_counter() - t
    return {"value": w["n"] * w["nsteps"] / sec, "unit": UNIT, "cores": 1, "kind": "oracle",
            "sample": "the whole run: N = 1024 x 2000 steps, FP64 C oracle, one instance on one core"}


def bench_pcg1d(S, torch, dev, args):
    """The paper's own stationary test (Sec. IV, closing remarks) on the GPU:
    N = 1024, b = -a = 51.2, r_s = 40, tau = h^2; the packet propagated to
    t_max = 20 by the GPU step is the right-hand side of 30 solves,
    E = k^2/2 for k = 0.2 .. 6, by COCG with the banded preconditioner
    (N_l = 10) to 1e-12, for the three absorbers of that test."""
    import numpy as np
    g = json.load(open(os.path.join(ROOT, "tests", "golden", "paper_test_setup.json")))
    n, rmax, rs, v0 = g["N"], g["rmax"], g["r_s"], g["v0"]
    Es = [0.5 * (0.2 * k) ** 2 for k in range(1, 31)]
    h = 2 * rmax / n
    tau = h * h
    x = -rmax + h * (np.arange(n) + 0.5)
    psi0 = math.pi ** -0.25 * np.exp(-x ** 2 / 2 + 1j * v0 * x)
    st = torch.cuda.current_stream(dev)
    res = {}
    for name, kind in (("secs", S.CONTOUR_SECS), ("tfecs", S.CONTOUR_TFECS), ("tfap", S.ABSORB_TFAP)):
        plan = S.soft_create(n, (-rmax, rmax), rs, math.pi / 4, tau, prec=S.SOFT_C128, contour=kind,
                             charge=0.0, tfecs_alpha=g["tfecs_alpha"], cap_energy=g["cap_energy"],
                             tfap_kmin=g["tfap_kmin"])
        d = torch.tensor(psi0, dtype=torch.complex128, device=dev)
        S.soft_step(plan, d, int(round(g["t_max"] / tau)), 0.0, stream=st)
        out = torch.zeros((len(Es), n), dtype=torch.complex128, device=dev)
        S.sse_pcg_solve(plan, Es, d, out, tol=g["pcg_tolerance"], maxit=2000, precond=1, stream=st)   # warm-up
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(st)
        rc, its, rr = S.sse_pcg_solve(plan, Es, d, out, tol=g["pcg_tolerance"], maxit=2000, precond=1, stream=st)
        e1.record(st)
        torch.cuda.synchronize()
        sec = e0.elapsed_time(e1) / 1e3
        res[name] = {"status": rc, "iterations_mean": float(np.mean(its)), "iterations_max": int(max(its)),
                     "seconds": sec, "solves_per_s": len(Es) / sec, "max_relres": float(max(rr)),
                     "paper_iterations": g["claims"]["pcg_iterations_" + name]}
        if name != "tfap":
            # the whole t&E-SURFF extraction: sampled propagation to t_max,
            # the 30 solves, the amplitudes (Filon-Simpson); error against
            # Eq. Ateor for 1 <= |k| <= 6
            nst = int(round(g["t_max"] / tau))
            samp = torch.zeros((nst + 1, 4), dtype=torch.complex128, device=dev)
            d2 = torch.tensor(psi0, dtype=torch.complex128, device=dev)
            a_, b_ = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a_.record(st)
            S.soft_step_surface(plan, d2, nst, 0.0, samp, stream=st)
            S.sse_pcg_solve(plan, Es, d2, out, tol=g["pcg_tolerance"], maxit=2000, precond=1, stream=st)
            amp = S.sse_surff(plan, Es, out, samp, t0=0.0, rule=1, stream=st)
            b_.record(st)
            torch.cuda.synchronize()
            ks = np.array([math.sqrt(2 * E) for E in Es])
            a_np = amp.cpu().numpy()
            sel = ks >= 1.0 - 1e-9
            ate = lambda k: math.pi ** -0.25 * np.exp(-(k - v0) ** 2 / 2)
            err = max(np.abs(a_np[sel, 0] - ate(ks[sel])).max(), np.abs(a_np[sel, 1] - ate(-ks[sel])).max())
            res[name]["tE_SURFF"] = {"seconds": a_.elapsed_time(b_) / 1e3, "steps": nst, "amplitudes": 2 * len(Es),
                                     "max_error_vs_Ateor_1_le_absk_le_6": float(err)}
        S.soft_destroy(plan)
    res["setup"] = ("N = 1024, [-51.2, 51.2], r_s = 40, 30 energies k = 0.2 .. 6, banded preconditioner "
                    "N_l = 10, tolerance 1e-12, one launch for all energies (one CTA per energy)")
    return res


def measure_w2(S, torch, dev, args, prec_name, steps, warmup, world=1, with_e2e=True, persistent=1, autotune=1):
    """The laser batch through one batch plan: the persistent kernel over all
    4096 instances (one graph per call: pulse table, queue reset, the
    kernel, time advance).  Device-timed region of `steps` calls, the graph
    call timed alone for the roofline, and the end-to-end rate with host
    copies of the whole packed state every call."""
    import numpy as np
    prec = S.SOFT_C64 if prec_name == "c64" else S.SOFT_C128
    cdt_np = np.complex64 if prec == S.SOFT_C64 else np.complex128
    spc = args.steps_per_call
    ws = workload(args.instances)
    plan = S.soft_create_batch([w["n"] for w in ws], [(w["a"], w["b"]) for w in ws],
                               [w["R0"] for w in ws], [w["theta"] for w in ws],
                               [(w["E0"], w["omega"], w["ncyc"]) for w in ws], W2_DT,
                               prec=prec, contour=ws[0]["contour"], persistent=persistent, autotune=autotune)
    offs, total = S.soft_batch_layout(plan)
    h0 = np.concatenate([w["psi0"] for w in ws]).astype(cdt_np)
    state = torch.from_numpy(h0).to(dev)
    stream = torch.cuda.current_stream(dev)
    ns = [w["n"] for w in ws]
    pts_call = float(sum(ns)) * spc
    nbs = [n // 4 + 2 for n in ns]           # strip block: 2 x N/8 strip rows + 2 coupled neighbours
    flops_call = flops_per_call(ns, nbs, spc)
    t = 0.0
    for _ in range(warmup):
        t = S.soft_step_batch(plan, state, spc, t, stream=stream)
    torch.cuda.synchronize()
    launches = S.soft_last_launches(plan)
    if world > 1:
        import torch.distributed as dist
        dist.barrier()
    torch.cuda.synchronize()
    clk = ClockSampler(dev.index or 0)
    clk.start()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for k in range(steps):
        ev[k][0].record(stream)
        t = S.soft_step_batch(plan, state, spc, t, stream=stream)
        ev[k][1].record(stream)
    e1.record(stream)
    torch.cuda.synchronize()
    clocks = clk.stop()
    ms = max_over_ranks(e0.elapsed_time(e1), world, dev)
    kms = sum(a.elapsed_time(b) for a, b in ev) / steps
    # the plan's schedule (the autotuner keeps the faster): 3 launches per
    # call with the persistent kernel (pulse table, kernel, time advance),
    # 2 + one per size group otherwise
    nsizes = len(set(ns))
    sched = ("soft1d_persist_kernel" if launches == 3 and nsizes > 1 else
             "soft1d_kernel x %d size groups" % nsizes)
    out = {"value": whole_job_value(pts_call, steps, world, ms), "ms_per_step": ms / steps,
           "call_ms": kms, "flops_per_call": flops_call, "gpu_launches": int(launches * steps),
           "clocks": clocks, "points": int(total), "instances": len(ws), "schedule": sched,
           "steps_per_call": spc}
    if sched.startswith("soft1d_kernel"):
        # the dominant kernel (the largest N's group) timed alone, one launch
        # per call, events on the launching stream
        nmax = max(ns)
        wd = [w for w in ws if w["n"] == nmax]
        pd = S.soft_create_batch([w["n"] for w in wd], [(w["a"], w["b"]) for w in wd],
                                 [w["R0"] for w in wd], [w["theta"] for w in wd],
                                 [(w["E0"], w["omega"], w["ncyc"]) for w in wd], W2_DT,
                                 prec=prec, contour=wd[0]["contour"], persistent=0, autotune=0)
        sd = torch.from_numpy(np.concatenate([w["psi0"] for w in wd]).astype(cdt_np)).to(dev)
        td = S.soft_step_batch(pd, sd, spc, 0.0, stream=stream)
        kd = max(2, min(steps, 5 if prec == S.SOFT_C128 else steps))
        evd = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(kd)]
        for a_, b_ in evd:
            a_.record(stream)
            td = S.soft_step_batch(pd, sd, spc, td, stream=stream)
            b_.record(stream)
        torch.cuda.synchronize()
        out["dominant"] = {"kernel": "soft1d_kernel, N = %d group alone (%d instances, %d steps per launch)"
                                     % (nmax, len(wd), spc),
                           "ms": sum(a_.elapsed_time(b_) for a_, b_ in evd) / kd,
                           "flops": flops_per_call([nmax] * len(wd), [nmax // 4 + 2] * len(wd), spc),
                           "instances": len(wd), "n": nmax}
        S.soft_destroy(pd)
        del sd
    if with_e2e:
        hb = torch.from_numpy(h0).pin_memory()
        ob = torch.empty_like(hb).pin_memory()

        def e2e_call(tt):
            state.copy_(hb, non_blocking=True)
            tt = S.soft_step_batch(plan, state, spc, tt, stream=stream)
            ob.copy_(state, non_blocking=True)
            return tt
        t = e2e_call(t)
        torch.cuda.synchronize()
        ke = max(3, steps // 2)
        a_, b_ = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a_.record(stream)
        for _ in range(ke):
            t = e2e_call(t)
        b_.record(stream)
        torch.cuda.synchronize()
        out["e2e"] = {"value": pts_call * ke * world / (a_.elapsed_time(b_) / 1e3), "unit": UNIT,
                      "h2d_bytes_per_step": int(h0.nbytes), "d2h_bytes_per_step": int(h0.nbytes)}
    S.soft_destroy(plan)
    del state
    return out


# DRAM bytes (read + write) per launch of the complex128 N = 16384 group
# kernel, from an ncu capture of 69 instances x 16 steps (29.30 MB) scaled by
# the instance count: each instance's 256 KB state is read and written back
# once per launch and stays in L2 between steps (the tables are shared).
# Valid while the kernel sources hash to src_sha1.
TRAFFIC_C128 = {"src_sha1": "a55f0e092028fe20c4774a2cfdc64a50d55e9298",
                "per_instance": (25108992 + 4186368) / 69}


def roofline_w2(torch, dev, m, prec_name):
    """The dominant kernel against the ALU peak of its precision:
    algorithmic FLOPs per launch over its launch duration.  With one kernel
    per size group that is the largest N's group timed alone; with the
    persistent kernel, the whole call (one launch)."""
    ap_ = alu_peaks(torch, dev.index or 0)
    c64 = prec_name == "c64"
    peak = ap_["fp32_tflops"] if c64 else ap_["fp64_tflops"]
    dom = m.get("dominant")
    if dom:
        achieved = dom["flops"] / (dom["ms"] / 1e3) / 1e12
        kern = "%s, %.3f ms per launch" % (dom["kernel"], dom["ms"])
        traffic = None
        if not c64 and dom["n"] == 16384 and TRAFFIC_C128["src_sha1"] == _kernel_src_sha1():
            traffic = TRAFFIC_C128["per_instance"] * dom["instances"]
    else:
        achieved = m["flops_per_call"] / (m["call_ms"] / 1e3) / 1e12
        kern = ("%s, all %d instances, %d steps per call, %.3f ms per call (graph: pulse table, queue reset, "
                "the persistent kernel, time advance)" % (m["schedule"], m["instances"], m["steps_per_call"],
                                                          m["call_ms"]))
        traffic = None
    whole = m["flops_per_call"] / (m["call_ms"] / 1e3) / 1e12
    return {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "TFLOP/s", "frac": achieved / peak,
            "traffic": traffic,
            "traffic_note": "DRAM read + write per launch, ncu capture scaled by instances" if traffic else None,
            "kernel": kern,
            "whole_call": {"achieved": whole, "frac": whole / peak,
                           "schedule": m["schedule"], "ms_per_call": m["call_ms"]},
            "peak_source": "derived: %d SMs x %d %s FMA per clock x 2 x %.0f MHz" % (
                ap_["sms"], FP32_FMA_PER_SM_CLK if c64 else FP64_FMA_PER_SM_CLK, "FP32" if c64 else "FP64",
                ap_["sm_max_mhz"]),
            "flop_count": "per time step and instance 10 N log2 N (two FFTs) + 12 N (phase products) + "
                          "6 N (field) + 32 per strip row"}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="native", choices=["native", "reference"])
    ap.add_argument("--prec", default="c128", choices=["c64", "c128"],
                    help="precision of the headline line (the other is reported beside it)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--instances", type=int, default=N_INST,
                    help="fewer instances for profiling captures (not a bench line)")
    ap.add_argument("--steps-per-call", type=int, default=STEPS_PER_CALL)
    ap.add_argument("--no-extra", action="store_true",
                    help="skip the other precision, the 2D step and the stationary-solver measurements")
    ap.add_argument("--only", choices=["2d", "3d", "pcg", "learned", "conv", "accuracy", "peaks", "w2",
                                       "pcg1d", "w1"],
                    default=None,
                    help="run one measurement alone (for profiling captures; not a bench line)")
    ap.add_argument("--persistent", type=int, default=1, choices=[0, 1],
                    help="0: one kernel per size group instead of the persistent kernel (comparison)")
    ap.add_argument("--autotune", type=int, default=1, choices=[0, 1],
                    help="0: no timing runs at plan creation (profiling captures)")
    ap.add_argument("--pcg-precond", default="1,4,5",
                    help="stationary-solver modes to time (sse_pcg_solve precond values)")
    ap.add_argument("--pcg-energies", type=int, default=0,
                    help="solve only the first K energies of the stationary workload (profiling captures)")
    args = ap.parse_args()
    if args.impl == "reference":
        return run_reference(args)
    if args.only:
        import torch
        import paper_1505_06707_gb300 as S
        dev = torch.device("cuda", 0)
        torch.cuda.set_device(dev)
        if args.only == "accuracy":
            r = bench_accuracy(S, torch, dev, args, sizes=(2048, 4096, 8192, 16384))
        elif args.only == "peaks":
            r = {"derived": alu_peaks(torch, 0), "probe": alu_probe()}
        elif args.only == "w2":
            r = measure_w2(S, torch, dev, args, args.prec, args.steps, args.warmup, with_e2e=False,
                           persistent=args.persistent, autotune=args.autotune)
            r["roofline"] = roofline_w2(torch, dev, r, args.prec)
        else:
            fn = {"2d": bench_2d, "3d": bench_3d, "pcg": bench_pcg, "learned": bench_learned,
                  "conv": bench_conv, "pcg1d": bench_pcg1d, "w1": bench_w1}[args.only]
            r = fn(S, torch, dev, args)
        print(json.dumps({"only": args.only, "result": r}))
        return

    import torch
    import torch.distributed as dist

    import paper_1505_06707_gb300 as S

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)

    # weak scaling: every rank runs its own 4096-instance batch (independent problems)
    m = measure_w2(S, torch, dev, args, args.prec, args.steps, args.warmup, world, persistent=args.persistent)
    peaks, src = _peaks()
    hbm = _hbm_peak(peaks)
    dname = {"c64": "c64 (f32)", "c128": "c128 (f64)"}
    out = {"metric": METRIC, "value": m["value"], "unit": UNIT, "n_gpus": world, "steps": args.steps,
           "warmup": args.warmup, "ms_per_step": m["ms_per_step"], "higher_is_better": True,
           "scaling": "weak", "vs_baseline": None, "dtype": dname[args.prec], "data": "synthetic",
           "config": config(args.prec, args.instances, args.steps_per_call)}
    out["roofline"] = roofline_w2(torch, dev, m, args.prec)
    bytes_pt = 16 if args.prec == "c64" else 32
    out["hbm_effective"] = {"GBps": m["value"] / world * bytes_pt / 1e9, "peak": hbm,
                            "frac": m["value"] / world * bytes_pt / 1e9 / hbm,
                            "peak_source": src, "note": "state stays in shared memory for a whole "
                            "call; this is the rate a one-pass-per-step design would need"}
    out["e2e"] = m["e2e"]
    out["gpu_launches"] = m["gpu_launches"]
    out["clocks"] = m["clocks"]
    if not args.no_extra:
        other = "c64" if args.prec == "c128" else "c128"
        o_steps = args.steps if other == "c64" else min(args.steps, 5)
        mo = measure_w2(S, torch, dev, args, other, o_steps, min(args.warmup, 3), world)
        mo["roofline"] = roofline_w2(torch, dev, mo, other)
        mo["dtype"] = dname[other]
        if other == "c64":
            g = measure_w2(S, torch, dev, args, "c64", o_steps, 2, world, with_e2e=False, persistent=0)
            mo["group_kernels_ms_per_step"] = g["ms_per_step"]
        out[other] = mo
        out["fp32_accuracy"] = bench_accuracy(S, torch, dev, args, sizes=(2048, 4096, 8192, 16384))
        out["w1_1d"] = bench_w1(S, torch, dev, args)
        out["pcg1d_paper_test"] = bench_pcg1d(S, torch, dev, args)
        out["w3_2d"] = bench_2d(S, torch, dev, args)
        out["w6_3d"] = bench_3d(S, torch, dev, args)
        out["w4_pcg"] = bench_pcg(S, torch, dev, args)
        out["w5_learned"] = bench_learned(S, torch, dev, args)
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        out["cpu_baseline"] = cpu_baseline_sample()
        if not args.no_extra:
            out["w1_1d"]["cpu_baseline"] = oracle_w1_sample()
            out["w3_2d"]["cpu_baseline"] = oracle_2d_sample()
            out["w6_3d"]["cpu_baseline"] = oracle_3d_sample()
            pc = out["w4_pcg"]
            its = (pc.get("band_fp64") or pc.get("mixed_fp32_reliable") or {}).get("iterations_mean", 378.0)
            out["w4_pcg"]["cpu_baseline"] = oracle_pcg_sample(its)
    if rank == 0:
        print(json.dumps(out))
    if world > 1:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
