"""Benchmark of the ADG hot path on GB300: DOF-stage updates per second.

One step = one SSP-RK3 time step (three stages of: Gauss-point thermo, chemistry
and flux, face fluxes with AT fluxes at delayed PE faces, Eq. (5) assembly and
stage update, troubled-cell indicator and (AT-)WENO limiter, history-ring writes)
over the whole synthetic workload. A DOF is the paper's vector DOF w_j^e
(Sec. 3.1), so one step updates n_elem * (p+1) * 3 DOF-stages.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--workload NAME]
    python bench.py --impl reference ...   # the FP64 CPU oracle, bounded sample

Prints one JSON line (rank 0). Under torchrun (N > 1) every rank advances its own
independent replica of the workload (weak scaling, no data-path collective); the
timing is the maximum over ranks.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

from paper_2501_01747_gb300 import inputs as I  # noqa: E402

DEFAULT_WORKLOAD = "ignition-9sp-4096x4"
METRIC = "DOF-stage updates/s (mixed vs FP64, same GB300) at stated error; % HBM roofline"
L2_BYTES = 129 * 1024 * 1024

# FP64 peak of GB300 from its unit counts and clock: 152 SMs x 2 FP64 FMA
# (4 flop) per clock per SM x 2.07 GHz = 1.259 TFLOP/s (a microbenchmark of
# independent FMA chains measured 1.19 TFLOP/s at 1.99 GHz on this machine).
FP64_PEAK_TFLOPS = 152 * 4 * 2.07e9 / 1e12
# FP64 elementary functions counted by the FP64-pipe time they take on this GPU:
# a double exp runs at 29.5 G/s, i.e. the time of 40 flops at the FMA peak.
FLOP_EXP = 40.0
FLOP_LOG = 40.0


def stage_kernel_flops(wl, mech, mixed=False):
    """Algorithmic flops of one stage-kernel launch, counted on the minimal
    formulation of the method (FMA = 2, add/mul/div/sqrt = 1, exp/log = 40):
    per Gauss point: modal->nodal 2 nv Q; thermo 10 ns + 12; ln T and 1/T 41;
    per species concentration and g_i/(R T) 6; per reaction ln k_f 4, the Gibbs
    sum 1 + 2 per species with nonzero net nu, k_f and k_r one exp each (80),
    the mass-action products (sum of the coefficients), q 1, the accumulation 2
    per net species; flux nv + 4. Per element: one face flux (2 thermo + 6 nv),
    volume and source quadrature 7 nv Q^2, assembly 8 nv Q and the SSP-RK3
    update 4 nv Q. Returns (FP64 flops, FP32 flops): in the mixed variant the
    point flux, the face flux, the quadratures and the assembly are FP32."""
    ns, nr = mech.ns, mech.nr
    nv, Q = ns + 2, wl.p + 1
    pt64 = 2 * nv * Q + (10 * ns + 12) + (FLOP_LOG + 1) + 6 * ns
    for j in range(nr):
        nx = int(np.count_nonzero(mech.nu_r[j].astype(int) - mech.nu_f[j].astype(int)))
        prods = int(mech.nu_f[j].sum() + mech.nu_r[j].sum())
        pt64 += 4 + (1 + 2 * nx) + 2 * FLOP_EXP + prods + 1 + 2 * nx
    pt_dg = nv + 4
    el_dg = 2 * (10 * ns + 12) + 6 * nv + 7 * nv * Q * Q + 8 * nv * Q
    el64 = 4 * nv * Q
    if mixed:
        return wl.n_elem * (Q * pt64 + el64), wl.n_elem * (Q * pt_dg + el_dg)
    return wl.n_elem * (Q * (pt64 + pt_dg) + el_dg + el64), 0.0


def stage_kernel_bytes(wl, mech):
    """Algorithmic DRAM bytes of one stage launch: read w^n and w^(s), write
    w^(s+1), FP64, n_vars per vector DOF (24 n_vars bytes per DOF)."""
    return 24.0 * (mech.ns + 2) * wl.n_elem * (wl.p + 1)


def load_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        with open(path) as f:
            return json.load(f), "measured"
    return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0}, "fallback"


class ClockSampler:
    """nvidia-smi samples of SM clock and throttle reasons during the timed region."""

    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.FIELDS,
                 "--format=csv,noheader,nounits", "-lms", "100"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except OSError:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.t.join(timeout=2)
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 8:
                continue
            try:
                sm.append(float(parts[0]))
                mx.append(float(parts[1]))
            except ValueError:
                continue
            for nm, val in zip(names, parts[4:8]):
                if val.lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(mx) if mx else None, "reasons": sorted(reasons),
                "samples": len(sm)}


def dist_setup():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def cpu_baseline(wl, mech, budget_s=12.0, max_steps=40):
    """The FP64 oracle (single-threaded C) on this host: the workload's first steps,
    as many as fit in about budget_s seconds."""
    import oracle as O
    o = O.Oracle(wl, mech)
    o.set_primitive(wl.primitive(mech))
    t0 = time.perf_counter()
    n = 0
    while n < max_steps:
        o.step(1)
        n += 1
        if time.perf_counter() - t0 > budget_s:
            break
    dt = time.perf_counter() - t0
    dofs = wl.n_elem * (wl.p + 1) * 3 * n
    return {"value": dofs / dt, "unit": "DOF-stage/s", "cores": 1, "kind": "oracle",
            "sample": "%s, first %d steps (%.1f s, 1 thread)" % (wl.name, n, dt)}


def run_reference(args, ws, rank):
    if rank != 0:
        return 0
    wl = I.load_workloads()[args.workload]
    mech = wl.mechanism()
    cb = cpu_baseline(wl, mech, budget_s=max(5.0, 60.0 / max(1, args.steps + args.warmup)),
                      max_steps=max(1, args.steps))
    line = {"impl": "reference", "metric": METRIC, "value": cb["value"], "unit": cb["unit"],
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1e3 * wl.n_elem * (wl.p + 1) * 3 / cb["value"],
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": workload_config(wl, mech, args),
            "cpu_baseline": cb,
            "e2e": {"value": cb["value"], "unit": cb["unit"], "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line))
    return 0


def workload_config(wl, mech, args):
    return {"workload": wl.name, "n_elem": wl.n_elem, "p": wl.p, "n_species": mech.ns,
            "n_reactions": mech.nr, "n_pe": wl.n_pe, "max_delay": wl.max_delay,
            "at_order": wl.at_order, "delay_mode": ["sync", "caa", "saa"][wl.delay_mode],
            "flux": ["lf", "hllc"][wl.flux], "limiter": ["none", "weno"][wl.limiter],
            "dt": wl.dt, "precision": args.precision,
            "l2": "flushed between timed steps (256 MiB write)", "launch": "CUDA graph per step",
            "parallelism": "replicas" if args.gpus > 1 else "single"}


def mass_fractions(w, p):
    x, _ = np.polynomial.legendre.leggauss(p + 1)
    V = np.polynomial.legendre.legvander(x, p)
    r = np.einsum("inj,qj->inq", w[2:], V)
    return r / r.sum(axis=0, keepdims=True)


def measure(adg, torch, wl, mech, prim, prec, args, dev, pg, ws):
    """Warm-up, autotune, K device-timed steps and the end-to-end run of one
    precision variant on its own context."""
    g = adg.ADG(mech, [wl], device=dev, precision=prec)
    g.set_primitive(prim)
    stream = torch.cuda.current_stream(dev)
    flush = torch.empty(2 * L2_BYTES // 4, dtype=torch.float32, device=dev)

    g.step(args.warmup, stream)
    g.check()
    torch.cuda.synchronize(dev)
    if args.tuning:
        te, nt = (int(x) for x in args.tuning.split(","))
        tuning = g.set_tuning(0, te, nt)
    else:
        tuning = g.autotune(stream) if not args.no_autotune else g.tuning()
    torch.cuda.synchronize(dev)

    # device-resident timing: every step is one replay of the step's CUDA graph
    # (with an event pair around every kernel and around the whole step), timed
    # alone, with the L2 flushed between steps
    sampler = ClockSampler(dev.index or 0)
    if pg:
        pg.barrier()
    torch.cuda.synchronize(dev)
    sampler.start()
    time.sleep(0.3)
    g.enable_kernel_timing(True)
    wall0 = time.perf_counter()
    for k in range(args.steps):
        flush.zero_()
        g.step(1, stream)
    torch.cuda.synchronize(dev)
    wall = time.perf_counter() - wall0
    kms, kn = g.kernel_times()
    g.enable_kernel_timing(False)
    clocks = sampler.stop()
    g.check()
    ms = float(kms[2])
    if pg:
        t = torch.tensor([ms], dtype=torch.float64, device=dev)
        pg.all_reduce(t, op=pg.ReduceOp.MAX)
        ms = float(t.item())
    dof_stage = wl.n_elem * (wl.p + 1) * 3
    value = dof_stage * args.steps * ws / (ms / 1e3)

    # end to end through the C ABI with host buffers: H2D state, step, D2H state
    nbytes = g.nv * wl.n_elem * (wl.p + 1) * 8
    host_in = torch.empty(nbytes // 8, dtype=torch.float64, pin_memory=True)
    host_out = torch.empty(nbytes // 8, dtype=torch.float64, pin_memory=True)
    g.read_state(host_in.numpy(), stream=stream)
    torch.cuda.synchronize(dev)
    n_e2e = max(10, args.steps // 3)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    t0 = time.perf_counter()
    e0.record(stream)
    for k in range(n_e2e):
        g.write_state(host_in.numpy(), stream=stream)
        g.step(1, stream)
        g.read_state(host_out.numpy(), stream=stream)
        stream.synchronize()
    e1.record(stream)
    torch.cuda.synchronize(dev)
    e2e_ms = max(e0.elapsed_time(e1), (time.perf_counter() - t0) * 1e3)
    g.check()
    e2e_value = dof_stage * n_e2e * ws / (e2e_ms / 1e3)
    g.close()
    del flush
    return {"value": value, "ms": ms, "kms": kms, "kn": kn, "tuning": tuning,
            "clocks": clocks, "wall": wall, "nbytes": nbytes,
            "e2e": {"value": e2e_value, "unit": "DOF-stage/s", "h2d_bytes_per_step": nbytes,
                    "d2h_bytes_per_step": nbytes}}


def mixed_error(adg, torch, wl, mech, prim, dev, n_steps):
    """Error of the mixed path against the FP64 path (which matches the FP64
    oracle to 1e-10) after n_steps from the same state: the largest relative
    error of T at the Gauss points, and the error of every mass fraction at the
    Gauss points where it is above 1e-8, relative to the largest value of that
    species (relative L-infinity) and, for information, to the local value."""
    out = {}
    for prec in ("fp64", "mixed"):
        g = adg.ADG(mech, [wl], device=dev, precision=prec)
        g.set_primitive(prim)
        g.step(n_steps)
        g.check()
        out[prec] = (g.temperature(), mass_fractions(g.get_state(), wl.p))
        g.close()
    (T0, Y0), (T1, Y1) = out["fp64"], out["mixed"]
    eY, eP = 0.0, 0.0
    for i in range(Y0.shape[0]):
        big = Y0[i] > 1e-8
        if big.any():
            d = np.abs(Y1[i] - Y0[i])[big]
            eY = max(eY, float(d.max() / Y0[i].max()))
            eP = max(eP, float((d / Y0[i][big]).max()))
    return {"steps": n_steps, "reference": "FP64 GPU path (<= 1e-10 from the FP64 oracle)",
            "T_rel_max": float((np.abs(T1 - T0) / T0).max()),
            "Y_rel_linf": eY, "Y_rel_pointwise": eP,
            "bar": "1e-4: T at every Gauss point; Y_i relative to max Y_i where Y_i > 1e-8"}


def roofline(wl, mech, r, mixed, peaks, src):
    stage_ms = r["kms"][0] / max(1, r["kn"][0])
    f64, f32 = stage_kernel_flops(wl, mech, mixed)
    achieved = f64 / (stage_ms / 1e3) / 1e12
    hbm = stage_kernel_bytes(wl, mech) / (stage_ms / 1e3) / 1e9
    traffic = STAGE_TRAFFIC.get((wl.name, KERNEL_REV, "mixed" if mixed else "fp64"))
    return {"bound": "alu", "achieved": achieved, "peak": FP64_PEAK_TFLOPS,
            "unit": "TFLOP/s", "frac": achieved / FP64_PEAK_TFLOPS, "traffic": traffic,
            "kernel": "stage_kernel<%d,%s>" % (wl.p + 1, "mixed" if mixed else "fp64"),
            "kernel_ms": stage_ms, "fp32_tflops": f32 / (stage_ms / 1e3) / 1e12,
            "kernel_share": r["kms"][0] / max(1e-9, r["kms"][0] + r["kms"][1]),
            "peak_source": "FP64 pipe: 152 SM x 4 flop/clk x 2.07 GHz (derived)",
            "hbm_achieved_gbs": hbm, "hbm_peak_gbs": peaks.get("hbm_gbs"),
            "hbm_frac": hbm / peaks.get("hbm_gbs", 6800.0),
            "hbm_peak_source": src}


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=300)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--workload", default=DEFAULT_WORKLOAD)
    ap.add_argument("--precision", default="mixed", choices=["mixed", "fp64"],
                    help="the headline variant; the other one is timed beside it")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-autotune", action="store_true")
    ap.add_argument("--tuning", default="", help="TE,NT: set the stage launch configuration "
                    "instead of autotuning it")
    ap.add_argument("--only", action="store_true", help="time the headline variant only")
    args = ap.parse_args(argv)
    args.warmup = max(args.warmup, 3)
    ws, rank, local = dist_setup()
    if args.impl == "reference":
        return run_reference(args, ws, rank)

    import torch
    from paper_2501_01747_gb300 import adg

    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    pg = None
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=dev)
        pg = dist
    wl = I.load_workloads()[args.workload]
    mech = wl.mechanism()
    prim = wl.primitive(mech)
    head = measure(adg, torch, wl, mech, prim, args.precision, args, dev, pg, ws)
    other_prec = "fp64" if args.precision == "mixed" else "mixed"
    other = None if args.only else measure(adg, torch, wl, mech, prim, other_prec, args, dev,
                                           pg, ws)
    err = mixed_error(adg, torch, wl, mech, prim, dev, 200) if not args.only else None

    if rank != 0:
        return 0
    peaks, src = load_peaks()
    mixed = args.precision == "mixed"
    line = {
        "metric": METRIC, "value": head["value"], "unit": "DOF-stage/s", "n_gpus": ws,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": head["ms"] / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f32+f64" if mixed else "f64",
        "data": "synthetic", "config": dict(workload_config(wl, mech, args),
                                            tuning=head["tuning"]),
        "roofline": roofline(wl, mech, head, mixed, peaks, src),
        "clocks": head["clocks"],
        "e2e": head["e2e"],
        "gpu_launches": int(head["kn"][0] + head["kn"][1] + head["kn"][2]),
        "wall_s": head["wall"],
    }
    if other is not None:
        line[other_prec] = {
            "value": other["value"], "ms_per_step": other["ms"] / args.steps,
            "e2e": other["e2e"], "roofline": roofline(wl, mech, other, not mixed, peaks, src),
            "clocks": other["clocks"], "tuning": other["tuning"]}
        fp64_v = other["value"] if mixed else head["value"]
        mix_v = head["value"] if mixed else other["value"]
        line["speedup_mixed_vs_fp64"] = mix_v / fp64_v
    if err is not None:
        line["mixed_error"] = err
    if not args.no_cpu_baseline and ws == 1:
        line["cpu_baseline"] = cpu_baseline(wl, mech)
    print(json.dumps(line))
    return 0


# DRAM bytes (read + write) per stage-kernel launch from ncu, per (workload,
# kernel revision, precision); the summaries are under profiles/.
STAGE_TRAFFIC = {}

KERNEL_REV = "v8"

if __name__ == "__main__":
    sys.exit(main())
