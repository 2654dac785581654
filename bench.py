"""Benchmark of the ADG hot path on GB300: DOF-stage updates per second.

One step = one SSP-RK3 time step (three stages of: Gauss-point thermo, chemistry
and flux, face fluxes with AT fluxes at delayed PE faces, Eq. (5) assembly and
stage update, troubled-cell indicator and (AT-)WENO limiter, history-ring writes)
over the whole synthetic workload. A DOF is the paper's vector DOF w_j^e
(Sec. 3.1), so one step updates n_elem * (p+1) * 3 DOF-stages.

The headline workload is the batched ensemble of 512 independent ignition
instances (8.58 M Gauss points, the largest single-GPU configuration), in the
mixed variant (FP32 flux, DG operator and limiter; FP64 temperature and
chemistry), with the FP64 and the float-chemistry variants timed beside it. The
9-species ignition (4096 x p4) and the 53-species detonation (65536 x p3) are
measured as sub-records.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--workload NAME]
    python bench.py --impl reference ...   # the FP64 CPU oracle, bounded sample

Prints one JSON line (rank 0). Under torchrun (N > 1) the ensemble's instances
are sharded over the ranks (a single-instance workload runs as one replica per
rank); no data moves between ranks, and the timing is the maximum over ranks.
"""
from __future__ import annotations

import argparse
import dataclasses
import json
import os
import statistics
import subprocess
import sys
import threading
import time
from concurrent.futures import ThreadPoolExecutor

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

from paper_2501_01747_gb300 import inputs as I  # noqa: E402
from paper_2501_01747_gb300 import shard as SH  # noqa: E402

ENSEMBLE = "ensemble-9sp-512"
IGNITION = "ignition-9sp-4096x4"
LARGE = "detonation-53sp-65536x3"
DEFAULT_WORKLOAD = ENSEMBLE
METRIC = "DOF-stage updates/s (mixed vs FP64, same GB300) at stated error; % HBM roofline"
L2_BYTES = 129 * 1024 * 1024
MIXED_VARIANTS = ("mixed", "mixed_f32chem")

# Pipe peaks of this GPU model, measured with tests/cuda/fma_peak.cu (independent
# FMA chains on every SM, CUDA events, best of 5): the ALU denominators of the
# stage kernel. The derived figures are 152 SMs x 2.07 GHz x 4 flop/clk (FP64)
# and x 256 flop/clk (FP32): 1.259 and 80.5 TFLOP/s.
FP64_PEAK_TFLOPS = 1.056
FP32_PEAK_TFLOPS = 77.18
PEAK_NOTE = "FMA chains on 152 SMs (tests/cuda/fma_peak.cu), measured on GB300"


def stage_kernel_flops(wl, mech):
    """Algorithmic flops of one RK stage of one instance, the per-Gauss-point
    count of the method: DG operator nv (4 (p+1) + 6) FMA (modal-to-nodal, flux,
    volume and source quadrature, surface terms, update), thermodynamics 3 ns FMA,
    chemistry 12 nr flops (Arrhenius and equilibrium arguments, mass action,
    accumulation), with FMA = 2 flops. The 2 nr exponentials per point are
    counted apart (returned second): they run on the integer pipeline."""
    ns, nr = mech.ns, mech.nr
    nv, Q = ns + 2, wl.p + 1
    per_pt = 2 * nv * (4 * Q + 6) + 2 * 3 * ns + 12 * nr
    pts = wl.n_elem * Q
    return pts * per_pt, pts * 2 * nr


def stage_kernel_fp64_flops(wl, mech, prec):
    """FP64 flops one RK stage of one instance does by design in a mixed variant
    (FMA = 2), per Gauss point: the modal-to-nodal state 2 nv (p+1); the face
    traces for the flux 2 nv (ADG_MIXED_F32CHEM only: ADG_MIXED sums them in
    float); the temperature inversion 7 ns (the species sums of rho, q and c_v,
    and of R for the pressure) plus about 45 for u, T, ln T and 1/T (three Newton
    reciprocals and the table logarithm); the Arrhenius and equilibrium exponents
    8 nr (ADG_MIXED only); the RK accumulation 4 nv (on average over the three
    SSP-RK3 stages). The exponentials run on the integer pipe and are not
    counted."""
    ns, nr = mech.ns, mech.nr
    nv, Q = ns + 2, wl.p + 1
    per_pt = 2 * nv * Q + 7 * ns + 45 + 4 * nv
    per_pt += 8 * nr if prec == "mixed" else 2 * nv
    return wl.n_elem * Q * per_pt


def stage_kernel_bytes(wl, mech, prec):
    """Algorithmic DRAM bytes of one stage of one instance: the minimum traffic of
    a fused stage per vector DOF, 24 n_vars + 16 bytes in FP64 (read w^n and
    w^(s), write w^(s+1), 8 bytes each per variable, plus a 16-byte temperature
    guess) and 16 n_vars + 16 in the mixed variants (an FP64 read of w^n and FP32
    stage reads and writes)."""
    nv = mech.ns + 2
    per = (16 * nv + 16) if prec in MIXED_VARIANTS else (24 * nv + 16)
    return float(per) * wl.n_elem * (wl.p + 1)


def bench_workloads(name, instances=0):
    """The instances of a bench workload and their shared mechanism (for the
    ensemble, its first `instances` members when instances > 0)."""
    if name == ENSEMBLE:
        wls = I.ensemble_workloads()
        if instances > 0:
            wls = wls[:instances]
        return wls, wls[0].mechanism()
    wl = I.load_workloads()[name]
    return [wl], wl.mechanism()


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


def cpu_baseline(wls, mech, budget_s=12.0, max_steps=40):
    """The FP64 oracle (plain C, one instance per thread) on this host's cores,
    on a bounded sample of the workload: a single instance runs its first steps
    on one thread, as many as fit in about budget_s seconds; an ensemble runs
    its first instances, one step at a time, one per thread over all host cores
    (the oracle's ctypes calls release the interpreter lock), until the budget
    is spent. DOF-stages of the steps done over the wall time."""
    import oracle as O
    if len(wls) == 1:
        wl = wls[0]
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
        dofs = wl.n_elem * (wl.p + 1) * rk_stages(wl) * n
        return {"value": dofs / dt, "unit": "DOF-stage/s", "cores": 1, "kind": "oracle",
                "sample": "%s, first %d steps (%.1f s, 1 thread)" % (wl.name, n, dt)}
    cores = os.cpu_count() or 1
    sample = wls[:cores]
    done = [0] * len(sample)
    oracles = []
    for wl in sample:  # set-up outside the timed region
        o = O.Oracle(wl, mech)
        o.set_primitive(wl.primitive(mech))
        oracles.append(o)
    stop = time.perf_counter() + budget_s

    def work(k):
        while done[k] < max_steps and time.perf_counter() < stop:
            oracles[k].step(1)
            done[k] += 1
        return done[k]

    t0 = time.perf_counter()
    with ThreadPoolExecutor(cores) as ex:
        list(ex.map(work, range(len(sample))))
    dt = time.perf_counter() - t0
    dofs = sum(w.n_elem * (w.p + 1) * rk_stages(w) * n for w, n in zip(sample, done))
    return {"value": dofs / dt, "unit": "DOF-stage/s", "cores": cores, "kind": "oracle",
            "sample": "%s: instances 0..%d, %d to %d steps each, one per thread on %d "
                      "cores (%.1f s)" % (ENSEMBLE if len(wls) > 1 else wls[0].name,
                                          len(sample) - 1, min(done), max(done), cores, dt)}


def rk_stages(w):
    return 5 if getattr(w, "integrator", I.RK_SSP3) == I.RK_LS4 else 3


def dof_stages_per_step(wls):
    return sum(w.n_elem * (w.p + 1) * rk_stages(w) for w in wls)


def run_reference(args, ws, rank):
    if rank != 0:
        return 0
    wls, mech = bench_workloads(args.workload, args.instances)
    if args.viscous:
        wls = [I.viscous(w, name=w.name + "-viscous") for w in wls]
    cb = cpu_baseline(wls, mech, budget_s=max(5.0, 60.0 / max(1, args.steps + args.warmup)),
                      max_steps=max(1, args.steps))
    line = {"impl": "reference", "metric": METRIC, "value": cb["value"], "unit": cb["unit"],
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1e3 * dof_stages_per_step(wls) / cb["value"],
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": workload_config(wls, mech, args),
            "cpu_baseline": cb,
            "e2e": {"value": cb["value"], "unit": cb["unit"], "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line))
    return 0


def workload_config(wls, mech, args, mode="single", ws=1):
    """The whole job's workload (`wls`: every instance, over all ranks)."""
    par = {"single": "single", "replicas": "replicas x%d" % ws,
           "sharded": "instances sharded over %d ranks" % ws}[mode if ws > 1 else "single"]
    common = {"n_species": mech.ns, "n_reactions": mech.nr, "precision": args.precision,
              "l2": "flushed between timed steps (256 MiB write)",
              "launch": "CUDA graph per step", "parallelism": par}
    if len(wls) > 1:
        return dict(common, workload=args.workload, instances=len(wls),
                    n_elem_total=sum(w.n_elem for w in wls),
                    gauss_points=sum(w.n_elem * (w.p + 1) for w in wls),
                    degrees=sorted(set(w.p for w in wls)), delay_mode="saa",
                    max_delay=max(w.max_delay for w in wls), limiter="weno", flux="lf")
    wl = wls[0]
    return dict(common, workload=wl.name, n_elem=wl.n_elem, p=wl.p, n_pe=wl.n_pe,
                max_delay=wl.max_delay, at_order=wl.at_order,
                delay_mode=["sync", "caa", "saa"][wl.delay_mode],
                flux=["lf", "hllc"][wl.flux], limiter=["none", "weno"][wl.limiter], dt=wl.dt)


def mass_fractions(w, p):
    x, _ = np.polynomial.legendre.leggauss(p + 1)
    V = np.polynomial.legendre.legvander(x, p)
    r = np.einsum("inj,qj->inq", w[2:], V)
    return r / r.sum(axis=0, keepdims=True)


def measure(adg, torch, wls, mech, prims, prec, args, dev, pg, steps, autotune=True):
    """Warm-up, autotune, device-timed steps and the end-to-end run of one
    precision variant on its own context."""
    g = adg.ADG(mech, wls, device=dev, precision=prec)
    for k, prim in enumerate(prims):
        g.set_primitive(prim, k)
    stream = torch.cuda.current_stream(dev)
    flush = torch.empty(2 * L2_BYTES // 4, dtype=torch.float32, device=dev)

    g.step(args.warmup, stream)
    g.check()
    torch.cuda.synchronize(dev)
    if args.tuning:
        # "TE,NT[,EPB]" for every group, or "TE,NT[,EPB];..." per group in order
        parts = [x for x in args.tuning.split(";") if x]
        tuning = None
        for gi in range(len(g.tuning())):
            vals = [int(x) for x in parts[min(gi, len(parts) - 1)].split(",")]
            tuning = g.set_tuning(gi, vals[0], vals[1])
            if len(vals) > 2:
                tuning = g.set_limiter_tuning(gi, vals[2])
    else:
        tuning = g.autotune(stream) if autotune and not args.no_autotune else g.tuning()
    torch.cuda.synchronize(dev)

    # device-resident timing: every step is one replay of the step's CUDA graph,
    # bracketed by an event pair on the launching stream, timed alone, with the
    # L2 flushed between steps. A second pass replays the instrumented graph
    # (an event pair around every kernel) for the per-kernel times; its event
    # nodes separate the kernels, so its step time is not the headline.
    sampler = ClockSampler(dev.index or 0)
    if pg:
        pg.barrier()
    torch.cuda.synchronize(dev)
    sampler.start()
    time.sleep(0.3)
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
           for _ in range(steps)]
    wall0 = time.perf_counter()
    for a, b in evs:
        flush.zero_()
        a.record(stream)
        g.step(1, stream)
        b.record(stream)
    torch.cuda.synchronize(dev)
    wall = time.perf_counter() - wall0
    ms = float(sum(a.elapsed_time(b) for a, b in evs))
    g.check()
    g.enable_kernel_timing(True)
    for k in range(steps):
        flush.zero_()
        g.step(1, stream)
    torch.cuda.synchronize(dev)
    kms, kn = g.kernel_times()
    g.enable_kernel_timing(False)
    clocks = sampler.stop()
    g.check()
    launches = g.launches_per_step() * steps
    # the longest rank's time and the units of all ranks (this rank's instances:
    # its shard of an ensemble, or a replica of a single problem)
    dof_stage = dof_stages_per_step(wls)
    ms, dof_all = SH.reduce_rate(pg, ms, dof_stage, dev)
    value = dof_all * steps / (ms / 1e3)

    # end to end through the C ABI with host buffers: every step copies every
    # instance's state in from pinned host memory, steps it and copies it out
    # (adg_step_io: the same as adg_write_states + adg_step + adg_read_states,
    # with each degree group's copies overlapped with other groups' stages)
    n_all = g.states_doubles()
    host_in = torch.empty(n_all, dtype=torch.float64, pin_memory=True)
    host_out = torch.empty(n_all, dtype=torch.float64, pin_memory=True)
    g.read_states(host_in.numpy(), stream=stream)
    nbytes = 8 * n_all
    # one untimed call captures the step's graph for this pair of buffers
    g.step_io(host_in.numpy(), host_out.numpy(), stream=stream)
    torch.cuda.synchronize(dev)
    n_e2e = max(3, steps // 3)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    t0 = time.perf_counter()
    e0.record(stream)
    for _ in range(n_e2e):
        g.step_io(host_in.numpy(), host_out.numpy(), stream=stream)
        stream.synchronize()
    e1.record(stream)
    torch.cuda.synchronize(dev)
    e2e_ms = max(e0.elapsed_time(e1), (time.perf_counter() - t0) * 1e3)
    g.check()
    e2e_ms, _ = SH.reduce_rate(pg, e2e_ms, dof_stage, dev)
    e2e_value = dof_all * n_e2e / (e2e_ms / 1e3)
    g.close()
    del flush
    return {"value": value, "ms": ms, "kms": kms, "kn": kn, "launches": launches,
            "ms_instrumented": float(kms[2]), "tuning": tuning, "steps": steps,
            "clocks": clocks, "wall": wall, "nbytes": nbytes,
            "e2e": {"value": e2e_value, "unit": "DOF-stage/s", "h2d_bytes_per_step": nbytes,
                    "d2h_bytes_per_step": nbytes, "call": "adg_step_io"}}


def state_scales(w, mech):
    """Physical scale of every conserved variable of a modal state [nv][N][Q]:
    max rho (|u| + a) for the momentum (the acoustic scale: at early times the
    momentum itself is near zero), max |rho E| for the energy, and
    max(max rho Y_i, 1e-5 max rho) for the partial densities (cell averages)."""
    ru = 8.314462618
    scale = np.abs(w).max(axis=(1, 2))
    r = w[2:, :, 0]
    rho = r.sum(axis=0)
    u = w[0, :, 0] / rho
    q = ((mech.h_f - mech.cp * 298.15) / mech.W)[:, None]
    cv = ((mech.cp - ru) / mech.W)[:, None]
    T = (w[1, :, 0] - 0.5 * rho * u * u - (r * q).sum(0)) / (r * cv).sum(0)
    cpm = (r * (mech.cp / mech.W)[:, None]).sum(0)
    cvm = (r * cv).sum(0)
    a = np.sqrt(np.abs(cpm / cvm * (cpm - cvm) / rho * T))
    scale[0] = max(scale[0], float(np.max(rho * (np.abs(u) + a))))
    scale[2:] = np.maximum(scale[2:], 1e-5 * rho.max())
    return np.maximum(scale, 1e-300)


def unsync_measure(adg, torch, wl, mech, prim, prec, dev, warmup, steps):
    """The truly unsynchronised mode on the same instance: one cooperative launch
    of `steps` steps (one CTA per PE, no lockstep), device-timed; the delays the
    PEs used; its distance from the seeded-delay synchronous run of the same
    number of steps (L-infinity per conserved variable in the scales of
    state_scales), beside the same distance of the synchronous run without
    delays; the drift of total mass and energy."""
    stream = torch.cuda.current_stream(dev)
    g = adg.ADG(mech, [wl], device=dev, precision=prec)
    g.set_primitive(prim)
    w0 = g.get_state()
    g.step_unsync(warmup, stream=stream)
    g.check()
    g.unsync_delays()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize(dev)
    e0.record(stream)
    g.step_unsync(steps, stream=stream)
    e1.record(stream)
    torch.cuda.synchronize(dev)
    ms = e0.elapsed_time(e1)
    g.check()
    hist = g.unsync_delays()
    w = g.get_state()
    g.close()
    ref = {}
    for mode, cfg in (("seeded", wl), ("sync", dataclasses.replace(wl, delay_mode=I.DELAY_SYNC))):
        r = adg.ADG(mech, [cfg], device=dev, precision=prec)
        r.set_primitive(prim)
        r.step(warmup + steps, stream)
        r.check()
        ref[mode] = r.get_state()
        r.close()
    wr = ref["seeded"]
    scale = state_scales(wr, mech)
    ev = np.abs(w - wr).max(axis=(1, 2)) / scale
    es = np.abs(ref["sync"] - wr).max(axis=(1, 2)) / scale
    drift = {"mass": float(abs(w[2:, :, 0].sum() - w0[2:, :, 0].sum()) / w0[2:, :, 0].sum()),
             "energy": float(abs(w[1, :, 0].sum() - w0[1, :, 0].sum()) / abs(w0[1, :, 0].sum()))}
    value = dof_stages_per_step([wl]) * steps / (ms / 1e3)
    return {"value": value, "unit": "DOF-stage/s", "ms_per_step": ms / steps, "steps": steps,
            "warmup": warmup, "precision": prec, "launches": 3,
            "l2": "resident (one launch runs every step)",
            "delays_flux": [int(x) for x in hist[0, :wl.max_delay + 1]],
            "delays_limiter": [int(x) for x in hist[1, :wl.max_delay + 1]],
            "error_vs_seeded": float(ev.max()),
            "error_vs_seeded_per_variable": [float(x) for x in ev],
            "sync_vs_seeded": float(es.max()),
            "error_scales": "momentum: max rho(|u|+a); energy: max|rho E|; "
                            "rho Y_i: max(max rho Y_i, 1e-5 max rho)",
            "relative_drift": drift}


def decomposed_measure(adg, torch, wl, mech, prim, dev, warmup, steps, n_sub=4):
    """One problem cut into n_sub subdomains of whole PEs (domain.py), held as the
    instances of one context on this GPU and stepped half-stage by half-stage,
    with their boundary blocks moved by adg_part_block between the halves: first
    as plain launches and device copies on one stream, then the same step
    captured as one CUDA graph and replayed (the headline of the record). The
    rate counts the whole domain's DOFs only (not the buffer elements); the
    state after both runs is compared bit for bit with the whole-domain run of
    the same steps."""
    from paper_2501_01747_gb300 import domain as D
    subs = [D.subdomain(wl, pb, pe) for pb, pe in D.split_pes(wl.n_pe, n_sub)]
    g = adg.ADG(mech, subs, device=dev, precision="mixed")
    parts = [D.AdgPart(g, k) for k in range(len(subs))]
    for k, part in enumerate(parts):
        g.set_primitive(D.local_slice(prim, wl.n_elem, part.elem0, part.n_local, axis=1), k)
    ex = D.LocalExchange(parts)
    S = rk_stages(wl)
    stream = torch.cuda.current_stream(dev)
    D.advance(warmup, S, g.step_stage, ex)
    torch.cuda.synchronize(dev)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    # plain launches, then the same step captured as a CUDA graph and replayed
    e0.record(stream)
    D.advance(steps, S, g.step_stage, ex)
    e1.record(stream)
    torch.cuda.synchronize(dev)
    ms_plain = e0.elapsed_time(e1)
    graph = D.capture_step(S, g.step_stage, ex, dev)
    torch.cuda.synchronize(dev)
    e0.record(stream)
    for _ in range(steps):
        graph.replay()
    e1.record(stream)
    torch.cuda.synchronize(dev)
    ms = e0.elapsed_time(e1)
    g.check()
    got = np.concatenate([D.owned(g.get_state(k), *p_.cut, axis=1)
                          for k, p_ in enumerate(parts)], axis=1)
    g.close()
    w = adg.ADG(mech, [wl], device=dev, precision="mixed")
    w.set_primitive(prim)
    w.step(warmup + 2 * steps)
    ref = w.get_state()
    w.close()
    rate = dof_stages_per_step([wl]) * steps
    return {"workload": wl.name, "precision": "mixed", "subdomains": n_sub,
            "pe_ranges": D.split_pes(wl.n_pe, n_sub),
            "launch": "one CUDA graph per step: per half-stage the stage or limiter kernels "
                      "and the block moves (adg_part_block) of every subdomain; buffer "
                      "elements computed and discarded",
            "value": rate / (ms / 1e3), "unit": "DOF-stage/s", "steps": steps,
            "ms_per_step": ms / steps,
            "plain_launches": {"value": rate / (ms_plain / 1e3), "ms_per_step": ms_plain / steps},
            "bit_identical_to_whole_domain": bool(np.array_equal(got, ref))}


def mixed_error(adg, torch, wls, mech, prims, dev, n_steps, variant="mixed"):
    """Error of a mixed variant against the FP64 path (which matches the FP64
    oracle to 1e-10) after n_steps from the same state: the largest relative
    error of T at the Gauss points, and the error of every mass fraction at the
    Gauss points where it is above 1e-8, relative to the largest value of that
    species (relative L-infinity) and, for information, to the local value."""
    out = {}
    for prec in ("fp64", variant):
        g = adg.ADG(mech, wls, device=dev, precision=prec)
        for k, prim in enumerate(prims):
            g.set_primitive(prim, k)
        g.step(n_steps)
        g.check()
        out[prec] = [(g.temperature(k), mass_fractions(g.get_state(k), wl.p))
                     for k, wl in enumerate(wls)]
        g.close()
    eT, eY, eP = 0.0, 0.0, 0.0
    for (T0, Y0), (T1, Y1) in zip(out["fp64"], out[variant]):
        eT = max(eT, float((np.abs(T1 - T0) / T0).max()))
        for i in range(Y0.shape[0]):
            big = Y0[i] > 1e-8
            if big.any():
                d = np.abs(Y1[i] - Y0[i])[big]
                eY = max(eY, float(d.max() / Y0[i].max()))
                eP = max(eP, float((d / Y0[i][big]).max()))
    return {"steps": n_steps, "reference": "FP64 GPU path (<= 1e-10 from the FP64 oracle)",
            "T_rel_max": eT, "Y_rel_linf": eY, "Y_rel_pointwise": eP,
            "bar": "1e-4: T at every Gauss point; Y_i relative to max Y_i where Y_i > 1e-8"}


def roofline(wls, mech, r, prec, peaks, src, traffic_key=None):
    """Roofline of the stage kernel (the dominant one) over one RK stage of every
    instance, all degree groups, against the stage kernels' time for that stage.
    The kernel does more FP64 work per DRAM byte (about 1.4 flop/byte in
    ADG_MIXED on the ensemble) than the FP64 ridge point (the measured FP64 FMA
    peak over the measured HBM copy bandwidth, 0.16 flop/byte), and ncu finds the
    FP64 pipe its busiest unit, so its roof is the FP64 pipe: the primary figure
    is the FP64 flops the variant does by design (all algorithmic flops in FP64,
    stage_kernel_fp64_flops in the mixed variants) against the measured FP64 FMA
    peak. Beside it: the algorithmic bytes (stage_kernel_bytes) against the
    measured HBM copy bandwidth, and in the mixed variants all algorithmic flops
    against the FP32 pipe."""
    n_st = max(rk_stages(w) for w in wls)  # stage launches per step (uniform here)
    stage_s = r["kms"][0] / 1e3 / (n_st * r["steps"])
    nbytes = sum(stage_kernel_bytes(w, mech, prec) for w in wls)
    flops = sum(stage_kernel_flops(w, mech)[0] for w in wls)
    n_exp = sum(stage_kernel_flops(w, mech)[1] for w in wls)
    hbm = peaks.get("hbm_gbs", 6800.0)
    mixed = prec in MIXED_VARIANTS
    f64 = sum(stage_kernel_fp64_flops(w, mech, prec) for w in wls) if mixed else flops
    tr = STAGE_TRAFFIC.get((traffic_key, KERNEL_REV, prec)) if traffic_key else None
    out = {"bound": "alu", "pipe": "fp64",
           "achieved": f64 / stage_s / 1e12, "peak": FP64_PEAK_TFLOPS, "unit": "TFLOP/s",
           "frac": f64 / stage_s / 1e12 / FP64_PEAK_TFLOPS, "traffic": tr,
           "peak_source": PEAK_NOTE,
           "kernel": "stage_kernel (%s), all degree groups of one RK stage" % prec,
           "fp64_flops_per_stage": f64,
           "fp64_flops_per_dram_byte": f64 / (tr or nbytes),
           "ridge_flops_per_byte": FP64_PEAK_TFLOPS * 1e12 / (hbm * 1e9),
           "exp_per_s": n_exp / stage_s,
           "kernel_ms": stage_s * 1e3,
           "kernel_share": r["kms"][0] / max(1e-9, r["kms"][0] + r["kms"][1]),
           "limiter_ms": r["kms"][1] / (n_st * r["steps"]),
           "hbm": {"achieved": nbytes / stage_s / 1e9, "peak": hbm, "unit": "GB/s",
                   "frac": nbytes / stage_s / 1e9 / hbm,
                   "peak_source": "%s (MEASURED_PEAKS.json hbm_gbs)" % src,
                   "algorithmic_bytes_per_stage": nbytes,
                   "bytes_per_vector_dof": (16 if mixed else 24) * (mech.ns + 2) + 16}}
    if mixed:
        out["fp32"] = {"achieved": flops / stage_s / 1e12, "peak": FP32_PEAK_TFLOPS,
                       "unit": "TFLOP/s", "frac": flops / stage_s / 1e12 / FP32_PEAK_TFLOPS,
                       "algorithmic_flops_per_stage": flops, "peak_source": PEAK_NOTE}
    return out


def compare(adg, torch, wls, mech, prims, args, dev, pg, steps, autotune=True,
            err_steps=200, variants=None):
    """The precision variants on the same workload, the headline one first; the
    mixed variants' error against the FP64 path."""
    variants = variants or [args.precision] + [v for v in ("fp64", "mixed", "mixed_f32chem")
                                               if v != args.precision]
    if args.only:
        variants = variants[:1]
    res = {}
    for v in variants:
        res[v] = measure(adg, torch, wls, mech, prims, v, args, dev, pg, steps, autotune)
    err = {}
    if "fp64" in variants:
        for v in variants:
            if v in MIXED_VARIANTS:
                err[v] = mixed_error(adg, torch, wls, mech, prims, dev, err_steps, v)
    return res, err


def variant_record(wls, mech, r, prec, steps, peaks, src, key):
    return {"value": r["value"], "unit": "DOF-stage/s", "ms_per_step": r["ms"] / steps,
            "e2e": r["e2e"], "roofline": roofline(wls, mech, r, prec, peaks, src, key),
            "clocks": r["clocks"], "tuning": r["tuning"], "gpu_launches": int(r["launches"])}


def sub_record(wls, all_wls, mech, res, err, steps, peaks, src, key, args, mode, ws):
    """Every variant of one workload as a nested record."""
    rec = {"config": workload_config(all_wls, mech, args, mode, ws), "steps": steps}
    for v, r in res.items():
        rec[v] = variant_record(wls, mech, r, v, steps, peaks, src, key)
    if "fp64" in res:
        for v in MIXED_VARIANTS:
            if v in res:
                rec["speedup_%s_vs_fp64" % v] = res[v]["value"] / res["fp64"]["value"]
    if err:
        rec["mixed_error"] = err
    return rec


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--workload", default=DEFAULT_WORKLOAD,
                    help="a base workload name or %s" % ENSEMBLE)
    ap.add_argument("--precision", default="mixed", choices=["mixed", "fp64", "mixed_f32chem"],
                    help="the headline variant; the others are timed beside it")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-autotune", action="store_true")
    ap.add_argument("--tuning", default="", help="TE,NT[,EPB] (every group) or TE,NT[,EPB];... "
                    "(one per group, in the order of config.tuning): set the stage launch "
                    "configuration (and the limiter's elements per CTA) of the headline "
                    "variant instead of autotuning it")
    ap.add_argument("--only", action="store_true",
                    help="time the headline variant of the headline workload only")
    ap.add_argument("--instances", type=int, default=0,
                    help="run the first N instances of the ensemble (0: all 512), for "
                         "profiling captures of a smaller case")
    ap.add_argument("--sub-steps", type=int, default=100,
                    help="timed steps of the 9-species ignition sub-record (0: none)")
    ap.add_argument("--large-steps", type=int, default=10,
                    help="timed steps of the 53-species detonation sub-record (0: none)")
    ap.add_argument("--unsync-steps", type=int, default=100,
                    help="steps of the unsynchronised-mode measurement on the 9-species "
                         "ignition (0 to skip)")
    ap.add_argument("--lserk-steps", type=int, default=100,
                    help="timed steps of the LSERK4 measurement (the 5-stage 4th-order "
                         "low-storage integrator) on the 9-species ignition; 0 to skip")
    ap.add_argument("--domain-steps", type=int, default=20,
                    help="steps of the domain-decomposed run (4 subdomains of the ignition "
                         "workload in one context); 0 leaves it out")
    ap.add_argument("--viscous", action="store_true",
                    help="run the headline workload with the viscous terms")
    ap.add_argument("--visc-steps", type=int, default=100,
                    help="timed steps of the viscous measurement (the diffusive flux with "
                         "the LDG auxiliary kernel) on the 9-species ignition; 0 to skip")
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
    peaks, src = load_peaks()

    def shard(name, viscous=False):
        wls_all, mech = bench_workloads(name, args.instances if name == ENSEMBLE else 0)
        if viscous:
            wls_all = [I.viscous(w, name=w.name + "-viscous") for w in wls_all]
        idx, mode = SH.assign(len(wls_all), rank, ws)
        wls = [wls_all[k] for k in idx]
        return wls_all, wls, mech, mode

    all_wls, wls, mech, mode = shard(args.workload, args.viscous)
    prims = [w.primitive(mech) for w in wls]
    err_steps = 48 if len(wls) == 1 else 20
    res, err = compare(adg, torch, wls, mech, prims, args, dev, pg, args.steps,
                       err_steps=err_steps)
    head = res[args.precision]
    # measured traffic exists for the full workloads only
    key = args.workload if not (args.viscous or args.instances) else None

    subs = {}
    single = None  # the 9-species ignition instance, for the mode measurements
    if not args.only and args.sub_steps > 0 and args.workload != IGNITION:
        s_all, s_wls, s_mech, s_mode = shard(IGNITION)
        s_prims = [w.primitive(s_mech) for w in s_wls]
        sargs = argparse.Namespace(**vars(args))
        sargs.tuning = ""
        # the mixed error after 48 steps: beyond, the FP64 scheme's own response to
        # a single-precision change of its state exceeds the mixed bar
        sres, serr = compare(adg, torch, s_wls, s_mech, s_prims, sargs, dev, pg,
                             args.sub_steps, err_steps=48)
        subs["ignition"] = sub_record(s_wls, s_all, s_mech, sres, serr, args.sub_steps, peaks,
                                      src, IGNITION, sargs, s_mode, ws)
        single = (s_wls[0], s_mech, s_prims[0])
    elif len(wls) == 1:
        single = (wls[0], mech, prims[0])
    if not args.only and args.large_steps > 0 and args.workload != LARGE:
        l_all, l_wls, l_mech, l_mode = shard(LARGE)
        l_prims = [w.primitive(l_mech) for w in l_wls]
        largs = argparse.Namespace(**vars(args))
        largs.tuning = ""
        lres, lerr = compare(adg, torch, l_wls, l_mech, l_prims, largs, dev, pg,
                             args.large_steps, err_steps=10, variants=["mixed", "fp64"])
        subs["detonation_53sp"] = sub_record(l_wls, l_all, l_mech, lres, lerr, args.large_steps,
                                             peaks, src, LARGE, largs, l_mode, ws)

    uns = lsk = vis = dec = None
    if single is not None and not args.only:
        swl, smech, sprim = single
        if args.domain_steps > 0 and swl.n_pe >= 4:
            dec = decomposed_measure(adg, torch, swl, smech, sprim, dev, args.warmup,
                                     args.domain_steps)
        if args.unsync_steps > 0:
            uns = unsync_measure(adg, torch, swl, smech, sprim, "mixed", dev, args.warmup,
                                 args.unsync_steps)
        if args.lserk_steps > 0:
            lw = dataclasses.replace(swl, integrator=I.RK_LS4, name=swl.name + "-lserk4")
            lsk = (lw, smech, measure(adg, torch, [lw], smech, [sprim], "mixed", args, dev, pg,
                                      args.lserk_steps))
        if args.visc_steps > 0 and not args.viscous:
            vw = I.viscous(swl, name=swl.name + "-viscous")
            vis = (vw, smech, measure(adg, torch, [vw], smech, [sprim], "mixed", args, dev, pg,
                                      args.visc_steps))

    if rank != 0:
        return 0
    mixed = args.precision in MIXED_VARIANTS
    line = {
        "metric": METRIC, "value": head["value"], "unit": "DOF-stage/s", "n_gpus": ws,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": head["ms"] / args.steps,
        "higher_is_better": True,
        # replicas keep the per-GPU work fixed; a sharded ensemble, the total
        "scaling": "strong" if (mode == "sharded" and ws > 1) else "weak", "vs_baseline": None,
        "dtype": "f32+f64" if mixed else "f64",
        "data": "synthetic", "config": dict(workload_config(all_wls, mech, args, mode, ws),
                                            tuning=head["tuning"]),
        "roofline": roofline(wls, mech, head, args.precision, peaks, src, key),
        "clocks": head["clocks"],
        "e2e": head["e2e"],
        "gpu_launches": int(head["launches"]),
        "ms_per_step_instrumented": head["ms_instrumented"] / args.steps,
        "value_scalar_dofs": head["value"] * (mech.ns + 2),  # x N_var conserved variables
        "wall_s": head["wall"],
    }
    for v, r in res.items():
        if v != args.precision:
            line[v] = variant_record(wls, mech, r, v, args.steps, peaks, src, key)
    if "fp64" in res:
        for v in MIXED_VARIANTS:
            if v in res:
                line["speedup_%s_vs_fp64" % v] = res[v]["value"] / res["fp64"]["value"]
    if err:
        line["mixed_error"] = err
    line.update(subs)
    if uns is not None:
        line["unsync"] = uns
    if dec is not None:
        whole = subs.get("ignition", {}).get("mixed", {}).get("value")
        if whole:
            dec["vs_whole_domain_graph"] = dec["value"] / whole
        line["decomposed"] = dec
    if vis is not None:
        vw, vmech, r = vis
        line["viscous"] = {
            "terms": "diffusive flux of Sec. 2 by LDG (auxiliary kernel + viscous stage "
                     "kernel; the stage time includes the auxiliary kernel)",
            "workload": vw.name, "precision": "mixed",
            "dt": vw.dt, "dt_note": "p = 4 runs the viscous terms at dt/8 (explicit "
                                    "diffusive limit), so a step covers 1/8 of the time",
            "value": r["value"], "unit": "DOF-stage/s", "steps": args.visc_steps,
            "ms_per_step": r["ms"] / args.visc_steps, "e2e": r["e2e"],
            "roofline": dict(roofline([vw], vmech, r, "mixed", peaks, src),
                             note="algorithmic bytes and flops of the Euler terms only"),
            "clocks": r["clocks"], "tuning": r["tuning"]}
    if lsk is not None:
        lw, lmech, r = lsk
        line["lserk4"] = {
            "integrator": "LSERK 5-stage 4th order (2N storage), limiter after every stage",
            "workload": lw.name, "precision": "mixed",
            "stages_per_step": 5, "value": r["value"], "unit": "DOF-stage/s",
            "steps": args.lserk_steps, "ms_per_step": r["ms"] / args.lserk_steps,
            "e2e": r["e2e"], "roofline": roofline([lw], lmech, r, "mixed", peaks, src),
            "clocks": r["clocks"], "tuning": r["tuning"]}
    if not args.no_cpu_baseline and ws == 1:
        line["cpu_baseline"] = cpu_baseline(wls, mech)
    print(json.dumps(line))
    return 0


# DRAM bytes (read + write) of the stage-kernel launches of one RK stage (all
# degree groups) from ncu, per (workload, kernel revision, precision); the
# summaries are under profiles/.
STAGE_TRAFFIC = {
    (ENSEMBLE, "v20", "mixed"): 2.655e9,
    (ENSEMBLE, "v20", "fp64"): 2.663e9,
    (ENSEMBLE, "v20", "mixed_f32chem"): 2.656e9,
    (ENSEMBLE, "v21", "mixed"): 2.655e9,
    (ENSEMBLE, "v21", "fp64"): 2.662e9,
    (ENSEMBLE, "v21", "mixed_f32chem"): 2.656e9,
}

KERNEL_REV = "v21"

if __name__ == "__main__":
    sys.exit(main())
