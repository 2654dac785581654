"""Parity of the CUDA path (through the C ABI) with the FP64 oracle.

Bar (FP64 path): relative L-infinity error <= 1e-10 on every conserved variable,
the error of variable v being max|w_gpu - w_oracle| / scale_v over all elements
and modes, with the physical scale of each variable: max|rho E| for the energy,
max rho (|u| + a) for the momentum, max|rho Y_i| for a partial density, floored
at 1e-5 of the largest density. Relative to its own maximum, the momentum of a
gas at rest or a species at a mass fraction of 1e-12 moves by 1e-6 when the
oracle's own input moves by 1e-15; in these scales the oracle moves by less than
1e-11 (tests/test_oracle_conditioning.py), ten times below the bar.
Troubled-cell flags must be identical (per stage of the last step and counted
over the whole run)."""
import dataclasses

import numpy as np
import pytest

import oracle as O
from paper_2501_01747_gb300 import adg
from paper_2501_01747_gb300 import inputs as I
from tests import helpers as H

pytestmark = pytest.mark.gpu

TOL = 1e-10


def scales(w, mech):
    return H.parity_scales(w, mech)


def rel_err(a, b, mech=None):
    mech = mech if mech is not None else CURRENT_MECH[0]
    return H.parity_error(a, b, mech)


CURRENT_MECH = [None]


def run_both(wl, mech, prim, n_steps, chunks=1):
    CURRENT_MECH[0] = mech
    g = adg.ADG(mech, [wl])
    g.set_primitive(prim)
    o = O.Oracle(wl, mech)
    o.set_primitive(prim)
    per = n_steps // chunks
    for _ in range(chunks):
        g.step(per)
        o.step(per)
    g.check()
    return g, o


def assert_parity(g, o, tol=TOL, flags=True):
    w, ref = g.get_state(), o.state()
    err = rel_err(w, ref)
    assert np.all(np.isfinite(w))
    assert err.max() <= tol, err
    if flags:
        gl, gc = g.flags()
        ol, oc = o.flags()
        assert np.array_equal(gc, oc), np.flatnonzero(gc != oc)[:10]
        assert np.array_equal(gl, ol)
    return err


def W():
    return I.load_workloads()


def test_ignition_5sp_full_run():
    """The 5-species ignition workload as configured: 200 x p3, 4 PEs, SAA delays
    (set 1), AT order 4, WENO, 500 steps."""
    wl = W()["ignition-5sp-200x3"]
    mech = wl.mechanism()
    prim = wl.primitive(mech)
    g, o = run_both(wl, mech, prim, 500, chunks=5)
    assert g.steps_done() == 500
    assert_parity(g, o)
    T = g.temperature()
    assert np.abs(T - o.temperature()).max() <= 1e-9 * T.max()


@pytest.mark.parametrize("mode", [I.DELAY_SYNC, I.DELAY_CAA, I.DELAY_SAA])
@pytest.mark.parametrize("flux", [I.FLUX_LF, I.FLUX_HLLC])
def test_delay_modes_and_fluxes(mode, flux):
    wl = W()["ignition-5sp-200x3"]
    wl.delay_mode, wl.flux = mode, flux
    mech = wl.mechanism()
    g, o = run_both(wl, mech, wl.primitive(mech), 120)
    assert_parity(g, o)


@pytest.mark.parametrize("p", [1, 2, 3, 4])
def test_every_degree_ragged_mesh_shock(p):
    """Prime element count (ragged last tile), reflecting wall and outflow, HLLC,
    WENO on a shock, SAA delays with AT order p+1, the 9-species mechanism."""
    base = W()["detonation-9sp-16384x3"]
    wl = I.scaled(base, 97, 7)
    wl.p = p
    wl.at_order = p + 1
    wl.dt = base.dt * 0.05
    mech = wl.mechanism()
    g, o = run_both(wl, mech, wl.primitive(mech), 60)
    assert_parity(g, o)
    assert o.flags()[1].sum() > 0


@pytest.mark.parametrize("case", ["20sp", "53sp"])
def test_large_mechanisms_small_mesh(case):
    """Mechanisms whose temperature inversion sums its species on 4 lanes per
    Gauss point (16 to 31 species: a 20-species, 12-reaction draw on the
    ignition shape) and on 8 (32 and more: the 53-species, 325-reaction
    mechanism on the detonation shape), on 97 ragged elements and 7 PEs with
    SAA delays and WENO: full comparison with the oracle, flags included."""
    if case == "20sp":
        base = W()["ignition-5sp-200x3"]
        wl = dataclasses.replace(I.scaled(base, 97, 7), ns=20, nr=12, mech_seed=5, attempts=None)
        steps = 40
    else:
        base = W()["detonation-53sp-65536x3"]
        wl = I.scaled(base, 97, 7)
        wl.dt = base.dt * 0.25
        steps = 20
    mech = wl.mechanism()
    g, o = run_both(wl, mech, wl.primitive(mech), steps)
    assert_parity(g, o)
    assert o.flags()[1].sum() > 0


def test_one_element_per_pe_and_single_pe():
    wl = W()["ignition-5sp-200x3"]
    mech = wl.mechanism()
    for n_pe, steps in [(1, 60), (200, 40)]:
        w = I.scaled(wl, 200, n_pe)
        w.dt = wl.dt * 0.25
        g, o = run_both(w, mech, w.primitive(mech), steps)
        assert_parity(g, o)


def test_no_limiter_and_tvb():
    wl = W()["ignition-5sp-200x3"]
    mech = wl.mechanism()
    wl.limiter = I.LIM_NONE
    g, o = run_both(wl, mech, wl.primitive(mech), 80)
    assert_parity(g, o)
    assert g.flags()[1].sum() == 0
    wl2 = W()["ignition-5sp-200x3"]
    wl2.tvb_M = 50.0
    g, o = run_both(wl2, mech, wl2.primitive(mech), 80)
    assert_parity(g, o)


def test_ignition_9sp_full_size():
    """4096 x p4, 21 reactions, 64 PEs, delays up to 4 with AT order 5, 48 steps:
    well past the first step (8) at which the largest delay can be in force."""
    wl = W()["ignition-9sp-4096x4"]
    mech = wl.mechanism()
    g, o = run_both(wl, mech, wl.primitive(mech), 48, chunks=2)
    assert_parity(g, o)


def test_detonation_9sp_full_size():
    """16384 x p3, HLLC, WENO, reflecting/outflow, 256 PEs, delays up to 3, 40
    steps (the largest delay can be in force from step 6)."""
    wl = W()["detonation-9sp-16384x3"]
    mech = wl.mechanism()
    g, o = run_both(wl, mech, wl.primitive(mech), 40, chunks=2)
    assert_parity(g, o)
    assert o.flags()[1].sum() > 0


def test_detonation_53sp_full_size_windows():
    """65536 x p3 with 53 species / 325 reactions, 1024 PEs, SAA delays up to 4
    with AT order 4: 10 full-size GPU steps (the largest delay can be in force
    from step 7), checked on windows of three whole PEs. An element's update in
    one step depends on the elements within 6 of it (a face flux and a limiter
    stencil in each of 3 stages), so an oracle run on the window alone, with its
    PE faces numbered as in the full run (the same SAA draws), agrees with the
    full run on the elements further than 60 from a cut; that part holds both of
    the window's inner PE faces, where the AT flux and the AT-WENO neighbour
    read the history ring. Windows: at the reflecting wall, across the driver's
    shock, and in the ambient gas."""
    from concurrent.futures import ThreadPoolExecutor
    wl = W()["detonation-53sp-65536x3"]
    mech = wl.mechanism()
    prim = wl.primitive(mech)
    n_steps = 10
    assert n_steps >= wl.max_delay + wl.at_order + 2
    g = adg.ADG(mech, [wl])
    g.set_primitive(prim)
    g.step(n_steps)
    g.check()
    w = g.get_state()
    gl, gc = g.flags()
    scale = scales(w, mech)
    epe = wl.n_elem // wl.n_pe
    dx = wl.length / wl.n_elem
    reach = 6 * n_steps

    def window(j):
        """Oracle on global PEs j-1, j, j+1: (first element, valid range, oracle)."""
        e0 = epe * (j - 1)
        win = I.scaled(wl, 3 * epe, 3)
        win.x0 = wl.x0 + e0 * dx
        win.face0 = j - 1
        win.bc_left = wl.bc_left if j == 1 else I.BC_OUTFLOW
        win.bc_right = wl.bc_right if j + 2 == wl.n_pe else I.BC_OUTFLOW
        o = O.Oracle(win, mech)
        o.set_primitive(prim[:, e0:e0 + 3 * epe])
        o.step(n_steps)
        lo = 0 if j == 1 else reach
        hi = 3 * epe if j + 2 == wl.n_pe else 3 * epe - reach
        return e0, lo, hi, o

    shock = int(0.05 * wl.n_elem) // epe
    with ThreadPoolExecutor(3) as ex:
        res = list(ex.map(window, [1, shock, 700]))
    for e0, lo, hi, o in res:
        assert lo < epe and hi > 2 * epe  # both inner PE faces are checked
        ref = o.state()[:, lo:hi]
        got = w[:, e0 + lo:e0 + hi]
        err = (np.abs(got - ref) / np.maximum(scale, 1e-300)[:, None, None]).max()
        assert err <= TOL, (e0, err)
        ol, oc = o.flags()
        assert np.array_equal(gl[:, e0 + lo:e0 + hi], ol[:, lo:hi]), e0
        assert np.array_equal(gc[e0 + lo:e0 + hi], oc[lo:hi]), e0


def test_ensemble_of_instances_in_one_context():
    """Several instances of different degree and size stepping together."""
    ens = I.ensemble_workloads()
    mech = ens[0].mechanism()
    pick = []
    for p in (2, 3, 4):
        k = next(i for i, w in enumerate(ens) if w.p == p)
        pick.append(I.scaled(ens[k], 67 + 10 * p, 3))
    g = adg.ADG(mech, pick)
    oracles = []
    for k, wl in enumerate(pick):
        prim = wl.primitive(mech)
        g.set_primitive(prim, k)
        o = O.Oracle(wl, mech)
        o.set_primitive(prim)
        oracles.append(o)
    g.step(30)
    g.check()
    for k, o in enumerate(oracles):
        o.step(30)
        err = rel_err(g.get_state(k), o.state(), mech)
        assert err.max() <= TOL, (k, err)
        assert np.array_equal(g.flags(k)[1], o.flags()[1])


def test_state_roundtrip_zero_steps_and_determinism():
    wl = W()["ignition-5sp-200x3"]
    mech = wl.mechanism()
    prim = wl.primitive(mech)
    g = adg.ADG(mech, [wl])
    g.set_primitive(prim)
    w0 = g.get_state()
    g.step(0)
    assert np.array_equal(g.get_state(), w0)
    g.set_state(w0)
    assert np.array_equal(g.get_state(), w0)
    g.step(30)
    a = g.get_state()
    g.set_state(w0)
    g.step(30)
    assert np.array_equal(g.get_state(), a)


def test_all_states_in_one_buffer():
    """adg_write_states / adg_read_states move every instance's state with one
    call, in instance order, and agree with the per-instance calls."""
    import torch
    base = W()["ignition-5sp-200x3"]
    wls = [base, I.scaled(base, 97, 7), I.scaled(base, 64, 4)]
    wls[1].p, wls[1].at_order = 2, 3
    mech = base.mechanism()
    g = adg.ADG(mech, wls)
    for k, w in enumerate(wls):
        g.set_primitive(w.primitive(mech), k)
    g.step(5)
    n = g.states_doubles()
    assert n == sum(g.nv * w.n_elem * (w.p + 1) for w in wls)
    buf = torch.empty(n, dtype=torch.float64, pin_memory=True)
    g.read_states(buf.numpy())
    torch.cuda.synchronize()
    flat = np.concatenate([g.get_state(k).ravel() for k in range(len(wls))])
    assert np.array_equal(buf.numpy(), flat)
    new = torch.from_numpy(flat * 1.0001).pin_memory()
    g.write_states(new.numpy())
    torch.cuda.synchronize()
    got = np.concatenate([g.get_state(k).ravel() for k in range(len(wls))])
    assert np.array_equal(got, new.numpy())
    # pageable host memory takes the per-instance copies
    page = flat * 0.9999
    g.write_states(page)
    torch.cuda.synchronize()
    back = np.zeros(n)
    g.read_states(back)
    torch.cuda.synchronize()
    assert np.array_equal(back, page)
    g.close()


def test_nonphysical_state_is_reported():
    """A state with negative density (made on the host) is reported by
    adg_status as ADG_ERR_NONPHYSICAL; the context stays usable."""
    wl = W()["ignition-5sp-200x3"]
    mech = wl.mechanism()
    g = adg.ADG(mech, [wl])
    g.set_primitive(wl.primitive(mech))
    w = g.get_state()
    bad = w.copy()
    bad[2:, 17, 0] *= -1.0
    g.set_state(bad)
    g.step(1)
    rc, where = g.status()
    assert rc == -4
    assert where[0] == 0
    g.set_state(w)
    g.step(2)
    g.check()


def test_invalid_arguments_raise():
    wl = W()["ignition-5sp-200x3"]
    mech = wl.mechanism()
    g = adg.ADG(mech, [wl])
    with pytest.raises(adg.AdgError):
        g.get_state(k=3)
    with pytest.raises(adg.AdgError):
        g.step(-1)


def test_graph_replay_and_timed_steps_agree():
    """adg_step replays a captured CUDA graph; with kernel timing on it runs a
    graph with event pairs and waits per step. Both give the same state bit for
    bit, and the timing counts every kernel."""
    wl = W()["ignition-5sp-200x3"]
    mech = wl.mechanism()
    g = adg.ADG(mech, [wl])
    g.set_primitive(wl.primitive(mech))
    w0 = g.get_state()
    g.step(12)
    a = g.get_state()
    g.set_state(w0)
    g.enable_kernel_timing(True)
    g.step(12)
    ms, n = g.kernel_times()
    g.enable_kernel_timing(False)
    assert np.array_equal(g.get_state(), a)
    assert n[0] == 36 and n[1] == 36 and n[2] == 12
    assert ms[2] >= ms[0] + ms[1] > 0
    assert g.launches_per_step() == 7


def test_autotune_keeps_the_trajectory():
    """The autotuner times candidate launch configurations of the stage kernel
    (elements per tile, threads per CTA) and keeps the fastest; a configuration
    set by hand takes effect too; the result still matches the oracle."""
    wl = W()["ignition-9sp-4096x4"]
    wl = I.scaled(wl, 1024, 16)
    mech = wl.mechanism()
    CURRENT_MECH[0] = mech
    prim = wl.primitive(mech)
    g = adg.ADG(mech, [wl])
    g.set_primitive(prim)
    g.step(8)
    tun = g.autotune()
    assert tun and tun[0]["elements_per_tile"] >= 2 and tun[0]["threads_per_cta"] >= 64
    assert tun[0]["limiter_elements_per_cta"] in (16, 32)  # the FP64 limiter's sizes
    g.step(8)
    tun = g.set_tuning(0, 3, 96)
    assert tun[0]["elements_per_tile"] == 3 and tun[0]["threads_per_cta"] == 96
    assert tun[0]["tiles"] == (wl.n_elem + 2) // 3
    other = 48 - tun[0]["limiter_elements_per_cta"]  # the other FP64 limiter size
    assert g.set_limiter_tuning(0, other)[0]["limiter_elements_per_cta"] == other
    g.step(8)
    g.check()
    with pytest.raises(adg.AdgError):
        g.set_tuning(0, 3, 100)
    for bad in (8, 12, 64):
        with pytest.raises(adg.AdgError):
            g.set_limiter_tuning(0, bad)
    o = O.Oracle(wl, mech)
    o.set_primitive(prim)
    o.step(24)
    assert_parity(g, o)


def ensemble_sample(ens):
    """The smallest and largest instance and the first of each degree."""
    ks = {min(range(len(ens)), key=lambda k: ens[k].n_elem),
          max(range(len(ens)), key=lambda k: ens[k].n_elem)}
    for p in (2, 3, 4):
        ks.add(next(k for k, w in enumerate(ens) if w.p == p))
    return sorted(ks)


def test_ensemble_512_full_size_sampled():
    """The batched 512-instance ensemble (8.58 M Gauss points, three degree
    groups) in one context, in the autotuned launch configuration the benchmark
    times, 3 steps; sampled instances against the oracle run on them alone."""
    ens = I.ensemble_workloads()
    mech = ens[0].mechanism()
    g = adg.ADG(mech, ens)
    for k, wl in enumerate(ens):
        g.set_primitive(wl.primitive(mech), k)
    g.step(1)
    g.autotune()
    g.step(2)
    g.check()
    for k in ensemble_sample(ens):
        wl = ens[k]
        o = O.Oracle(wl, mech)
        o.set_primitive(wl.primitive(mech))
        o.step(3)
        err = rel_err(g.get_state(k), o.state(), mech)
        assert err.max() <= TOL, (k, err)
        assert np.array_equal(g.flags(k)[1], o.flags()[1]), k
