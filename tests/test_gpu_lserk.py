"""The low-storage explicit RK integrators of Sec. 3.1 on the CUDA path (through
the C ABI) against the FP64 oracle: Williamson's 3-stage third-order scheme and
the 5-stage fourth-order 2N-storage scheme of Carpenter and Kennedy, limiting
after every stage, AT fluxes and AT-WENO at delayed PE faces.

Bars as for SSP-RK3: FP64 relative L-infinity <= 1e-10 in the physical scales of
tests/test_gpu_parity.py with identical troubled-cell flags (every stage of the
last step, and counts over the run); the mixed-precision bar of
tests/test_gpu_mixed.py."""
import dataclasses

import numpy as np
import pytest

import oracle as O
from paper_2501_01747_gb300 import adg
from paper_2501_01747_gb300 import inputs as I
from tests import helpers as H
from tests.test_gpu_mixed import errors as mixed_errors

pytestmark = pytest.mark.gpu

TOL = 1e-10
LSERK = [I.RK_LS3, I.RK_LS4]


def W():
    return I.load_workloads()


def with_rk(wl, integrator, **kw):
    return dataclasses.replace(wl, integrator=integrator, **kw)


def run_both(wl, mech, prim, n_steps, chunks=1, precision="fp64"):
    g = adg.ADG(mech, [wl], precision=precision)
    g.set_primitive(prim)
    o = O.Oracle(wl, mech)
    o.set_primitive(prim)
    for _ in range(chunks):
        g.step(n_steps // chunks)
        o.step(n_steps // chunks)
    g.check()
    return g, o


def assert_parity(g, o, mech, k=0):
    w, ref = g.get_state(k), o.state()
    assert np.all(np.isfinite(w))
    err = H.parity_error(w, ref, mech)
    assert err.max() <= TOL, err
    gl, gc = g.flags(k)
    ol, oc = o.flags()
    assert gl.shape == ol.shape
    assert np.array_equal(gc, oc), np.flatnonzero(gc != oc)[:10]
    assert np.array_equal(gl, ol)


@pytest.mark.parametrize("integrator", LSERK)
def test_ignition_5sp(integrator):
    """200 x p3, 4 PEs, SAA delays up to 2, AT order 4, WENO, 90 steps in three
    calls."""
    wl = with_rk(W()["ignition-5sp-200x3"], integrator)
    mech = wl.mechanism()
    g, o = run_both(wl, mech, wl.primitive(mech), 90, chunks=3)
    assert_parity(g, o, mech)


@pytest.mark.parametrize("mode", [I.DELAY_CAA, I.DELAY_SAA])
def test_detonation_hllc_walls_lserk4(mode):
    """The 9-species detonation shape (reflecting wall, outflow, HLLC, WENO with
    troubled cells at the front, PE faces across the front) on 384 elements x p3
    and 48 PEs, LSERK4, 40 steps of dt/8. LSERK4 is not strong-stability
    preserving: near the front its intermediate stages make the result far more
    sensitive to rounding than SSP-RK3's, and every limiter decision at the front
    adds to that. With the indicator's rounding guard at 1e-10 the oracle itself
    moves by 1.5e-10 (CAA) and 8.6e-11 (SAA) at dt/4 when its input moves by
    1e-15, at the bar; at dt/8 by 7e-12, below it, as the SSP-RK3 detonation
    tests run at dt/20."""
    base = W()["detonation-9sp-16384x3"]
    wl = with_rk(I.scaled(base, 384, 48), I.RK_LS4, delay_mode=mode)
    wl.dt = base.dt * 0.125
    mech = wl.mechanism()
    g, o = run_both(wl, mech, wl.primitive(mech), 40, chunks=2)
    assert o.flags()[1].sum() > 0  # the limiter acts
    assert_parity(g, o, mech)


@pytest.mark.parametrize("p", [1, 2, 4])
def test_every_degree_ragged_lserk4(p):
    base = W()["ignition-9sp-4096x4"]
    wl = with_rk(I.scaled(base, 97, 7), I.RK_LS4, p=p, at_order=p + 1)
    mech = wl.mechanism()
    g, o = run_both(wl, mech, wl.primitive(mech), 30)
    assert_parity(g, o, mech)


def test_full_size_9sp_lserk4():
    """4096 x p4, 21 reactions, 64 PEs, SAA delays up to 4, AT order 5: 6 steps."""
    wl = with_rk(W()["ignition-9sp-4096x4"], I.RK_LS4)
    mech = wl.mechanism()
    g, o = run_both(wl, mech, wl.primitive(mech), 6)
    assert_parity(g, o, mech)


def test_three_integrators_in_one_context():
    """SSP-RK3, LSERK3 and LSERK4 instances of one problem in one context: two
    groups (3 and 5 stages) in one step graph, each instance at the FP64 bar."""
    base = W()["ignition-5sp-200x3"]
    wls = [with_rk(base, r) for r in (I.RK_SSP3, I.RK_LS3, I.RK_LS4)]
    mech = base.mechanism()
    prim = base.primitive(mech)
    g = adg.ADG(mech, wls)
    for k in range(3):
        g.set_primitive(prim, k)
    g.step(30)
    g.check()
    assert sorted(t["stages"] for t in g.tuning()) == [3, 5]
    assert g.launches_per_step() == 1 + 2 * 3 + 2 * 5
    for k, wl in enumerate(wls):
        o = O.Oracle(wl, mech)
        o.set_primitive(prim)
        o.step(30)
        assert_parity(g, o, mech, k)


def test_mixed_lserk4():
    """The mixed-precision variant with LSERK4 on the 5-species workload, 200
    steps: the mixed bar (T and Y within 1e-4). By step 300 the oracle's own
    response to a 1e-7 change of its input exceeds the bar (the limiter's
    decisions under the non-SSP integrator; tests/test_oracle_conditioning.py),
    so the bar is checked where it still tests the arithmetic."""
    wl = with_rk(W()["ignition-5sp-200x3"], I.RK_LS4)
    mech = wl.mechanism()
    g, o = run_both(wl, mech, wl.primitive(mech), 200, chunks=2, precision="mixed")
    eT, eY = mixed_errors(g, o, wl)
    assert eT <= 1e-4 and eY <= 1e-4, (eT, eY)


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_unsync_without_delay_equals_sync_lserk4(precision):
    wl = with_rk(W()["ignition-5sp-200x3"], I.RK_LS4, max_delay=0, delay_probs=(1.0,))
    mech = wl.mechanism()
    prim = wl.primitive(mech)
    a = adg.ADG(mech, [wl], precision=precision)
    b = adg.ADG(mech, [wl], precision=precision)
    a.set_primitive(prim)
    b.set_primitive(prim)
    a.step(20)
    b.step_unsync(20)
    a.check()
    b.check()
    assert np.array_equal(a.get_state(), b.get_state())
    assert np.array_equal(a.flags()[0], b.flags()[0])
    h = b.unsync_delays()
    assert h[0, 0] == 20 * 5 * 2 * wl.n_pe


def test_noalloc_rejects_lserk():
    import torch
    wl = with_rk(W()["ignition-5sp-200x3"], I.RK_LS4)
    mech = wl.mechanism()
    w = torch.zeros((mech.ns + 2, wl.n_elem, wl.p + 1), dtype=torch.float64, device="cuda")
    with pytest.raises(adg.AdgError) as ex:
        adg.step_noalloc(mech, wl, w, w, 1)
    assert ex.value.code == -1
