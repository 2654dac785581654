"""The viscous terms (Sec. 2 diffusive flux, Sec. 3.1 local DG) on the CUDA path
(through the C ABI) against the FP64 oracle, which tests/test_oracle_viscous.py
pins to the primitive-variable definition, binary diffusion and Stokes-Kirchhoff
attenuation. Bars as for the Euler terms: FP64 relative L-infinity <= 1e-10 in the
physical scales of tests/test_gpu_parity.py with identical troubled-cell flags;
the mixed-precision bar of tests/test_gpu_mixed.py. Every case here was checked
with the oracle to move by less than 4e-12 when its input moves by 1e-15."""
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


def W():
    return I.load_workloads()


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
    assert np.array_equal(gc, oc), np.flatnonzero(gc != oc)[:10]
    assert np.array_equal(gl, ol)


@pytest.mark.parametrize("integrator", [I.RK_SSP3, I.RK_LS4])
def test_viscous_ignition_5sp(integrator):
    """200 x p3, 4 PEs, SAA delays up to 2 with AT order 4 (AT flux and AT mean of
    w for q at the PE faces), WENO, 60 steps in three calls."""
    wl = I.viscous(W()["ignition-5sp-200x3"], integrator=integrator)
    mech = wl.mechanism()
    g, o = run_both(wl, mech, wl.primitive(mech), 60, chunks=3)
    assert_parity(g, o, mech)
    # the viscous terms act: the Euler run differs
    e = adg.ADG(mech, [dataclasses.replace(wl, viscous=0)])
    e.set_primitive(wl.primitive(mech))
    e.step(60)
    assert H.parity_error(e.get_state(), o.state(), mech).max() > 1e-9


@pytest.mark.parametrize("p", [1, 2, 3, 4])
def test_viscous_every_degree_ragged(p):
    """97 elements x p (ragged last tile), 7 PEs, the 9-species ignition shape."""
    wl = I.viscous(I.scaled(W()["ignition-9sp-4096x4"], 97, 7), p=p, at_order=p + 1)
    mech = wl.mechanism()
    g, o = run_both(wl, mech, wl.primitive(mech), 30)
    assert_parity(g, o, mech)


def test_viscous_detonation_walls():
    """Reflecting wall and outflow (mirror and copy ghosts for w and q), HLLC, WENO
    with troubled cells, 97 x p3, 7 PEs, 60 steps of dt/20."""
    base = W()["detonation-9sp-16384x3"]
    wl = I.viscous(I.scaled(base, 97, 7))
    wl.dt = base.dt * 0.05
    mech = wl.mechanism()
    g, o = run_both(wl, mech, wl.primitive(mech), 60)
    assert o.flags()[1].sum() > 0
    assert_parity(g, o, mech)


def test_viscous_full_size_9sp():
    """4096 x p4, 21 reactions, 64 PEs, SAA delays up to 4, AT order 5, dt/8: 4 steps."""
    wl = I.viscous(W()["ignition-9sp-4096x4"])
    mech = wl.mechanism()
    g, o = run_both(wl, mech, wl.primitive(mech), 4)
    assert_parity(g, o, mech)


def test_strong_diffusion_binary_mixture():
    """The binary-diffusion pin of the oracle (two identical molecules, uniform T
    and P, a sine of Y_1; 16 x p3, mu = 8e-4 Pa s): the GPU at the FP64 bar."""
    mech = H.inert_mechanism()
    L, p, ne = 0.01, 3, 16
    wl = I.viscous(H.workload(ne, p, n_pe=4, length=L, dt=2e-8), mu_ref=8e-4, T_mu=300.0)
    x = wl.nodes_x()
    prim = np.zeros((mech.ns + 3,) + x.shape)
    prim[0], prim[1] = 300.0, 1e5
    prim[3] = 0.5 + 0.1 * np.sin(2 * np.pi * x / L)
    prim[4] = 1 - prim[3]
    g, o = run_both(wl, mech, prim, 200)
    assert_parity(g, o, mech)


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_viscous_and_euler_instances_in_one_context(precision):
    """A viscous and an Euler instance of one problem in one group: the viscous
    stage kernel skips the terms for the Euler instance."""
    base = W()["ignition-5sp-200x3"]
    wls = [I.viscous(base), base]
    mech = base.mechanism()
    prim = base.primitive(mech)
    g = adg.ADG(mech, wls, precision=precision)
    for k in range(2):
        g.set_primitive(prim, k)
    g.step(30)
    g.check()
    for k, wl in enumerate(wls):
        o = O.Oracle(wl, mech)
        o.set_primitive(prim)
        o.step(30)
        if precision == "fp64":
            assert_parity(g, o, mech, k)
        else:
            T, To = g.temperature(k), o.temperature()
            assert float((np.abs(T - To) / To).max()) <= 1e-4


def test_viscous_mixed_precision():
    """The mixed variant (viscous terms in FP64, subtracted in FP32) on the
    5-species workload over 300 steps: the mixed bar."""
    wl = I.viscous(W()["ignition-5sp-200x3"])
    mech = wl.mechanism()
    g, o = run_both(wl, mech, wl.primitive(mech), 300, chunks=3, precision="mixed")
    eT, eY = mixed_errors(g, o, wl)
    assert eT <= 1e-4 and eY <= 1e-4, (eT, eY)


def test_viscous_rejected_by_unsync_and_noalloc():
    import torch
    wl = I.viscous(W()["ignition-5sp-200x3"])
    mech = wl.mechanism()
    g = adg.ADG(mech, [wl])
    g.set_primitive(wl.primitive(mech))
    with pytest.raises(adg.AdgError) as ex:
        g.step_unsync(1)
    assert ex.value.code == -1
    w = torch.zeros((mech.ns + 2, wl.n_elem, wl.p + 1), dtype=torch.float64, device="cuda")
    with pytest.raises(adg.AdgError) as ex:
        adg.step_noalloc(mech, wl, w, w, 1)
    assert ex.value.code == -1
