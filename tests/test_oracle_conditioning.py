"""Conditioning of the scheme, measured on the oracle: the state after a run moves
by less than 1e-11, in the physical scales of the parity tests, when the initial
state moves by 1e-15 relative. This is what makes a 1e-10 bar between two FP64
implementations meaningful (and why the scales are not each variable's own
maximum, which moves by up to 1e-6 for momentum at rest and for trace species)."""
import numpy as np
import pytest

import oracle as O
from paper_2501_01747_gb300 import inputs as I
from tests import helpers as H


def _cases():
    W = I.load_workloads()
    base = W["detonation-9sp-16384x3"]
    out = []
    for p in (2, 4):
        wl = I.scaled(base, 97, 7)
        wl.p, wl.at_order, wl.dt = p, p + 1, base.dt * 0.05
        out.append(("shock-p%d" % p, wl, 60))
    out.append(("ignition-5sp", W["ignition-5sp-200x3"], 300))
    wl = I.scaled(W["ignition-9sp-4096x4"], 256, 4)
    out.append(("ignition-9sp-256", wl, 12))
    return out


@pytest.mark.parametrize("name,wl,n", _cases(), ids=lambda x: x if isinstance(x, str) else "")
def test_perturbation_response_below_parity_bar(name, wl, n):
    mech = wl.mechanism()
    a = O.Oracle(wl, mech)
    a.set_primitive(wl.primitive(mech))
    w0 = a.state()
    a.step(n)
    worst = 0.0
    own = 0.0
    for seed in range(2):
        b = O.Oracle(wl, mech)
        b.set_state(w0 * (1 + 1e-15 * np.random.default_rng(seed).standard_normal(w0.shape)))
        b.step(n)
        worst = max(worst, float(H.parity_error(b.state(), a.state(), mech).max()))
        d = np.abs(b.state() - a.state()).max(axis=(1, 2)) / np.abs(a.state()).max(axis=(1, 2))
        own = max(own, float(d.max()))
    assert worst < 1e-11, worst
    # each variable's own maximum would be a much less stable yardstick
    assert own > 10 * worst


def _ignition_shape(limiter=I.LIM_WENO):
    """The 9-species premixed ignition shape on 64 elements x p4 over 1/8 of the
    length (as the mixed-precision ignition test), limiter on or off."""
    base = I.load_workloads()["ignition-9sp-4096x4"]
    wl = I.scaled(base, 64, 4)
    wl.length = base.length / 8
    wl.dt = base.dt * (wl.length / wl.n_elem) / (base.length / base.n_elem)
    wl.limiter = limiter
    return wl


def _mass_fractions(w, p):
    x, _ = np.polynomial.legendre.leggauss(p + 1)
    V = np.polynomial.legendre.legvander(x, p)
    r = np.einsum("inj,qj->inq", w[2:], V)
    return r / r.sum(axis=0, keepdims=True)


def _response(wl, eps, checkpoints):
    """The mixed-precision bar's two errors (T relative at every Gauss point; Y
    relative to each species' largest value where Y > 1e-8) between the oracle's
    run and its run from the initial state moved by eps relative, at each
    checkpoint (steps)."""
    mech = wl.mechanism()
    a = O.Oracle(wl, mech)
    a.set_primitive(wl.primitive(mech))
    w0 = a.state()
    b = O.Oracle(wl, mech)
    b.set_state(w0 * (1 + eps * np.random.default_rng(5).standard_normal(w0.shape)))
    out, done = [], 0
    for n in checkpoints:
        a.step(n - done)
        b.step(n - done)
        done = n
        Ta, Tb = a.temperature(), b.temperature()
        eT = float((np.abs(Tb - Ta) / Ta).max())
        Ya, Yb = _mass_fractions(a.state(), wl.p), _mass_fractions(b.state(), wl.p)
        eY = 0.0
        for i in range(Ya.shape[0]):
            big = Ya[i] > 1e-8
            if big.any():
                eY = max(eY, float(np.abs(Yb[i] - Ya[i])[big].max() / Ya[i].max()))
        out.append(max(eT, eY))
    return out


def _lserk4_5sp():
    import dataclasses
    return dataclasses.replace(I.load_workloads()["ignition-5sp-200x3"], integrator=I.RK_LS4)


HORIZONS = [
    # (case, workload factory, horizon of the mixed bar, a later checkpoint)
    ("ignition-9sp-64x4", _ignition_shape, 200, 250),
    ("ignition-5sp-lserk4", _lserk4_5sp, 200, 300),
    ("ignition-9sp-4096x4", lambda: I.load_workloads()["ignition-9sp-4096x4"], 48, 100),
]


@pytest.mark.parametrize("name,make,horizon,later", HORIZONS,
                         ids=[h[0] for h in HORIZONS])
def test_mixed_bar_horizon(name, make, horizon, later):
    """Where the mixed-precision bar (1e-4 on T and Y) is meaningful. The
    paper's indicator is a TVD test without a threshold: the limiter flags the
    smooth extrema whose face deviations exceed the rounding guard, and its
    decisions, with the WENO reconstruction of those cells in characteristic
    variables, make the limited scheme respond to a small change of the state
    far more than the scheme without the limiter (ignition shape: about 1e6
    through ignition, 4 without the limiter). A run in single precision differs
    from the FP64 one by about one single-precision rounding of the state, 1e-7
    relative. Up to `horizon` steps the oracle's own response to a 1e-7
    perturbation of its input stays below the bar, so the bar is a test of the
    mixed arithmetic there; by `later` steps the response alone exceeds it, and
    the bar no longer separates a good run from a bad one."""
    r = _response(make(), 1e-7, [horizon, later])
    assert r[0] < 1e-4, r
    assert r[1] > 1e-4, r


def test_run_through_ignition_without_limiter_is_well_conditioned():
    """The same ignition run without the limiter: a perturbation of 1e-8 of the
    input moves T and Y by less than 100 times that through ignition (520
    steps), so the amplification above comes from the limiter's decisions."""
    r = _response(_ignition_shape(I.LIM_NONE), 1e-8, [520])
    assert r[0] < 1e-6, r
