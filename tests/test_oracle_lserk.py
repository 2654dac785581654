"""Pins of the oracle's low-storage explicit Runge-Kutta integrators (Sec. 3.1
cites Williamson 1980 and Kennedy, Carpenter & Lewis 2000): Williamson's 3-stage
third-order scheme and the 5-stage fourth-order 2N-storage scheme of Carpenter and
Kennedy, both in the 2N form dq <- A_s dq + dt L(w), w <- w + B_s dq.

* The 2N coefficients, turned into a Butcher tableau, satisfy every order
  condition of their order (4 conditions for order 3, 8 for order 4) and give the
  published stage times C_s.
* In the full scheme (a smooth entropy wave of an inert mixture, fixed mesh) the
  temporal error falls as dt^3 and dt^4 respectively, and SSP-RK3 as dt^3.
* With CAA delays at the PE faces and LSERK4 the AT flux keeps the asynchrony
  error far below that of the plain delayed flux (AT order 1)."""
import numpy as np
import pytest

import oracle as O
from paper_2501_01747_gb300 import inputs as I
from tests import helpers as H

RU = 8.314462618


def butcher(A, B):
    """Butcher tableau (a, b, c) of a 2N-storage scheme: with Y_0 = y_n,
    dq_s = A_s dq_{s-1} + h f(Y_s) and Y_{s+1} = Y_s + B_s dq_s, the weight of
    f(Y_j) in Y_s is sum_{l=j}^{s-1} B_l prod_{i=j+1}^{l} A_i."""
    S = len(A)

    def weight(j, upto):
        tot = 0.0
        for l in range(j, upto):
            pr = 1.0
            for i in range(j + 1, l + 1):
                pr *= A[i]
            tot += B[l] * pr
        return tot

    a = np.array([[weight(j, s) if j < s else 0.0 for j in range(S)] for s in range(S)])
    b = np.array([weight(j, S) for j in range(S)])
    return a, b, a.sum(axis=1)


@pytest.mark.parametrize("integrator, order", [(I.RK_LS3, 3), (I.RK_LS4, 4)])
def test_order_conditions(integrator, order):
    A, B, C = O.lserk_coeffs(integrator)
    assert len(A) == O.rk_stages(integrator) and A[0] == 0.0
    a, b, c = butcher(A, B)
    assert np.allclose(c, C, rtol=0, atol=1e-15)
    conds = [(b.sum(), 1.0), (b @ c, 1 / 2), (b @ c**2, 1 / 3), (b @ a @ c, 1 / 6)]
    if order >= 4:
        conds += [(b @ c**3, 1 / 4), (b @ (c * (a @ c)), 1 / 8), (b @ a @ c**2, 1 / 12),
                  (b @ a @ a @ c, 1 / 24)]
    for got, want in conds:
        assert abs(got - want) <= 1e-14, (got, want)
    # and not of the next order (the bushy-tree condition b.c^order = 1/(order+1)
    # fails): the schemes are exactly of their stated order
    assert abs(b @ c**order - 1 / (order + 1)) > 1e-5


def _wave(integrator, n, t_end=3e-3):
    mech = H.inert_mechanism()
    wl = H.workload(16, 3, n_pe=1, dt=t_end / n)
    wl.integrator = integrator
    prim = H.two_species_ic(wl, mech, lambda x: 1.0 + 0.3 * np.sin(6 * np.pi * x), 50.0, 1e5)
    o = O.Oracle(wl, mech)
    o.set_primitive(prim)
    o.step(n)
    return o.state()


@pytest.mark.parametrize("integrator, order", [(I.RK_SSP3, 3), (I.RK_LS3, 3), (I.RK_LS4, 4)])
def test_temporal_order_in_the_full_scheme(integrator, order):
    """Entropy wave, 16 elements x p3, dt from CFL 0.6/(2p+1) down by 2 and 4,
    against dt/16 on the same mesh."""
    a0 = np.sqrt(29.1 / (29.1 - RU) * RU * 350.0 / 0.029)
    n0 = int(np.ceil(3e-3 / (0.6 / 16 / (7 * (50.0 + 1.2 * a0)))))
    ref = _wave(integrator, 16 * n0)
    errs = [np.abs(_wave(integrator, m * n0) - ref).max() / np.abs(ref).max() for m in (1, 2, 4)]
    rates = [np.log2(errs[i] / errs[i + 1]) for i in range(2)]
    assert all(order - 0.25 <= r <= order + 0.4 for r in rates), (errs, rates)


def test_steps_in_chunks_equal_one_call():
    wl = H.workload(16, 3, n_pe=4, dt=2e-7, delay_mode=I.DELAY_SAA, max_delay=2)
    wl.integrator = I.RK_LS4
    mech = H.inert_mechanism()
    prim = H.two_species_ic(wl, mech, lambda x: 1.0 + 0.3 * np.sin(2 * np.pi * x), 50.0, 1e5)
    a, b = O.Oracle(wl, mech), O.Oracle(wl, mech)
    a.set_primitive(prim)
    b.set_primitive(prim)
    a.step(30)
    for _ in range(3):
        b.step(10)
    assert np.array_equal(a.state(), b.state())
    assert a.flags()[0].shape == (5, 16)


def test_at_flux_pays_off_with_lserk4():
    """CAA with delays up to 2 on 8 PEs (32 x p3): the deviation from the synchronous LSERK4
    run with the AT flux (order 4) is far below that with the plain delayed flux
    (AT order 1)."""
    mech = H.inert_mechanism()
    n, t_end = 3200, 2e-3  # AT extrapolation of order 4 narrows the stable CFL
    prim = None
    out = {}
    for mode, o_at in ((I.DELAY_SYNC, 4), (I.DELAY_CAA, 4), (I.DELAY_CAA, 1)):
        wl = H.workload(32, 3, n_pe=8, dt=t_end / n, delay_mode=mode, max_delay=2,
                        at_order=o_at)
        wl.integrator = I.RK_LS4
        if prim is None:
            prim = H.two_species_ic(wl, mech, lambda x: 1.0 + 0.2 * np.sin(2 * np.pi * x),
                                    50.0, 1e5)
        o = O.Oracle(wl, mech)
        o.set_primitive(prim)
        o.step(n)
        out[(mode, o_at)] = o.state()
    ref = out[(I.DELAY_SYNC, 4)]
    e4 = np.abs(out[(I.DELAY_CAA, 4)] - ref).max() / np.abs(ref).max()
    e1 = np.abs(out[(I.DELAY_CAA, 1)] - ref).max() / np.abs(ref).max()
    assert 0 < e4 < 0.01 * e1, (e4, e1)
