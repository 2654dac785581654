"""Pins of the oracle's full ADG scheme: exact reductions, invariants, design
order on a smooth problem, the error law in P, and a textbook shock tube."""
import numpy as np
import pytest

import oracle as O
from paper_2501_01747_gb300 import inputs as I
from tests import helpers as H

RU = 8.314462618


def _run(wl, mech, prim, n):
    o = O.Oracle(wl, mech)
    o.set_primitive(prim)
    o.step(n)
    return o


def _c1(**kw):
    wl = I.load_workloads()["ignition-5sp-200x3"]
    for k, v in kw.items():
        setattr(wl, k, v)
    return wl


def test_zero_delays_reduce_exactly_to_synchronous():
    """SAA whose probability set puts all mass on delay 0 is bit-for-bit the
    synchronous algorithm (the AT weights at k = 0 are (1, 0, .., 0))."""
    wl_s = _c1(delay_mode=I.DELAY_SYNC)
    wl_a = _c1(delay_mode=I.DELAY_SAA, delay_probs=(1.0, 0.0, 0.0))
    mech = wl_s.mechanism()
    prim = wl_s.primitive(mech)
    a = _run(wl_s, mech, prim, 40)
    b = _run(wl_a, mech, prim, 40)
    assert np.array_equal(a.state(), b.state())
    assert np.array_equal(a.flags()[1], b.flags()[1])
    c = _run(_c1(delay_mode=I.DELAY_CAA), mech, prim, 40)
    assert not np.array_equal(a.state(), c.state())


@pytest.mark.parametrize("mode", [I.DELAY_SYNC, I.DELAY_CAA, I.DELAY_SAA])
def test_conservation_with_delays_and_limiter(mode):
    """Periodic domain: total mass, momentum and energy are constant to round-off
    in every algorithm (common delayed level at PE faces, average-preserving
    limiter, mass-conserving chemistry)."""
    wl = _c1(delay_mode=mode)
    mech = wl.mechanism()
    prim = wl.primitive(mech)
    prim[0, 60:90] = 1500.0   # a hot slab with sharp edges, so that WENO acts
    o = O.Oracle(wl, mech)
    o.set_primitive(prim)
    w0 = o.state()
    o.step(80)
    w = o.state()
    assert o.flags()[1].sum() > 0  # the limiter did act
    mass0, mass = w0[2:, :, 0].sum(), w[2:, :, 0].sum()
    assert abs(mass - mass0) <= 1e-14 * mass0 * 10
    E0, E = w0[1, :, 0].sum(), w[1, :, 0].sum()
    assert abs(E - E0) <= 1e-13 * abs(E0)
    rho = w0[2:, :, 0].sum(0)
    mom_scale = np.sum(rho * 700.0)
    assert abs(w[0, :, 0].sum() - w0[0, :, 0].sum()) <= 1e-13 * mom_scale


def test_uniform_state_matches_reactor():
    """A spatially uniform mixture evolves like the 0D constant-volume reactor:
    fluxes cancel and only the projected source acts."""
    wl = _c1(n_elem=8, n_pe=2, p=2, at_order=3, delay_mode=I.DELAY_SAA, limiter=I.LIM_WENO)
    mech = wl.mechanism()
    Y = I.composition(mech, 0.02)
    prim = np.zeros((mech.ns + 3, 8, 3))
    prim[0] = 1400.0
    prim[1] = I.P_ATM
    prim[3:] = Y[:, None, None]
    o = _run(wl, mech, prim, 60)
    w = o.state()
    w0 = O.cons_from_prim(mech, 1400.0, I.P_ATM, 0.0, Y)
    r = O.reactor0d(mech, w0[2:].copy(), w0[1], wl.dt, 60)
    assert not np.allclose(r, w0[2:], rtol=1e-6)
    for e in range(8):
        assert np.allclose(w[2:, e, 0], r, rtol=1e-11, atol=1e-14 * r.sum())
    assert np.abs(w[:, :, 1:]).max() <= 1e-9
    assert o.flags()[1].sum() == 0


def _advection_error(n_elem, p, mode=I.DELAY_SYNC, at_order=None, n_pe=4, max_delay=2,
                     cfl=0.2, t_end=2e-3, ref=None):
    mech = H.inert_mechanism()
    u0, P0 = 50.0, 1e5
    a0 = np.sqrt(29.1 / (29.1 - RU) * RU * 300.0 / 0.029)
    dx = 1.0 / n_elem
    n = int(np.ceil(t_end / (cfl * dx / ((2 * p + 1) * (u0 + a0 * 1.2)))))
    dt = t_end / n
    wl = H.workload(n_elem, p, n_pe=n_pe, dt=dt, delay_mode=mode, max_delay=max_delay,
                    at_order=at_order)
    rho_fn = lambda x: 1.0 + 0.2 * np.sin(2 * np.pi * x)
    prim = H.two_species_ic(wl, mech, rho_fn, u0, P0)
    o = _run(wl, mech, prim, n)
    rho = H.modal_to_nodal(o.state()[2:].sum(0), p)
    if ref is not None:
        return H.gauss_l2(wl, rho, ref)
    exact = rho_fn(wl.nodes_x() - u0 * t_end)
    return H.gauss_l2(wl, rho, exact), rho


def _order(errs, ns):
    return np.polyfit(np.log(ns), np.log(errs), 1)[0] * -1


@pytest.mark.parametrize("p", [1, 2])
def test_design_order_synchronous(p):
    ns = [32, 64, 128]
    errs = [_advection_error(n, p)[0] for n in ns]
    assert _order(errs, ns) > p + 1 - 0.35


@pytest.mark.parametrize("p,ns", [(3, [16, 32, 64]), (4, [32, 64, 128])])
def test_design_order_synchronous_high_degree(p, ns):
    """Design order p+1 of the DG operator (Sec. 3.1) at p = 3 and 4. SSP-RK3's
    O(dt^3) error would hide it at a fixed CFL number, so dt shrinks like
    dx^((p+1)/3) and both errors fall at the rate of dx^(p+1)."""
    errs = [_advection_error(n, p, cfl=0.2 * (ns[0] / n) ** ((p + 1) / 3.0 - 1.0))[0]
            for n in ns]
    assert _order(errs, ns) > p + 1 - 0.35


@pytest.mark.parametrize("p", [1, 2])
def test_at_fluxes_keep_the_asynchrony_error_high_order(p):
    """Sec. 3.2: with AT order o = p+1 the deviation from the synchronous solution
    caused by the delays (CAA, up to 2 steps, 8 PEs) falls like dt^o / N_E, i.e.
    with order about p+2 in N_E at fixed CFL; a plain delayed flux (o = 1) only
    falls like dt / N_E and is orders of magnitude larger."""
    ns = [32, 64, 128]
    ea, e1 = [], []
    for n in ns:
        _, ref = _advection_error(n, p, n_pe=1, cfl=0.1)
        ea.append(_advection_error(n, p, mode=I.DELAY_CAA, n_pe=8, cfl=0.1, ref=ref))
        e1.append(_advection_error(n, p, mode=I.DELAY_CAA, n_pe=8, cfl=0.1, at_order=1,
                                   ref=ref))
    assert _order(ea, ns) > p + 1.5
    assert _order(e1, ns) < 2.0
    assert e1[-1] > 100 * ea[-1]


def test_error_grows_linearly_with_pe_count():
    """Sec. 5.1: the ADG error relative to the synchronous solution grows like P."""
    n_elem, p = 64, 1
    _, ref = _advection_error(n_elem, p, n_pe=1)
    Ps = [2, 4, 8, 16]
    errs = [_advection_error(n_elem, p, mode=I.DELAY_CAA, n_pe=P, ref=ref) for P in Ps]
    slope = np.polyfit(np.log(Ps), np.log(errs), 1)[0]
    assert 0.7 < slope < 1.3


@pytest.mark.parametrize("p", [1, 2])
def test_sod_shock_tube_against_exact_riemann(p):
    """Single-gas Sod problem with HLLC and the WENO limiter against the exact
    Riemann solution; L1 error of density shrinks with the mesh."""
    mech = H.inert_mechanism()
    g = 29.1 / (29.1 - RU)
    rl, pl, rr, pr = 1.0, 1e5, 0.125, 1e4
    t_end = 5e-4
    errs = []
    for n_elem in (100, 200):
        dx = 1.0 / n_elem
        n = int(np.ceil(t_end / (0.1 * dx / ((2 * p + 1) * 800.0))))
        wl = H.workload(n_elem, p, n_pe=4, dt=t_end / n, bc=(I.BC_OUTFLOW, I.BC_OUTFLOW),
                        flux=I.FLUX_HLLC, limiter=I.LIM_WENO, delay_mode=I.DELAY_SYNC)
        x = wl.nodes_x()
        rho0 = np.where(x < 0.5, rl, rr)
        P0 = np.where(x < 0.5, pl, pr)
        prim = np.zeros((mech.ns + 3,) + x.shape)
        prim[0] = P0 * 0.029 / (rho0 * RU)
        prim[1] = P0
        prim[3:] = 0.5
        o = _run(wl, mech, prim, n)
        rho = H.modal_to_nodal(o.state()[2:].sum(0), p)
        ex = H.exact_riemann(rl, 0.0, pl, rr, 0.0, pr, g, (x - 0.5) / t_end)[0]
        _, w = np.polynomial.legendre.leggauss(p + 1)
        errs.append(float(np.sum(np.abs(rho - ex) * w[None, :] * 0.5 * dx)))
        assert o.flags()[1].sum() > 0
    assert errs[0] < 0.02
    assert errs[1] < 0.75 * errs[0]


def test_limiter_leaves_linear_and_uniform_data_alone():
    mech = H.inert_mechanism()
    wl = H.workload(32, 2, n_pe=4, dt=1e-9, bc=(I.BC_OUTFLOW, I.BC_OUTFLOW),
                    limiter=I.LIM_WENO, delay_mode=I.DELAY_SAA, max_delay=2)
    # linear density at uniform pressure and velocity
    prim = H.two_species_ic(wl, mech, lambda x: 1.0 + 0.5 * x, 10.0, 1e5)
    o = _run(wl, mech, prim, 1)
    last, _ = o.flags()
    assert last[:, 1:-1].sum() == 0
    # uniform reacting mixture
    wl2 = _c1(n_elem=16, n_pe=4)
    m2 = wl2.mechanism()
    prim2 = np.zeros((m2.ns + 3, 16, 4))
    prim2[0] = 1300.0
    prim2[1] = I.P_ATM
    prim2[3:] = I.composition(m2, 0.02)[:, None, None]
    o2 = _run(wl2, m2, prim2, 30)
    assert o2.flags()[1].sum() == 0


def test_wall_and_outflow_keep_a_resting_gas_at_rest():
    mech = H.inert_mechanism()
    wl = H.workload(16, 2, n_pe=2, dt=1e-6, bc=(I.BC_REFLECT, I.BC_OUTFLOW),
                    flux=I.FLUX_HLLC, limiter=I.LIM_WENO)
    prim = H.two_species_ic(wl, mech, lambda x: np.full_like(x, 1.2), 0.0, 1e5)
    o = O.Oracle(wl, mech)
    o.set_primitive(prim)
    w0 = o.state()
    o.step(20)
    assert np.allclose(o.state(), w0, rtol=0, atol=1e-9 * np.abs(w0).max())


@pytest.mark.parametrize("mode", [I.DELAY_CAA, I.DELAY_SAA])
def test_at_weno_shock_tube_agrees_with_synchronous(mode):
    """Sec. 5.2 / Table 2: with AT fluxes and AT-WENO limiting at the PE faces, a
    shock computed with delays (12 PEs, delays up to 2) is as accurate as the
    synchronous one: its L1 error against the exact solution is no larger (within
    10 %), its deviation from the synchronous run is a fraction of that error, and
    on the plateaus behind the shock and the contact its mean is much closer to
    the synchronous mean than that is to the exact state. Limiter decisions near
    the shock differ between the two runs, so the deviation is a fraction of the
    discretisation error, not round-off."""
    mech = H.inert_mechanism()
    g = 29.1 / (29.1 - RU)
    rl, pl, rr, pr = 1.0, 1e5, 0.125, 1e4
    p, n_elem, t_end = 2, 120, 5e-4
    dx = 1.0 / n_elem
    n = int(np.ceil(t_end / (0.05 * dx / ((2 * p + 1) * 800.0))))
    out = {}
    for m in (I.DELAY_SYNC, mode):
        wl = H.workload(n_elem, p, n_pe=12, dt=t_end / n, bc=(I.BC_OUTFLOW, I.BC_OUTFLOW),
                        flux=I.FLUX_HLLC, limiter=I.LIM_WENO, delay_mode=m, max_delay=2,
                        probs=I.SAA_SETS[1])
        x = wl.nodes_x()
        rho0 = np.where(x < 0.5, rl, rr)
        P0 = np.where(x < 0.5, pl, pr)
        prim = np.zeros((mech.ns + 3,) + x.shape)
        prim[0] = P0 * 0.029 / (rho0 * RU)
        prim[1] = P0
        prim[3:] = 0.5
        o = _run(wl, mech, prim, n)
        out[m] = H.modal_to_nodal(o.state()[2:].sum(0), p)
    ex = H.exact_riemann(rl, 0.0, pl, rr, 0.0, pr, g, (x - 0.5) / t_end)[0]
    _, w = np.polynomial.legendre.leggauss(p + 1)
    l1 = lambda a, b: float(np.sum(np.abs(a - b) * w[None, :] * 0.5 * dx))
    e_exact = l1(out[I.DELAY_SYNC], ex)
    e_async = l1(out[mode], out[I.DELAY_SYNC])
    assert 0 < e_async < 0.35 * e_exact
    assert l1(out[mode], ex) <= 1.1 * e_exact
    # plateaus behind the shock and behind the contact: the delayed run is much
    # closer to the synchronous one than the synchronous one is to the exact state
    for lo, hi in [(0.62, 0.72), (0.52, 0.58)]:
        msk = (x > lo) & (x < hi)
        s, a, e = out[I.DELAY_SYNC][msk].mean(), out[mode][msk].mean(), ex[msk].mean()
        assert abs(a - s) < 0.25 * abs(s - e)
