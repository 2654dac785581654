"""Pins of the oracle's viscous terms (Sec. 2: the diffusive flux f^d with the
shear stress, the heat flux and mixture-averaged species diffusion; Sec. 3.1: the
local DG method with q = dw/dx from a central flux of w).

* Pointwise: f^d(w, q) from the conserved state and its derivative equals the
  definition written in primitive variables (tau = 4/3 mu u_x,
  q_h = -k T_x + sum h_i J_i, V_i = -(D_i / X_i) X_i,x plus the correction
  velocity), with the primitive derivatives taken independently by complex-step
  differentiation of a manufactured profile, to rounding, per component.
* Species diffusion of a binary mixture of identical molecules at rest decays as
  exp(-D k^2 t) (the heat equation), at the design order.
* A standing acoustic wave loses energy at the Stokes-Kirchhoff rate
  (4/3 nu + (gamma - 1) chi) k^2, and at 4/3 nu k^2 without conduction.
* The LDG gradient of a smooth periodic field converges to its derivative.
* With delays and the AT flux, the viscous scheme conserves mass, momentum and
  energy to rounding, and the AT flux keeps the asynchrony error far below that
  of the plain delayed flux."""
import dataclasses

import numpy as np
import pytest

import oracle as O
from paper_2501_01747_gb300 import inputs as I
from tests import helpers as H

RU = 8.314462618
TREF = 298.15


def visc(wl, **kw):
    return dataclasses.replace(wl, viscous=1, **kw)


def test_pointwise_flux_matches_primitive_definition():
    wl = visc(I.load_workloads()["ignition-5sp-200x3"], mu_ref=2e-5)
    mech = wl.mechanism()
    ns = mech.ns
    rng = np.random.default_rng(3)
    a, b = rng.uniform(0.5, 1.5, ns), rng.uniform(-0.3, 0.3, ns)

    def prim(x):
        Yr = a * (1 + b * np.sin(3 * x + np.arange(ns)))
        return (Yr / Yr.sum(), 900 + 200 * np.sin(2 * x + 0.3), 30 * np.cos(1.5 * x),
                1e5 * (1 + 0.1 * np.sin(x + 1)))

    def cons(x):
        Y, T, u, P = prim(x)
        rho = P / (RU * T * np.sum(Y / mech.W))
        e = np.sum(Y * (mech.h_f + mech.cp * (T - TREF) - RU * T) / mech.W)
        return np.concatenate([[rho * u, rho * (e + 0.5 * u * u)], rho * Y])

    def d(f, x):  # complex-step derivative
        return np.imag(f(x + 1e-30j)) / 1e-30

    for x0 in (0.2, 0.7, 1.9):
        w, q = np.real(cons(x0)), d(cons, x0)
        fd = O.visc_flux(wl, mech, w, q)
        Y, T, u, P = [np.real(v) for v in prim(x0)]
        Tx, ux = d(lambda x: prim(x)[1], x0), d(lambda x: prim(x)[2], x0)
        X = lambda x: (prim(x)[0] / mech.W) / np.sum(prim(x)[0] / mech.W)
        Xv, Xx = np.real(X(x0)), d(X, x0)
        rho = P / (RU * T * np.sum(Y / mech.W))
        mu = wl.mu_ref * (T / wl.T_mu) ** wl.mu_exp
        cpm = np.sum(Y * mech.cp / mech.W)
        kc = mu * cpm / wl.prandtl
        D = kc / (rho * cpm * mech.Le)
        V = -(D / Xv) * Xx
        J = rho * Y * (V - np.sum(Y * V))
        qh = -kc * Tx + np.sum((mech.h_f + mech.cp * (T - TREF)) / mech.W * J)
        tau = 4 / 3 * mu * ux
        ref = np.concatenate([[tau, tau * u - qh], -J])
        # per component; a species flux relative to the largest one (a single
        # J_i can cancel to far below the others)
        scale = np.abs(ref)
        scale[2:] = np.abs(J).max()
        assert np.all(np.abs(fd - ref) <= 1e-13 * scale), (fd - ref) / scale
        assert abs(np.sum(J)) <= 1e-15 * np.abs(J).max()


def _binary_diffusion(ne, p=3, L=0.01, mu=8e-4, t_end=2e-4):
    mech = H.inert_mechanism()
    a0 = np.sqrt(1.4 * RU * 300.0 / 0.029)
    n = int(np.ceil(t_end / (0.3 * (L / ne) / ((2 * p + 1) * a0))))
    wl = visc(H.workload(ne, p, n_pe=1, length=L, dt=t_end / n), mu_ref=mu, T_mu=300.0,
              mu_exp=0.7, prandtl=0.7)
    x = wl.nodes_x()
    prim = np.zeros((mech.ns + 3,) + x.shape)
    prim[0], prim[1] = 300.0, 1e5
    prim[3] = 0.5 + 0.1 * np.sin(2 * np.pi * x / L)
    prim[4] = 1 - prim[3]
    o = O.Oracle(wl, mech)
    o.set_primitive(prim)
    o.step(n)
    r = H.modal_to_nodal(o.state()[2:], p)
    Y = r[0] / r.sum(0)
    D = mu / (1e5 * 0.029 / (RU * 300.0) * 0.7)
    exact = 0.5 + 0.1 * np.exp(-D * (2 * np.pi / L) ** 2 * t_end) * np.sin(2 * np.pi * x / L)
    return np.abs(Y - exact).max()


def test_binary_diffusion_is_the_heat_equation():
    """Two identical molecules, uniform T and P, at rest: J_1 = -rho D dY_1/dx, no
    correction, no enthalpy flux, so Y_1 obeys Y_t = D Y_xx exactly; 8 and 16
    elements x p3 against exp(-D k^2 t), error falling at order ~p+1."""
    e8, e16 = _binary_diffusion(8), _binary_diffusion(16)
    assert e8 < 3e-5 and e16 < 2e-6
    assert np.log2(e8 / e16) > 3.3


def _acoustic_rate(mu, prandtl, ne=16, p=3, L=0.01):
    mech = H.inert_mechanism()
    gam, T0, P0 = 29.1 / (29.1 - RU), 300.0, 1e5
    rho0 = P0 * 0.029 / (RU * T0)
    c0, k = np.sqrt(gam * P0 / rho0), 2 * np.pi / L
    t_end = 3 * L / c0
    n = int(np.ceil(t_end / (0.3 * (L / ne) / ((2 * p + 1) * c0))))
    wl = visc(H.workload(ne, p, n_pe=1, length=L, dt=t_end / n), mu_ref=mu, T_mu=T0, mu_exp=0.0,
              prandtl=prandtl)
    x = wl.nodes_x()
    prim = np.zeros((mech.ns + 3,) + x.shape)
    prim[0], prim[1], prim[2], prim[3:] = T0, P0, np.sin(k * x), 0.5
    _, wg = np.polynomial.legendre.leggauss(p + 1)

    def energy(w):
        rho = H.modal_to_nodal(w[2:].sum(0), p)
        u = H.modal_to_nodal(w[0], p) / rho
        rhoe = H.modal_to_nodal(w[1], p) - 0.5 * rho * u * u
        P = (gam - 1) * (rhoe + rho * 29.1 * TREF / 0.029)  # e = cv T - cp T_ref / W
        dens = 0.5 * rho0 * u * u + (P - P0) ** 2 / (2 * rho0 * c0 ** 2)
        return np.sum(dens * wg[None, :] * 0.5 * L / ne)

    o = O.Oracle(wl, mech)
    o.set_primitive(prim)
    e0 = energy(o.state())
    o.step(n)
    rate = -np.log(energy(o.state()) / e0) / t_end
    nu = mu / rho0
    return rate, (4 / 3 * nu + (gam - 1) * nu / prandtl) * k * k


@pytest.mark.parametrize("prandtl", [0.7, 1e9])
def test_acoustic_attenuation_stokes_kirchhoff(prandtl):
    """A standing wave (u = sin kx, 1 m/s) over three periods: the energy decays at
    (4/3 nu + (gamma-1) nu/Pr) k^2 to 1e-3 (the inviscid scheme's own loss is
    2e-5 of that rate); Pr = 1e9 switches conduction off."""
    rate, theory = _acoustic_rate(8e-3, prandtl)
    assert abs(rate / theory - 1) < 1e-3, (rate, theory)
    inviscid, _ = _acoustic_rate(0.0, 0.7)
    assert abs(inviscid) < 1e-4 * theory


def test_ldg_gradient_converges():
    """q of a smooth periodic state (all variables sinusoidal) against the exact
    derivative, 8 -> 16 -> 32 elements, p = 2 and 3: error falls at order >= p."""
    mech = H.inert_mechanism()
    for p in (2, 3):
        errs = []
        for ne in (8, 16, 32):
            wl = visc(H.workload(ne, p, n_pe=1, length=1.0, dt=1e-6))
            xq, wq = np.polynomial.legendre.leggauss(p + 1)
            x = wl.nodes_x()
            f = lambda x, v: (v + 1.0) * (1.5 + np.sin(2 * np.pi * x + v))
            df = lambda x, v: (v + 1.0) * 2 * np.pi * np.cos(2 * np.pi * x + v)
            V = np.polynomial.legendre.legvander(xq, p)
            proj = lambda vals: (vals @ (wq[:, None] * V)) * (np.arange(p + 1) + 0.5)
            w = np.stack([proj(f(x, v)) for v in range(4)])
            q = O.aux_sync(wl, mech, w)
            qn = H.modal_to_nodal(q, p)
            errs.append(max(np.abs(qn[v] - df(x, v)).max() for v in range(4)))
        rates = [np.log2(errs[i] / errs[i + 1]) for i in range(2)]
        assert min(rates) >= p - 0.3, (p, errs, rates)


def _viscous_ignition(mode, at_order, n=40, n_pe=8):
    base = I.load_workloads()["ignition-5sp-200x3"]
    wl = visc(I.scaled(base, 96, n_pe), delay_mode=mode, max_delay=2, at_order=at_order,
              delay_probs=I.SAA_SETS[1], mu_ref=3e-5)
    mech = wl.mechanism()
    o = O.Oracle(wl, mech)
    o.set_primitive(wl.primitive(mech))
    w0 = o.state()
    o.step(n)
    return w0, o.state(), wl, mech


@pytest.mark.parametrize("mode", [I.DELAY_CAA, I.DELAY_SAA])
def test_viscous_with_delays_conserves(mode):
    w0, w, wl, mech = _viscous_ignition(mode, 4)
    for v, name in ((0, "momentum"), (1, "energy")):
        scale = np.abs(w0[1, :, 0]).sum() if v == 1 else H.parity_scales(w, mech)[0] * wl.n_elem
        assert abs(w[v, :, 0].sum() - w0[v, :, 0].sum()) <= 1e-12 * scale, name
    assert abs(w[2:, :, 0].sum() - w0[2:, :, 0].sum()) <= 1e-13 * w0[2:, :, 0].sum()


def test_at_flux_pays_off_viscous():
    _, ref, _, mech = _viscous_ignition(I.DELAY_SYNC, 4)
    _, w4, _, _ = _viscous_ignition(I.DELAY_CAA, 4)
    _, w1, _, _ = _viscous_ignition(I.DELAY_CAA, 1)
    e4 = H.parity_error(w4, ref, mech).max()
    e1 = H.parity_error(w1, ref, mech).max()
    assert 0 < e4 < 0.05 * e1, (e4, e1)
