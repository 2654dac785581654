"""Shared test fixtures: small inert mechanisms, hand-built workloads, exact
solutions written from textbook definitions (not from either implementation)."""
from __future__ import annotations

import dataclasses

import numpy as np

from paper_2501_01747_gb300 import inputs as I

RU = 8.314462618


def inert_mechanism(ns=2, W=0.029, cp=29.1):
    """ns identical, non-reacting species (an ideal gas with gamma = cp/(cp-R))."""
    z = np.zeros((0, ns), dtype=np.int8)
    return I.Mechanism(W=np.full(ns, W), cp=np.full(ns, cp), h_f=np.zeros(ns),
                       s0=np.full(ns, 200.0), nu_f=z, nu_r=z.copy(), A=np.zeros(0),
                       b=np.zeros(0), Ea=np.zeros(0), comp=np.zeros((ns, 4), dtype=int),
                       names=["s%d" % i for i in range(ns)])


def workload(n_elem, p, n_pe=1, length=1.0, dt=1e-6, bc=(0, 0), flux=I.FLUX_LF,
             limiter=I.LIM_NONE, at_order=None, delay_mode=I.DELAY_SYNC, max_delay=0,
             probs=None, seed=12345, ic_kind="advection", ic_params=None, ns=2, nr=0,
             n_steps=1):
    return I.Workload(
        name="test", n_elem=n_elem, p=p, n_pe=n_pe, length=length, dt=dt,
        bc_left=bc[0], bc_right=bc[1], flux=flux, limiter=limiter,
        at_order=(p + 1) if at_order is None else at_order, delay_mode=delay_mode,
        max_delay=max_delay, delay_probs=tuple(probs) if probs else
        tuple([1.0 / (max_delay + 1)] * (max_delay + 1)), seed=seed, ns=ns, nr=nr,
        mech_seed=0, ic_seed=1, ic_kind=ic_kind,
        ic_params=ic_params or {"T0": 300.0, "amp": 0.2, "u0": 50.0, "y_fuel": 0.5,
                                "y_ox": 0.0},
        n_steps=n_steps)


def two_species_ic(wl, mech, rho_fn, u, P):
    """Primitive IC of an entropy wave: rho(x), uniform u and P, Y = (0.5, 0.5)."""
    x = wl.nodes_x()
    Wbar = 1.0 / np.sum(0.5 / mech.W)
    rho = rho_fn(x)
    prim = np.zeros((mech.ns + 3, wl.n_elem, wl.p + 1))
    prim[0] = P * Wbar / (rho * RU)
    prim[1] = P
    prim[2] = u
    prim[3:] = 1.0 / mech.ns
    return prim


def gauss_l2(wl, values, exact):
    """L2 norm over the domain with the Gauss rule of the elements."""
    x, w = np.polynomial.legendre.leggauss(wl.p + 1)
    dx = wl.length / wl.n_elem
    return float(np.sqrt(np.sum(w[None, :] * 0.5 * dx * (values - exact) ** 2)))


def modal_to_nodal(w, p):
    """Evaluate modal Legendre coefficients [..., p+1] at the Gauss points."""
    x, _ = np.polynomial.legendre.leggauss(p + 1)
    V = np.polynomial.legendre.legvander(x, p)  # [q, j]
    return np.einsum("...j,qj->...q", w, V)


# ---------------------------------------------------------------------------
# Exact Riemann solver for the ideal-gas Euler equations (Toro, "Riemann Solvers
# and Numerical Methods for Fluid Dynamics", ch. 4): pressure function, Newton
# for p*, then sampling of the self-similar solution.

def exact_riemann(rl, ul, pl, rr, ur, pr, gamma, xi):
    g = gamma
    al = np.sqrt(g * pl / rl)
    ar = np.sqrt(g * pr / rr)

    def fk(p, rk, pk, ak):
        if p > pk:
            A = 2.0 / ((g + 1) * rk)
            B = (g - 1) / (g + 1) * pk
            f = (p - pk) * np.sqrt(A / (p + B))
            df = np.sqrt(A / (B + p)) * (1 - (p - pk) / (2 * (B + p)))
        else:
            f = 2 * ak / (g - 1) * ((p / pk) ** ((g - 1) / (2 * g)) - 1)
            df = 1.0 / (rk * ak) * (p / pk) ** (-(g + 1) / (2 * g))
        return f, df

    p = 0.5 * (pl + pr)
    for _ in range(100):
        f1, d1 = fk(p, rl, pl, al)
        f2, d2 = fk(p, rr, pr, ar)
        dp = (f1 + f2 + ur - ul) / (d1 + d2)
        p = max(p - dp, 1e-8)
        if abs(dp) < 1e-12 * p:
            break
    f1, _ = fk(p, rl, pl, al)
    f2, _ = fk(p, rr, pr, ar)
    us = 0.5 * (ul + ur) + 0.5 * (f2 - f1)
    out = np.zeros((3,) + np.shape(xi))
    for idx, s in np.ndenumerate(np.asarray(xi)):
        if s <= us:  # left of contact
            if p > pl:
                sl = ul - al * np.sqrt((g + 1) / (2 * g) * p / pl + (g - 1) / (2 * g))
                if s <= sl:
                    v = (rl, ul, pl)
                else:
                    r = rl * ((p / pl + (g - 1) / (g + 1)) / ((g - 1) / (g + 1) * p / pl + 1))
                    v = (r, us, p)
            else:
                shl = ul - al
                stl = us - al * (p / pl) ** ((g - 1) / (2 * g))
                if s <= shl:
                    v = (rl, ul, pl)
                elif s >= stl:
                    v = (rl * (p / pl) ** (1 / g), us, p)
                else:
                    c = 2 / (g + 1) + (g - 1) / ((g + 1) * al) * (ul - s)
                    v = (rl * c ** (2 / (g - 1)), 2 / (g + 1) * (al + (g - 1) / 2 * ul + s),
                         pl * c ** (2 * g / (g - 1)))
        else:
            if p > pr:
                sr = ur + ar * np.sqrt((g + 1) / (2 * g) * p / pr + (g - 1) / (2 * g))
                if s >= sr:
                    v = (rr, ur, pr)
                else:
                    r = rr * ((p / pr + (g - 1) / (g + 1)) / ((g - 1) / (g + 1) * p / pr + 1))
                    v = (r, us, p)
            else:
                shr = ur + ar
                str_ = us + ar * (p / pr) ** ((g - 1) / (2 * g))
                if s >= shr:
                    v = (rr, ur, pr)
                elif s <= str_:
                    v = (rr * (p / pr) ** (1 / g), us, p)
                else:
                    c = 2 / (g + 1) - (g - 1) / ((g + 1) * ar) * (ur - s)
                    v = (rr * c ** (2 / (g - 1)), 2 / (g + 1) * (-ar + (g - 1) / 2 * ur + s),
                         pr * c ** (2 * g / (g - 1)))
        out[(slice(None),) + idx] = v
    return out


def parity_scales(w, mech):
    """Physical scale of every conserved variable of a modal state [nv][N][Q]:
    max|rho E| for the energy, max rho (|u| + a) for the momentum and
    max(max|rho Y_i|, 1e-5 max rho) for the partial densities (cell averages).
    tests/test_oracle_conditioning.py shows that in these scales the oracle itself
    moves by less than 1e-11 when its input moves by 1e-15."""
    scale = np.abs(w).max(axis=(1, 2))
    r = w[2:, :, 0]
    rho = r.sum(axis=0)
    u = w[0, :, 0] / rho
    rhoe = w[1, :, 0] - 0.5 * rho * u * u
    q = ((mech.h_f - mech.cp * 298.15) / mech.W)[:, None]
    cv = ((mech.cp - RU) / mech.W)[:, None]
    T = (rhoe - (r * q).sum(0)) / (r * cv).sum(0)
    cpm = (r * (mech.cp / mech.W)[:, None]).sum(0)
    cvm = (r * cv).sum(0)
    a = np.sqrt(np.abs(cpm / cvm * (cpm - cvm) / rho * T))
    scale[0] = max(scale[0], float(np.max(rho * (np.abs(u) + a))))
    scale[2:] = np.maximum(scale[2:], 1e-5 * rho.max())
    return scale


def parity_error(a, b, mech):
    """Per-variable error of a against the reference b in those scales."""
    return np.abs(a - b).max(axis=(1, 2)) / np.maximum(parity_scales(b, mech), 1e-300)
