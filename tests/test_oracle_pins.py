"""Pins of the FP64 oracle to facts fixed by the paper and by mathematics.

Each test checks the oracle against something other than itself: numpy's library
routines, closed forms, printed values of the paper (Table 1), thermodynamic
identities, invariants and textbook exact solutions."""
import json
import os

import numpy as np
import pytest

import oracle as O
from paper_2501_01747_gb300 import inputs as I
from tests import helpers as H

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")
RU = 8.314462618


# --------------------------------------------------------------------------
# basis, quadrature, limiter tables

@pytest.mark.parametrize("q", range(1, 9))
def test_gauss_matches_library(q):
    x, w = O.gauss(q)
    xr, wr = np.polynomial.legendre.leggauss(q)
    assert np.allclose(x, xr, rtol=0, atol=2e-15)
    assert np.allclose(w, wr, rtol=0, atol=2e-15)


def test_legendre_values_and_derivatives():
    for x in np.linspace(-1, 1, 13):
        P, dP = O.legendre(6, x)
        for j in range(7):
            c = np.zeros(j + 1)
            c[j] = 1
            assert abs(P[j] - np.polynomial.legendre.legval(x, c)) < 1e-14
            assert abs(dP[j] - np.polynomial.legendre.legval(x, np.polynomial.legendre.legder(c))) < 1e-12
    # endpoint values used by the surface terms of Eq. (5): P_j(1)=1, P_j(-1)=(-1)^j
    P, _ = O.legendre(6, 1.0)
    assert np.all(P == 1.0)
    P, _ = O.legendre(6, -1.0)
    assert np.all(P == np.array([(-1.0) ** j for j in range(7)]))


def test_mass_and_stiffness_exact():
    """Eq. (6) with Legendre polynomials: M = diag(2/(2j+1)); S_ij = int P_j P_i' is
    2 when j < i and i + j is odd, else 0. The oracle evaluates S f with p+1 Gauss
    points: check that this reproduces S exactly for a polynomial flux."""
    for p in range(1, 6):
        x, w = O.gauss(p + 1)
        V = np.array([O.legendre(p, xi)[0] for xi in x])    # [q, j]
        dV = np.array([O.legendre(p, xi)[1] for xi in x])
        M = np.einsum("q,qi,qj->ij", w, V, V)
        S = np.einsum("q,qj,qi->ij", w, V, dV)
        assert np.allclose(M, np.diag(2.0 / (2 * np.arange(p + 1) + 1)), atol=1e-14)
        S_exact = np.zeros((p + 1, p + 1))
        for i in range(p + 1):
            for j in range(p + 1):
                if j < i and (i + j) % 2 == 1:
                    S_exact[i, j] = 2.0
        assert np.allclose(S, S_exact, atol=1e-13)


@pytest.mark.parametrize("p", range(1, 6))
def test_beta_matrix_against_numpy_polynomials(p):
    """beta = sum_s 2^(2s-1) int (d^s v / dxi^s)^2 (Eq. 10 mapped to [-1, 1])."""
    B = O.beta_matrix(p)
    L = np.polynomial.legendre.Legendre
    ref = np.zeros((p + 1, p + 1))
    for i in range(p + 1):
        for j in range(p + 1):
            acc = 0.0
            for s in range(1, p + 1):
                prod = L.basis(i).deriv(s) * L.basis(j).deriv(s)
                ii = prod.integ()
                acc += 2.0 ** (2 * s - 1) * (ii(1.0) - ii(-1.0))
            ref[i, j] = acc
    assert np.allclose(B, ref, rtol=1e-13, atol=1e-12)
    if p == 1:
        assert np.allclose(B, [[0, 0], [0, 4]])


@pytest.mark.parametrize("p", range(1, 6))
@pytest.mark.parametrize("direction", [-1, 1])
def test_shift_matrix_continues_the_neighbour(p, direction):
    """S maps a neighbour's modal coefficients to those of the same polynomial
    written in this cell's coordinate (xi' = xi - 2 dir)."""
    S = O.shift_matrix(p, direction)
    rng = np.random.default_rng(p)
    a = rng.normal(size=p + 1)
    xi = np.linspace(-1, 1, 9)
    lhs = np.polynomial.legendre.legval(xi, S @ a)
    rhs = np.polynomial.legendre.legval(xi - 2 * direction, a)
    assert np.allclose(lhs, rhs, rtol=1e-12, atol=1e-12)


# --------------------------------------------------------------------------
# AT coefficients (Sec. 3.2, Eq. 7-8, Table 1)

def _poly(coefs, k):
    return coefs[0] * k ** 3 + coefs[1] * k ** 2 + coefs[2] * k + coefs[3]


def test_at_coefficients_match_table1():
    tab = json.load(open(os.path.join(GOLDEN, "at_table1.json")))
    for order_s, rows in tab["printed"].items():
        order = int(order_s)
        for k in range(0, 6):
            c = O.at_coeffs(order, k)
            for m, (num, den, sign) in enumerate(rows):
                if order == tab["typo"]["order"] and m == tab["typo"]["m"]:
                    den = tab["typo"]["corrected_denominator"]
                expect = sign * _poly(num, k) / den
                assert c[m] == pytest.approx(expect, abs=1e-12), (order, k, m)


def test_table1_typo_breaks_consistency():
    """As printed, order-4 weights do not sum to one; corrected, they do."""
    tab = json.load(open(os.path.join(GOLDEN, "at_table1.json")))
    rows = tab["printed"]["4"]
    for k in range(1, 5):
        printed = sum(sign * _poly(num, k) / den for num, den, sign in rows)
        assert abs(printed - 1.0) > 0.5
        assert sum(O.at_coeffs(4, k)) == pytest.approx(1.0, abs=1e-12)


@pytest.mark.parametrize("order", range(1, 7))
def test_at_coefficients_solve_eq8(order):
    """Eq. (8) with r = 1: sum_l c^l (-l)^zeta / zeta! = delta_{zeta,0} for
    zeta < order, over l = k..k+order-1; solved here with numpy's linear solver."""
    from math import factorial
    for k in range(0, 6):
        ls = np.arange(k, k + order)
        A = np.array([[(-l) ** z / factorial(z) for l in ls] for z in range(order)], dtype=float)
        rhs = np.zeros(order)
        rhs[0] = 1.0
        ref = np.linalg.solve(A, rhs)
        c = O.at_coeffs(order, k)
        assert np.allclose(c, ref, rtol=1e-9, atol=1e-9)
        if k == 0:
            assert c[0] == 1.0 and np.all(c[1:] == 0.0)


def test_at2_worked_form():
    """Sec. 3.2: f^at = (k+1) f^{n-k} - k f^{n-k-1}."""
    for k in range(6):
        assert np.array_equal(O.at_coeffs(2, k), [k + 1.0, -float(k)])


# --------------------------------------------------------------------------
# delays (Sec. 4.1, 4.2)

def test_splitmix64_known_answer():
    """SplitMix64 (Steele, Lea and Flood 2014) from state 0: the published first
    output of java.util.SplittableRandom(0).nextLong(), -2152535657050944081."""
    assert O.splitmix64(0) == 0xE220A8397B1DCDAF


def test_caa_schedule():
    wl = H.workload(8, 1, n_pe=2, delay_mode=I.DELAY_CAA, max_delay=2)
    got = [O.delay(wl, n, 0) for n in range(10)]
    assert got == [0, 1, 2, 0, 1, 2, 0, 1, 2, 0]


@pytest.mark.parametrize("set_id", [1, 2, 3])
def test_saa_frequencies(set_id):
    probs = I.SAA_SETS[set_id]
    wl = H.workload(8, 1, n_pe=4, delay_mode=I.DELAY_SAA, max_delay=2, probs=probs,
                    seed=2501017490 + set_id)
    n = 20000
    counts = np.zeros(3)
    for step in range(n // 4):
        for f in range(4):
            counts[O.delay(wl, step, f)] += 1
    exp = np.array(probs) * n
    chi2 = float(((counts - exp) ** 2 / exp).sum())
    assert chi2 < 13.8  # 99.9 % quantile, 2 degrees of freedom


def test_saa_all_zero_set_is_synchronous():
    wl = H.workload(8, 1, n_pe=4, delay_mode=I.DELAY_SAA, max_delay=2, probs=(1.0, 0.0, 0.0))
    assert all(O.delay(wl, s, f) == 0 for s in range(100) for f in range(4))


# --------------------------------------------------------------------------
# thermodynamics

def test_temperature_closed_form():
    """For constant c_p, e(T) is linear, so the Newton root equals
    T = T_ref + (e - sum Y_i (h_f,i - R T_ref)/W_i) / c_v."""
    mech = I.make_mechanism(9, 21, 7)
    rng = np.random.default_rng(0)
    for _ in range(20):
        Y = rng.dirichlet(np.ones(9))
        T = rng.uniform(250, 4000)
        rho = rng.uniform(0.05, 20)
        e = np.sum(Y * (mech.h_f + mech.cp * (T - 298.15) - RU * T) / mech.W)
        cv = np.sum(Y * (mech.cp - RU) / mech.W)
        T_closed = 298.15 + (e - np.sum(Y * (mech.h_f - RU * 298.15) / mech.W)) / cv
        Tn, it = O.temperature(mech, rho * Y, rho * e, guess=1000.0)
        assert Tn == pytest.approx(T_closed, rel=1e-13)
        assert Tn == pytest.approx(T, rel=1e-12)
        assert 1 <= it <= 3


def test_single_species_ideal_gas():
    """One species: P = rho R T / W and a = sqrt(gamma R T / W), gamma = cp/(cp-R)."""
    mech = H.inert_mechanism(ns=1, W=0.028, cp=29.0)
    for T, P, u in [(300.0, 101325.0, 0.0), (1500.0, 3e6, 120.0), (3000.0, 5e4, -700.0)]:
        w = O.cons_from_prim(mech, T, P, u, np.array([1.0]))
        rho, uu, TT, PP, a = O.state(mech, w)
        assert rho == pytest.approx(P * 0.028 / (RU * T), rel=1e-14)
        assert uu == pytest.approx(u, abs=1e-9)
        assert TT == pytest.approx(T, rel=1e-12)
        assert PP == pytest.approx(P, rel=1e-12)
        g = 29.0 / (29.0 - RU)
        assert a == pytest.approx(np.sqrt(g * RU * T / 0.028), rel=1e-12)


def test_mixture_sound_speed_against_finite_difference():
    """Frozen a^2 = (dP/drho) at constant entropy and composition, checked by
    compressing the mixture isentropically with a small step."""
    mech = I.make_mechanism(9, 21, 3)
    Y = np.random.default_rng(2).dirichlet(np.ones(9))
    T0, P0 = 1200.0, 2e5
    w = O.cons_from_prim(mech, T0, P0, 0.0, Y)
    rho0, _, _, _, a = O.state(mech, w)
    cp = np.sum(Y * mech.cp / mech.W)
    cv = np.sum(Y * (mech.cp - RU) / mech.W)
    g = cp / cv
    eps = 1e-6
    rho1 = rho0 * (1 + eps)
    P1 = P0 * (1 + eps) ** g          # isentropic ideal gas with constant cp, cv
    assert a * a == pytest.approx((P1 - P0) / (rho1 - rho0), rel=1e-5)


# --------------------------------------------------------------------------
# kinetics

def test_mass_and_element_conservation_of_rates():
    mech = I.make_mechanism(9, 21, 11)
    rng = np.random.default_rng(5)
    for T in (600.0, 1500.0, 3000.0):
        conc = rng.uniform(0.0, 5.0, size=9)
        wd = O.wdot(mech, T, conc)
        scale = np.abs(wd).max()
        assert abs(np.sum(mech.W * wd)) <= 1e-13 * scale * mech.W.max() * 9
        el = mech.comp.T @ wd
        assert np.all(np.abs(el) <= 1e-12 * scale * 9 * 4)


def test_equilibrium_from_chemical_potentials():
    """At fixed T and V a reaction stops where sum_i nu_i mu_i = 0, with the
    ideal-gas chemical potential mu_i = g_i(T) + R T ln(c_i R T / P_atm). Pick all
    concentrations but one at random, solve that condition for the last one (in
    logs), and the oracle's rate of progress (law of mass action with K_c) must
    vanish there."""
    mech = I.make_mechanism(9, 21, 2)
    rng = np.random.default_rng(8)
    for j in range(mech.nr):
        nu = mech.nu_r[j].astype(float) - mech.nu_f[j].astype(float)
        for T in (900.0, 2200.0):
            g = (mech.h_f + mech.cp * (T - 298.15)) - T * (mech.s0 + mech.cp * np.log(T / 298.15))
            c = rng.uniform(0.5, 5.0, size=mech.ns)
            i = int(np.flatnonzero(nu)[-1])
            mu = g + RU * T * np.log(c * RU * T / I.P_ATM)
            rest = float(np.dot(nu, mu) - nu[i] * mu[i])
            mu_i = -rest / nu[i]
            c[i] = I.P_ATM / (RU * T) * np.exp((mu_i - g[i]) / (RU * T))
            single = I.Mechanism(W=mech.W, cp=mech.cp, h_f=mech.h_f, s0=mech.s0,
                                 nu_f=mech.nu_f[j:j + 1], nu_r=mech.nu_r[j:j + 1],
                                 A=mech.A[j:j + 1], b=mech.b[j:j + 1], Ea=mech.Ea[j:j + 1],
                                 comp=mech.comp, names=mech.names)
            kf, _ = O.rates(single, T, 0)
            fwd = kf * np.prod(c ** mech.nu_f[j])
            wd = O.wdot(single, T, c)
            assert abs(wd[i]) <= 1e-9 * fwd * abs(nu[i])
            # and away from equilibrium it is not zero
            c2 = c.copy()
            c2[i] *= 1.5
            assert abs(O.wdot(single, T, c2)[i]) > 1e-3 * fwd * abs(nu[i])


def test_van_t_hoff():
    """d ln K_p / dT = dH / (R T^2), K_p = K_c (R T / P_atm)^{sum nu}: pins the sign
    of nu, the enthalpies and the pressure factor of K_c."""
    mech = I.make_mechanism(9, 21, 4)
    for j in range(mech.nr):
        nu = mech.nu_r[j].astype(float) - mech.nu_f[j].astype(float)
        dn = nu.sum()
        for T in (700.0, 1800.0):
            h = 1e-3 * T

            def lnKp(t):
                _, Kc = O.rates(mech, t, j)
                return np.log(Kc) + dn * np.log(RU * t / I.P_ATM)

            d = (lnKp(T + h) - lnKp(T - h)) / (2 * h)
            dH = np.dot(nu, mech.h_f + mech.cp * (T - 298.15))
            assert d == pytest.approx(dH / (RU * T * T), rel=1e-5, abs=1e-9)


def test_arrhenius_plot():
    """With b = 0, ln k_f is linear in 1/T with slope -E_a/R; with E_a = 0, linear in
    ln T with slope b; both with intercept ln A."""
    mech = I.make_mechanism(5, 4, 9)
    m = I.Mechanism(**{**mech.__dict__})
    m.b = np.array([0.0, 0.7, 0.0, -0.4])
    m.Ea = np.array([1.2e5, 0.0, 3.0e4, 0.0])
    for j in range(4):
        k1, _ = O.rates(m, 800.0, j)
        k2, _ = O.rates(m, 1600.0, j)
        if m.b[j] == 0:
            slope = (np.log(k2) - np.log(k1)) / (1 / 1600.0 - 1 / 800.0)
            assert slope == pytest.approx(-m.Ea[j] / RU, rel=1e-10)
        else:
            slope = (np.log(k2) - np.log(k1)) / (np.log(1600.0) - np.log(800.0))
            assert slope == pytest.approx(m.b[j], rel=1e-10)
            assert np.log(k1) - m.b[j] * np.log(800.0) == pytest.approx(np.log(m.A[j]), rel=1e-12)


def test_reactor_conserves_mass_and_energy():
    wl = I.load_workloads()["ignition-5sp-200x3"]
    mech = wl.mechanism()
    Y = I.composition(mech, 0.02)
    w = O.cons_from_prim(mech, 1400.0, I.P_ATM, 0.0, Y)
    r = w[2:].copy()
    r1 = O.reactor0d(mech, r, w[1], wl.dt, 400)
    assert np.sum(r1) == pytest.approx(np.sum(r), rel=1e-14)
    assert not np.allclose(r1, r)  # it did react


# --------------------------------------------------------------------------
# fluxes and eigenvectors

def _random_state(mech, rng, T=None, P=None, u=None):
    Y = rng.dirichlet(np.ones(mech.ns))
    return O.cons_from_prim(mech, T or rng.uniform(300, 3000), P or rng.uniform(5e4, 3e6),
                            rng.uniform(-600, 600) if u is None else u, Y)


def test_physical_flux_definition():
    mech = I.make_mechanism(9, 21, 1)
    rng = np.random.default_rng(3)
    w = _random_state(mech, rng)
    rho, u, T, P, a = O.state(mech, w)
    f = O.phys_flux(mech, w)
    assert f[0] == pytest.approx(rho * u * u + P, rel=1e-13)
    assert f[1] == pytest.approx(u * (w[1] + P), rel=1e-13)
    assert np.allclose(f[2:], u * w[2:], rtol=1e-14)


@pytest.mark.parametrize("kind", [I.FLUX_LF, I.FLUX_HLLC])
def test_numerical_flux_consistency(kind):
    mech = I.make_mechanism(9, 21, 1)
    rng = np.random.default_rng(4)
    for _ in range(10):
        w = _random_state(mech, rng)
        assert np.allclose(O.num_flux(mech, kind, w, w), O.phys_flux(mech, w), rtol=1e-11,
                           atol=1e-9)


def test_hllc_upwinds_supersonic_and_keeps_contacts():
    mech = I.make_mechanism(9, 21, 1)
    rng = np.random.default_rng(6)
    # supersonic to the right: flux is the left flux
    wl = _random_state(mech, rng, T=400.0, u=1500.0)
    wr = _random_state(mech, rng, T=500.0, u=1400.0)
    assert np.allclose(O.num_flux(mech, I.FLUX_HLLC, wl, wr), O.phys_flux(mech, wl), rtol=1e-13)
    # stationary contact: equal P, u = 0, different T and composition -> flux (P, 0, 0..)
    P = 2e5
    wl = _random_state(mech, rng, T=400.0, P=P, u=0.0)
    wr = _random_state(mech, rng, T=2400.0, P=P, u=0.0)
    f = O.num_flux(mech, I.FLUX_HLLC, wl, wr)
    assert f[0] == pytest.approx(P, rel=1e-12)
    assert np.all(np.abs(f[1:]) <= 1e-9 * P)


def test_eigenvectors_diagonalise_the_jacobian():
    """A R = R Lambda and L R = I with A from central differences of f^c."""
    mech = I.make_mechanism(9, 21, 5)
    rng = np.random.default_rng(7)
    for _ in range(5):
        w = _random_state(mech, rng)
        R, L, lam = O.eigen(mech, w)
        nv = w.size
        A = np.zeros((nv, nv))
        for v in range(nv):
            h = 1e-6 * max(abs(w[v]), 1e-3 * np.abs(w[2:]).sum())
            wp = w.copy()
            wm = w.copy()
            wp[v] += h
            wm[v] -= h
            A[:, v] = (O.phys_flux(mech, wp) - O.phys_flux(mech, wm)) / (2 * h)
        scale = np.abs(A @ R).max()
        assert np.allclose(A @ R, R * lam[None, :], rtol=0, atol=2e-6 * scale)
        assert np.allclose(L @ R, np.eye(nv), atol=1e-9)
        rho, u, T, P, a = O.state(mech, w)
        assert lam[0] == pytest.approx(u - a) and lam[-1] == pytest.approx(u + a)
