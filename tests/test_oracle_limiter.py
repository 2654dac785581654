"""Pins of the oracle's troubled-cell indicator and (AT-)WENO reconstruction
(Sec. 3.3, Eq. 9-10) on hand-built states whose characteristic structure is
known in closed form, so that the expected flags and limited modes can be
worked out by hand from the definitions:

- a contact between two identical, inert species at rest (uniform density,
  pressure and temperature): only the two species fields of the frozen
  Jacobian vary, by +-d(rho Y_1), and the limiter acts on rho Y_1 as on a
  scalar;
- a weak acoustic perturbation along the right eigenvector r_+ or r_- of the
  Euler system, (rho u, rho E, rho Y_i) ~ (u +- a, H +- u a, Y_i): only the
  field of that wave varies (the others by second-order terms far below the
  indicator's rounding guard);
- flat data with noise at the level of double rounding.

The indicator is TVD minmod (M = 0) on both face deviations v(+1) - vbar and
vbar - v(-1) against the neighbours' mean differences; with modal Legendre
coefficients (c0, c1, c2) these deviations are c1 + c2 and c1 - c2.
WENO (Eq. 9-10) with gamma = (0.001, 0.998, 0.001), eps = 1e-6 and the
smoothness indicator beta = sum_s 2^(2s-1) int (d^s v / d xi^s)^2 d xi, which
for v = c0 + c1 P1 + c2 P2 is 4 c1^2 + 156 c2^2 (p = 2) and 4 c1^2 (p = 1).
A neighbour continued into the cell, x' = xi -+ 2 in its own coordinate, has
the modes (a0 + 2 a1 + 6 a2, a1 + 6 a2, a2) (left) and
(b0 - 2 b1 + 6 b2, b1 - 6 b2, b2) (right), from P2(xi + 2) = P2(xi) + 6 xi + 6;
its mean is replaced by the cell's own."""
import numpy as np
import pytest

import oracle as O
from paper_2501_01747_gb300 import inputs as I
from tests import helpers as H

RU = 8.314462618
RHO, P0 = 1.2, 1e5

# species-1 partial density modes (c0, c1, c2) per element of a periodic mesh
CELLS = np.array([
    [0.60, 0.00, 0.000],   # flat
    [0.60, 0.00, 0.000],   # flat
    [0.60, 0.05, 0.010],   # left neighbour mean equal: dm = 0           -> troubled
    [0.90, 0.08, -0.005],  # deviations 0.075, 0.085 within dp=0.1, dm=0.3
    [1.00, 0.02, 0.000],   # deviations 0.02 within dp = dm = 0.1
    [1.10, 0.01, 0.030],   # v(+1)-vbar = 0.04 fits, vbar-v(-1) = -0.02 has
                           # the wrong sign (p = 2 only)                  -> troubled
    [1.15, 0.02, 0.000],   # local maximum of the means: dp < 0 < dm      -> troubled
    [0.62, -0.01, 0.000],  # -0.01 within dp = -0.02, dm = -0.53
])
FLAGS_P2 = [0, 0, 1, 0, 0, 1, 1, 0]
FLAGS_P1 = [0, 0, 1, 0, 0, 0, 1, 0]   # cell 5 is within bounds without its c2


def _wl(p, n=8, limiter=I.LIM_WENO):
    return H.workload(n, p, n_pe=1, dt=1e-9, bc=(I.BC_PERIODIC, I.BC_PERIODIC),
                      limiter=limiter)


def _rest_state(mech):
    """Uniform rest state of the inert two-species gas: (rho e, T, a, H)."""
    W, cp = mech.W[0], mech.cp[0]
    T = P0 * W / (RHO * RU)
    e = (cp * (T - 298.15) - RU * T) / W
    gam = cp / (cp - RU)
    a = np.sqrt(gam * P0 / RHO)
    H_ = (RHO * e + P0) / RHO
    return RHO * e, T, a, H_


def contact_state(p, cells=CELLS):
    """Species contact: rho Y_1 takes the modes of `cells`, rho Y_2 = rho - rho Y_1,
    rho u = 0, rho E uniform (identical species have one e(T))."""
    mech = H.inert_mechanism()
    rhoE, _, _, _ = _rest_state(mech)
    n = len(cells)
    w = np.zeros((4, n, p + 1))
    w[1, :, 0] = rhoE
    w[2] = cells[:, :p + 1]
    w[3, :, 0] = RHO - cells[:, 0]
    w[3, :, 1:] = -cells[:, 1:p + 1]
    return mech, w


def weno_modes(own, left, right, p):
    """Limited modes 1..p of one cell from Eq. (9)-(10), by hand."""
    gam = (0.001, 0.998, 0.001)
    eps = 1e-6
    if p == 1:
        cands = [(left[1],), (own[1],), (right[1],)]
        beta = [4 * c[0] ** 2 for c in cands]
    else:
        cands = [(left[1] + 6 * left[2], left[2]), (own[1], own[2]),
                 (right[1] - 6 * right[2], right[2])]
        beta = [4 * c[0] ** 2 + 156 * c[1] ** 2 for c in cands]
    wt = [g / (eps + b) ** 2 for g, b in zip(gam, beta)]
    s = sum(wt)
    wt = [x / s for x in wt]
    return [sum(wt[t] * cands[t][i] for t in range(3)) for i in range(p)]


@pytest.mark.parametrize("p,expected", [(2, FLAGS_P2), (1, FLAGS_P1)])
def test_indicator_flags_of_a_species_contact(p, expected):
    mech, w = contact_state(p)
    flags, _ = O.limit_sync(_wl(p), mech, w)
    assert flags.tolist() == expected


@pytest.mark.parametrize("p", [1, 2])
def test_weno_modes_of_a_species_contact(p):
    """Limited modes of every troubled cell equal the hand-computed WENO of Eq.
    (9)-(10); cell averages and untroubled cells are untouched; rho Y_2 moves
    opposite to rho Y_1; momentum and energy keep their (zero) higher modes."""
    mech, w = contact_state(p)
    flags, out = O.limit_sync(_wl(p), mech, w)
    n = len(CELLS)
    assert flags.sum() >= 2
    assert np.array_equal(out[:, :, 0], w[:, :, 0])
    for e in range(n):
        if not flags[e]:
            assert np.array_equal(out[:, e], w[:, e])
            continue
        exp = weno_modes(CELLS[e], CELLS[(e - 1) % n], CELLS[(e + 1) % n], p)
        got = out[2, e, 1:]
        assert np.allclose(got, exp, rtol=1e-9, atol=1e-14), (e, got, exp)
        assert np.allclose(out[3, e, 1:], -got, rtol=0, atol=1e-14)
        assert np.abs(out[0:2, e, 1:]).max() <= 1e-13 * abs(w[1, e, 0])


def test_weno_weights_would_catch_plausible_slips():
    """The hand values above separate the reading from nearby mistakes: beta
    squared in place of (eps + beta), equal linear weights, or a dropped
    second-derivative term each move a limited mode by far more than the
    tolerance of the mode test."""
    own, left, right = CELLS[5], CELLS[4], CELLS[6]
    ref = weno_modes(own, left, right, 2)[0]
    c1 = [left[1] + 6 * left[2], own[1], right[1] - 6 * right[2]]
    c2 = [left[2], own[2], right[2]]
    gam, eps = (0.001, 0.998, 0.001), 1e-6

    def combine(wt):
        return sum(w_ * c for w_, c in zip(wt, c1)) / sum(wt)

    beta = [4 * a ** 2 + 156 * b ** 2 for a, b in zip(c1, c2)]
    slips = [
        combine([g / (eps + b ** 2) for g, b in zip(gam, beta)]),
        combine([(1 / 3) / (eps + b) ** 2 for b in beta]),
        combine([g / (eps + 4 * a ** 2 + 12 * b ** 2) ** 2 for g, a, b in zip(gam, c1, c2)]),
    ]
    for alt in slips:
        assert abs(alt - ref) > 1e-3 * abs(ref)


def acoustic_state(p, sign, amp=1e-6):
    """Rest state plus amp * (modes of CELLS) * r_sign, r_+- = (u +- a, H +- u a,
    Y_1, Y_2) at u = 0."""
    mech = H.inert_mechanism()
    rhoE, _, a, H_ = _rest_state(mech)
    r = np.array([sign * a, H_, 0.5, 0.5])
    n = len(CELLS)
    w = np.zeros((4, n, p + 1))
    w[1, :, 0] = rhoE
    w[2, :, 0] = RHO / 2
    w[3, :, 0] = RHO / 2
    w += amp * r[:, None, None] * CELLS[None, :, :p + 1]
    return mech, w


@pytest.mark.parametrize("sign", [+1, -1])
def test_indicator_flags_of_a_weak_acoustic_wave(sign):
    """A perturbation of relative amplitude ~1e-6 along one acoustic eigenvector
    flags the cells the minmod rule flags in that field alone; such a weak front
    stands far above the rounding guard."""
    mech, w = acoustic_state(2, sign)
    flags, _ = O.limit_sync(_wl(2), mech, w)
    assert flags.tolist() == FLAGS_P2


def test_rounding_noise_on_flat_data_flags_nothing():
    """Flat data with relative noise of 1e-14 on every mode (double rounding after
    a few operations) is below the guard: no cell is troubled and nothing
    changes."""
    mech, w = contact_state(2, cells=np.tile([0.6, 0.0, 0.0], (8, 1)))
    rng = np.random.default_rng(7)
    w = w * (1 + 1e-14 * rng.standard_normal(w.shape)) + 1e-14 * RHO * np.concatenate(
        [np.zeros((2, 8, 3)), rng.standard_normal((2, 8, 3))])
    flags, out = O.limit_sync(_wl(2), mech, w)
    assert flags.sum() == 0
    assert np.array_equal(out, w)


def test_limiter_off_reports_flags_but_keeps_the_state():
    mech, w = contact_state(2)
    flags, out = O.limit_sync(_wl(2, limiter=I.LIM_NONE), mech, w)
    assert flags.tolist() == FLAGS_P2
    assert np.array_equal(out, w)
