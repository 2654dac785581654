"""Whole-step arithmetic pin of the oracle: a few SSP-RK3 steps of the ADG
scheme on tiny periodic meshes (4-6 elements, p = 1-2, 2 PEs, CAA delays with
the AT flux of Eq. 7 in use), against an independent restatement of the same
scheme in 50-digit arithmetic (mpmath), to 1e-14 in the parity scales.

The restatement is written from the paper and the readings, not from the oracle:
- the p+1 Gauss-Legendre points are roots of P_{p+1} found by Newton's method in
  50 digits, the weights 2 / ((1 - x^2) P'_{p+1}(x)^2);
- the AT weights c_m(k) solve the moment conditions of Eq. (8) as a linear
  system, sum_m c_m (-(k+m))^l = delta_l0 for l = 0..o-1;
- Eq. (5): dw_i/dt = (2i+1)/dx [sum_q w_q f(xi_q) P_i'(xi_q) - fhat_{e+1}
  + (-1)^i fhat_e] + (2i+1)/2 sum_q w_q s(xi_q) P_i(xi_q), local Lax-Friedrichs
  faces, at delayed PE faces the AT sum of the fluxes of both traces at the
  common levels n-k-m of the same stage (Sec. 3.2);
- T in closed form from the internal energy (constant c_p), the reversible mass
  action with K_c from the Gibbs energies and clipped concentrations (Sec. 2);
- CAA delays k = n mod (d+1), synchronous until the ring holds level n-k-(o-1)
  (Sec. 4.1); SSP-RK3 in Shu-Osher form.
The oracle's double rounding over these steps stays near 1e-15 of each
variable's scale; a wrong index, sign or term anywhere moves the result by far
more."""
import numpy as np
import pytest

import oracle as O
from paper_2501_01747_gb300 import inputs as I
from tests import helpers as H

mpmath = pytest.importorskip("mpmath")
mp = mpmath.mp
RU, TREF, PATM = "8.314462618", "298.15", "101325"


def gauss_mp(Q):
    xs, ws = [], []
    for i in range(1, Q + 1):
        x = mpmath.cos(mpmath.pi * (i - mpmath.mpf(1) / 4) / (Q + mpmath.mpf(1) / 2))
        x = mpmath.findroot(lambda t: mpmath.legendre(Q, t), x)
        dP = Q * (x * mpmath.legendre(Q, x) - mpmath.legendre(Q - 1, x)) / (x * x - 1)
        xs.append(x)
        ws.append(2 / ((1 - x * x) * dP * dP))
    return xs, ws


def dlegendre(j, x):
    if j == 0:
        return mpmath.mpf(0)
    return j * (x * mpmath.legendre(j, x) - mpmath.legendre(j - 1, x)) / (x * x - 1)


def at_weights(o, k):
    A = mpmath.matrix(o, o)
    b = mpmath.matrix(o, 1)
    for l in range(o):
        for m in range(o):
            A[l, m] = mpmath.mpf(-(k + m)) ** l
        b[l] = 1 if l == 0 else 0
    c = mpmath.lu_solve(A, b)
    return [c[m] for m in range(o)]


class Scheme:
    """The ADG scheme in mpmath for one instance (limiter off, LF flux)."""

    def __init__(self, wl, mech):
        self.wl, self.ns, self.nr = wl, mech.ns, mech.nr
        self.nv, self.Q, self.N = mech.ns + 2, wl.p + 1, wl.n_elem
        f = mpmath.mpf
        self.W = [f(x) for x in mech.W]
        self.cp = [f(x) for x in mech.cp]
        self.hf = [f(x) for x in mech.h_f]
        self.s0 = [f(x) for x in mech.s0]
        self.A = [f(x) for x in mech.A]
        self.b = [f(x) for x in mech.b]
        self.Ea = [f(x) for x in mech.Ea]
        self.nuf = mech.nu_f.astype(int).tolist()
        self.nur = mech.nu_r.astype(int).tolist()
        self.R, self.Tref, self.Patm = f(RU), f(TREF), f(PATM)
        self.dx = f(wl.length) / wl.n_elem
        self.dt = f(wl.dt)
        self.xq, self.wq = gauss_mp(self.Q)
        self.Pq = [[mpmath.legendre(j, x) for j in range(self.Q)] for x in self.xq]
        self.dPq = [[dlegendre(j, x) for j in range(self.Q)] for x in self.xq]
        # PE faces: PE q owns [floor(qN/P), floor((q+1)N/P)); PE face q lies
        # between PE q and PE q+1 (periodic: the last one wraps to face 0)
        P = wl.n_pe
        self.face_pf = {}
        for q in range(P):
            first_next = ((q + 1) % P) * self.N // P
            self.face_pf[first_next] = q
        self.ring = {}  # (level, stage, pe face) -> (left trace, right trace)

    def thermo(self, w):
        r = w[2:]
        rho = sum(r)
        u = w[0] / rho
        rhoe = w[1] - w[0] * u / 2
        T = (rhoe - sum(ri * (h - c * self.Tref) / Wi for ri, h, c, Wi in
                        zip(r, self.hf, self.cp, self.W))) / sum(
            ri * (c - self.R) / Wi for ri, c, Wi in zip(r, self.cp, self.W))
        Rm = sum(ri * self.R / Wi for ri, Wi in zip(r, self.W))
        cpm = sum(ri * c / Wi for ri, c, Wi in zip(r, self.cp, self.W))
        cvm = sum(ri * (c - self.R) / Wi for ri, c, Wi in zip(r, self.cp, self.W))
        P = T * Rm
        a = mpmath.sqrt(cpm / cvm * P / rho)
        return rho, u, T, P, a

    def flux(self, w):
        rho, u, T, P, a = self.thermo(w)
        return [w[0] * u + P, u * (w[1] + P)] + [u * x for x in w[2:]], u, a

    def lf(self, wl_, wr_):
        fl, ul, al = self.flux(wl_)
        fr, ur, ar = self.flux(wr_)
        lam = max(abs(ul) + al, abs(ur) + ar)
        return [(fl[v] + fr[v] - lam * (wr_[v] - wl_[v])) / 2 for v in range(self.nv)]

    def source(self, w, T):
        conc = [max(x, 0) / Wi for x, Wi in zip(w[2:], self.W)]
        wdot = [mpmath.mpf(0)] * self.ns
        for j in range(self.nr):
            kf = self.A[j] * T ** self.b[j] * mpmath.exp(-self.Ea[j] / (self.R * T))
            dG, dnu = 0, 0
            for i in range(self.ns):
                nu = self.nur[j][i] - self.nuf[j][i]
                h = self.hf[i] + self.cp[i] * (T - self.Tref)
                s = self.s0[i] + self.cp[i] * mpmath.log(T / self.Tref)
                dG += nu * (h - T * s)
                dnu += nu
            Kc = mpmath.exp(-dG / (self.R * T)) * (self.Patm / (self.R * T)) ** dnu
            fwd, rev = kf, kf / Kc
            for i in range(self.ns):
                fwd *= conc[i] ** self.nuf[j][i]
                rev *= conc[i] ** self.nur[j][i]
            for i in range(self.ns):
                wdot[i] += (self.nur[j][i] - self.nuf[j][i]) * (fwd - rev)
        return [mpmath.mpf(0), mpmath.mpf(0)] + [Wi * x for Wi, x in zip(self.W, wdot)]

    def trace(self, we, side):
        """w(+1) of element modes we (side 1) or w(-1) (side 0), per variable."""
        return [sum(we[v][j] * (1 if side == 1 else (-1) ** j) for j in range(self.Q))
                for v in range(self.nv)]

    def rhs(self, w, n, s, delays):
        nv, Q, N = self.nv, self.Q, self.N
        o = self.wl.at_order
        fh = []
        for i in range(N):  # face i: left element i-1 (periodic), right element i
            el, er = (i - 1) % N, i
            pf = self.face_pf.get(i)
            k = delays.get(pf, 0) if pf is not None else 0
            if k > 0:
                c = at_weights(o, k)
                acc = [mpmath.mpf(0)] * nv
                for m in range(o):
                    tl, tr = self.ring[(n - k - m, s, pf)]
                    fa = self.lf(tl, tr)
                    acc = [x + c[m] * y for x, y in zip(acc, fa)]
                fh.append(acc)
            else:
                fh.append(self.lf(self.trace(w[el], 1), self.trace(w[er], 0)))
        out = []
        for e in range(N):
            V = [[mpmath.mpf(0)] * Q for _ in range(nv)]
            S = [[mpmath.mpf(0)] * Q for _ in range(nv)]
            for q in range(Q):
                wn = [sum(w[e][v][j] * self.Pq[q][j] for j in range(Q)) for v in range(nv)]
                f, _, _ = self.flux(wn)
                T = self.thermo(wn)[2]
                src = self.source(wn, T)
                for v in range(nv):
                    for i in range(Q):
                        V[v][i] += self.wq[q] * f[v] * self.dPq[q][i]
                        S[v][i] += self.wq[q] * src[v] * self.Pq[q][i]
            fr, fl = fh[(e + 1) % N], fh[e]
            out.append([[(2 * i + 1) / self.dx * (V[v][i] - fr[v] + (-1) ** i * fl[v]) +
                         (2 * i + 1) * S[v][i] / 2 for i in range(Q)] for v in range(nv)])
        return out

    def step(self, w, n):
        d, o = self.wl.max_delay, self.wl.at_order
        delays = {}
        for pf in range(self.wl.n_pe):
            k = n % (d + 1)
            delays[pf] = k if n >= k + o - 1 else 0
        w0, win = w, w
        for s in range(3):
            # the stage input's traces at the PE faces go to the history ring
            for face, pf in self.face_pf.items():
                self.ring[(n, s, pf)] = (self.trace(win[(face - 1) % self.N], 1),
                                         self.trace(win[face], 0))
            L = self.rhs(win, n, s, delays)
            nxt = []
            for e in range(self.N):
                rows = []
                for v in range(self.nv):
                    row = []
                    for i in range(self.Q):
                        a0, a, r = w0[e][v][i], win[e][v][i], L[e][v][i]
                        if s == 0:
                            row.append(a0 + self.dt * r)
                        elif s == 1:
                            row.append(a0 * 3 / 4 + (a + self.dt * r) / 4)
                        else:
                            row.append(a0 / 3 + 2 * (a + self.dt * r) / 3)
                    rows.append(row)
                nxt.append(rows)
            win = nxt
        return win


def _case(p, n_elem, max_delay):
    base = I.load_workloads()["ignition-5sp-200x3"]
    mech = base.mechanism()
    wl = H.workload(n_elem, p, n_pe=2, length=0.002, dt=2e-9, delay_mode=I.DELAY_CAA,
                    max_delay=max_delay, ns=mech.ns, nr=mech.nr)
    # smooth primitive data at the Gauss points, projected in 50 digits
    mp.dps = 50
    xq, wq = gauss_mp(p + 1)
    Y = I.composition(mech, 0.02)
    Y = Y + 1e-3 * np.arange(1, mech.ns + 1) / mech.ns
    Y = Y / Y.sum()
    w = np.zeros((mech.ns + 2, n_elem, p + 1))
    dx = wl.length / n_elem
    for e in range(n_elem):
        pts = []
        for x in xq:
            xx = (e + (float(x) + 1) / 2) * dx / wl.length
            T = 1150.0 + 150.0 * np.sin(2 * np.pi * xx)
            P = I.P_ATM * (1 + 0.05 * np.cos(2 * np.pi * xx))
            u = 30.0 * np.sin(4 * np.pi * xx)
            pts.append(O.cons_from_prim(mech, T, P, u, Y))
        for v in range(mech.ns + 2):
            for j in range(p + 1):
                w[v, e, j] = float(sum(wq[q] * pts[q][v] * mpmath.legendre(j, xq[q])
                                       for q in range(p + 1)) * (2 * j + 1) / 2)
    return wl, mech, w


def _scales(w, mech):
    """Parity scales: momentum max rho (|u| + a) (a from the frozen gamma), energy
    max |rho E|, partial densities max(max rho Y_i, 1e-5 max rho)."""
    sc = np.abs(w).max(axis=(1, 2))
    rho = w[2:, :, 0].sum(0)
    sc[0] = max(sc[0], float((rho * 1000.0).max()))
    sc[2:] = np.maximum(sc[2:], 1e-5 * rho.max())
    return sc


@pytest.mark.parametrize("p,n_elem,max_delay,n_steps", [(1, 4, 1, 5), (2, 6, 2, 6)])
def test_steps_match_a_50_digit_restatement(p, n_elem, max_delay, n_steps):
    wl, mech, w = _case(p, n_elem, max_delay)
    o = O.Oracle(wl, mech)
    o.set_state(w)
    o.step(n_steps)
    got = o.state()
    mp.dps = 50
    sch = Scheme(wl, mech)
    wm = [[[mpmath.mpf(float(w[v, e, j])) for j in range(p + 1)] for v in range(mech.ns + 2)]
          for e in range(n_elem)]
    used = set()
    for n in range(n_steps):
        k = n % (max_delay + 1)
        if n >= k + wl.at_order - 1 and k > 0:
            used.add(k)
        wm = sch.step(wm, n)
    assert used, "the AT flux at a delayed PE face was never exercised"
    ref = np.array([[[float(wm[e][v][j]) for j in range(p + 1)] for e in range(n_elem)]
                    for v in range(mech.ns + 2)])
    assert not np.allclose(ref, w, rtol=1e-6)   # the state did move
    err = (np.abs(got - ref).max(axis=(1, 2)) / _scales(ref, mech))
    assert err.max() <= 1e-14, err
