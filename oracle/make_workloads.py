"""Write paper_2501_01747_gb300/workloads.json: the time step of every workload and
the per-reaction draw numbers of its mechanism.

Both are stored inputs, computed here with the oracle only:

* dt_cfl = 0.4 dx / ((2p+1) s_ref), with s_ref the largest |u| + a over the
  initial Gauss points times a margin (1.5 for ignition, 2.5 for detonation,
  where the shocked gas moves and heats up).
* The AT flux extrapolates in time with weights that grow fast with the delay and
  the order (sum |c_m| = 49 for order 4 at delay 2, 769 for order 5 at delay 4),
  which shrinks the stable step. dt = dt_cfl * f / 2 with f the largest power of
  1/2 for which the workload, cut to a few hundred elements with the same element
  size, PE size and delays, runs a few hundred steps with bounded temperatures
  (and, for the smooth ignition cases, without a growing top mode).
* A reaction draw (A, b, E_a) is kept only if its explicit stiffness bound
  lambda_j dt stays below 0.25 over the workload's temperature range, with
  lambda_j = o_f k_f c^(o_f-1) + o_r k_r c^(o_r-1) and c the largest total molar
  concentration; otherwise the next independent draw of that reaction is taken.
  The summed bound per species must stay below 1 as well.

Run:  python oracle/make_workloads.py
"""
from __future__ import annotations

import json
import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(HERE))

import oracle as O  # noqa: E402
from paper_2501_01747_gb300 import inputs as I  # noqa: E402

RU = 8.314462618


def max_speed(wl, mech, prim, stride=1):
    s = 0.0
    for e in range(0, wl.n_elem, stride):
        for q in range(wl.p + 1):
            w = O.cons_from_prim(mech, prim[0, e, q], prim[1, e, q], prim[2, e, q],
                                 prim[3:, e, q])
            rho, u, T, P, a = O.state(mech, w)
            s = max(s, abs(u) + a)
    return s


def stiffness(mech, j, T_lo, T_hi, P_hi):
    lam = 0.0
    of = int(mech.nu_f[j].sum())
    orr = int(mech.nu_r[j].sum())
    for T in np.linspace(T_lo, T_hi, 24):
        c = P_hi / (RU * T)
        kf, Kc = O.rates(mech, T, j)
        lam = max(lam, kf * of * c ** (of - 1) + kf / Kc * orr * c ** (orr - 1))
    return lam


def accept(ns, nr, seed, dt, T_lo, T_hi, P_hi, kappa=0.25, kappa_sum=1.0):
    attempts = [0] * nr
    mech = I.make_mechanism(ns, nr, seed, attempts)
    lam = np.array([stiffness(mech, j, T_lo, T_hi, P_hi) for j in range(nr)])
    for it in range(200000):
        nu = (mech.nu_f.astype(int) + mech.nu_r.astype(int)) > 0
        per_species = (nu * lam[:, None]).sum(axis=0) * dt
        bad = np.where(lam * dt > kappa)[0]
        if len(bad) == 0:
            if per_species.max() <= kappa_sum:
                break
            i = int(np.argmax(per_species))
            js = np.where(nu[:, i])[0]
            bad = [int(js[np.argmax(lam[js])])]
        j = int(bad[0])
        attempts[j] += 1
        mech = I.make_mechanism(ns, nr, seed, attempts)
        lam[j] = stiffness(mech, j, T_lo, T_hi, P_hi)
    else:  # pragma: no cover
        raise RuntimeError("no acceptable mechanism")
    return attempts, float((lam * dt).max())


def stable_factor(wl, mech, n_steps, n_elem_small):
    """Largest f in {1, 1/2, 1/4, ...} for which the workload, cut down to
    n_elem_small elements with the same dx, PE size, AT order and delays, runs
    n_steps with dt * f without a non-physical state or a growing top mode."""
    small = I.scaled(wl, n_elem_small, max(1, wl.n_pe * n_elem_small // wl.n_elem))
    prim = I.primitive_ic(small, mech)
    smooth = wl.ic_kind.startswith("ignition")
    T_lo = prim[0].min()
    T_hi = 2.0 * prim[0].max() + 3000.0
    f = 1.0
    base = wl.dt
    while f > 1e-3:
        small.dt = base * f
        o = O.Oracle(small, mech)
        o.set_primitive(prim)
        ok = True
        try:
            o.step(n_steps)
            w = o.state()
            T = o.temperature()
            ok = bool(np.all(np.isfinite(w)) and T.min() > 0.5 * T_lo and T.max() < T_hi)
            if smooth:
                top = np.abs(w[1, :, -1]).max() / np.abs(w[1, :, 0]).min()
                ok = ok and bool(top < 1e-2)
        except RuntimeError:
            ok = False
        print("   %s f=%.4g %s" % (wl.name, f, "stable" if ok else "unstable"), flush=True)
        if ok:
            return f
        f *= 0.5
    raise RuntimeError("no stable dt")


def main():
    only = sys.argv[1:]
    path = os.path.join(os.path.dirname(HERE), "paper_2501_01747_gb300", "workloads.json")
    out = {"comment": "stored inputs written by oracle/make_workloads.py", "workloads": {}}
    if os.path.exists(path):
        with open(path) as f:
            out = json.load(f)
    W = I.base_workloads()
    small = {"ignition-5sp-200x3": (200, 500), "ignition-9sp-4096x4": (256, 400),
             "detonation-9sp-16384x3": (512, 400), "detonation-53sp-65536x3": (128, 150)}
    for name, wl in W.items():
        if only and name not in only:
            continue
        m0 = I.make_mechanism(wl.ns, wl.nr, wl.mech_seed)
        prim = I.primitive_ic(wl, m0)
        ign = wl.ic_kind.startswith("ignition")
        s = max_speed(wl, m0, prim, stride=max(1, wl.n_elem // 512))
        margin = 1.5 if ign else 2.5
        dx = wl.length / wl.n_elem
        dt = 0.4 * dx / ((2 * wl.p + 1) * s * margin)
        if ign:
            T_lo, T_hi, P_hi = 600.0, 3000.0, 4 * I.P_ATM
        else:
            T_lo, T_hi, P_hi = 250.0, 4500.0, 120 * I.P_ATM
        attempts, lmax = accept(wl.ns, wl.nr, wl.mech_seed, dt, T_lo, T_hi, P_hi)
        wl.dt = dt
        wl.attempts = attempts
        mech = wl.mechanism()
        ne_small, nst = small[name]
        f = stable_factor(wl, mech, nst, ne_small)
        out["workloads"][name] = {"dt": dt * f * 0.5, "dt_cfl": dt, "at_factor": f * 0.5,
                                  "attempts": attempts, "s_ref": s * margin,
                                  "lambda_dt_max": lmax}
        print(name, "dt %.4e" % (dt * f * 0.5), "max lambda*dt %.3f" % lmax,
              "redraws", sum(attempts), flush=True)
        with open(path, "w") as fh:
            json.dump(out, fh, indent=1)
    if only and "ensemble" not in only:
        return
    # ensemble: one shared mechanism, accepted at the largest instance dt; the AT
    # stability factor is searched once per polynomial degree
    ens = I.ensemble_workloads()
    m0 = I.make_mechanism(9, 21, I.SEED_MECH + 3)
    dts = []
    for wl in ens:
        prim = I.primitive_ic(wl, m0)
        s = max_speed(wl, m0, prim, stride=max(1, wl.n_elem // 64))
        dts.append(0.4 * (wl.length / wl.n_elem) / ((2 * wl.p + 1) * s * 1.5))
    attempts, lmax = accept(9, 21, I.SEED_MECH + 3, max(dts), 600.0, 3000.0, 4 * I.P_ATM)
    factors = {}
    for p in (2, 3, 4):
        i = next(k for k, wl in enumerate(ens) if wl.p == p)
        wl = ens[i]
        wl.dt = dts[i]
        wl.attempts = attempts
        factors[p] = stable_factor(wl, wl.mechanism(), 400, 256) * 0.5
    dts = [d * factors[wl.p] for d, wl in zip(dts, ens)]
    out["ensemble"] = {"dt": dts, "attempts": attempts, "lambda_dt_max": lmax,
                       "at_factor": {str(k): v for k, v in factors.items()}}
    print("ensemble", "dt range %.3e..%.3e" % (min(dts), max(dts)), "redraws", sum(attempts))
    with open(path, "w") as fh:
        json.dump(out, fh, indent=1)
    print("wrote", path)


if __name__ == "__main__":
    main()
