"""Seeded synthetic inputs for the 1D reacting-Euler ADG hot path.

This module only draws random numbers and does bookkeeping on them. It holds none
of the scheme's arithmetic (no thermodynamics, no rates, no DG operators), so the
oracle and the CUDA path can both take their inputs from it without sharing any of
the computation they are compared on.

What it produces:

* ``make_mechanism``: a synthetic, element-balanced, reversible mechanism in the
  shape of the detailed mechanisms of Sec. 5 (species with molecular weight,
  constant molar heat capacity, formation enthalpy and standard entropy; reactions
  with integer stoichiometry and Arrhenius parameters A, b, E_a).
* ``primitive_ic``: initial primitive fields (T, P, u, Y_1..Y_Ns) sampled at the
  Gauss-Legendre points of every element, for the auto-ignition (Sec. 5.1) and
  detonation (Sec. 5.2) shapes.
* ``Workload``: one named configuration (mesh, PEs, delays, flux, limiter, dt).

Units are SI throughout (kg/mol, J/mol/K, J/mol, m, s), except the Arrhenius
pre-exponential factor, which is drawn in cm-mol-s units and converted by the
reaction order (see ``make_mechanism``).
"""
from __future__ import annotations

import dataclasses
import itertools
import json
import os
from typing import Optional, Sequence

import numpy as np

# Pseudo-element masses (kg/mol): an "H"-like, a "C"-like, an "O"-like and an
# "N"-like element.  Species are count vectors over these elements.
ELEMENT_MASS = np.array([1.008e-3, 12.011e-3, 15.999e-3, 14.007e-3])

P_ATM = 101325.0
KCAL = 4184.0

# Boundary and option codes, mirroring include/adg.h.
BC_PERIODIC, BC_REFLECT, BC_OUTFLOW = 0, 1, 2
FLUX_LF, FLUX_HLLC = 0, 1
LIM_NONE, LIM_WENO = 0, 1
DELAY_SYNC, DELAY_CAA, DELAY_SAA = 0, 1, 2
# time integrators: SSP-RK3 (Shu-Osher), and the low-storage explicit RK schemes
# of Sec. 3.1 (Williamson's 3-stage 3rd order, Carpenter-Kennedy 5-stage 4th order)
RK_SSP3, RK_LS3, RK_LS4 = 0, 1, 2

# Delay probability sets of Sec. 4.2 (SAA), for a maximum delay of 2 (three bins).
SAA_SETS = {1: (0.3, 0.4, 0.3), 2: (0.5, 0.3, 0.2), 3: (0.8, 0.1, 0.1)}


@dataclasses.dataclass
class Mechanism:
    """Arrays in the layout of ``adg_mechanism`` (include/adg.h)."""
    W: np.ndarray        # [ns] kg/mol
    cp: np.ndarray       # [ns] J/mol/K (constant)
    h_f: np.ndarray      # [ns] J/mol at 298.15 K
    s0: np.ndarray       # [ns] J/mol/K at 298.15 K and 1 atm
    nu_f: np.ndarray     # [nr, ns] int8 reactant coefficients
    nu_r: np.ndarray     # [nr, ns] int8 product coefficients
    A: np.ndarray        # [nr] SI: (m^3/mol)^(order-1)/s
    b: np.ndarray        # [nr] temperature exponent
    Ea: np.ndarray       # [nr] J/mol
    comp: np.ndarray     # [ns, 4] element counts (bookkeeping only)
    names: list
    Le: Optional[np.ndarray] = None  # [ns] Lewis numbers (viscous runs; None: all 1)

    @property
    def ns(self) -> int:
        return int(self.W.shape[0])

    @property
    def nr(self) -> int:
        return int(self.A.shape[0])


def _species_pool(max_atoms: int) -> list:
    """All element-count vectors over the three reactive pseudo-elements with
    1..max_atoms atoms in total (the fourth, "N"-like element only forms the
    inert bath gas)."""
    pool = []
    for c in itertools.product(range(max_atoms + 1), repeat=3):
        n = sum(c)
        if 1 <= n <= max_atoms:
            pool.append((c[0], c[1], c[2], 0))
    return pool


def _candidate_reactions(comp: np.ndarray, reactive: Sequence[int]) -> list:
    """Every element-balanced reaction of the forms A <=> B + C, A + B <=> C + D
    and A + B <=> C among the reactive species (a species may appear twice).
    Returned as (reactants, products) tuples of species indices, one per
    unordered reaction, in a deterministic order."""
    sides = [(i,) for i in reactive]
    sides += [(i, j) for i, j in itertools.combinations_with_replacement(reactive, 2)]
    groups = {}
    for s in sides:
        key = tuple(int(x) for x in comp[list(s)].sum(axis=0))
        groups.setdefault(key, []).append(s)
    out = []
    for key in sorted(groups):
        g = groups[key]
        for a, b in itertools.combinations(g, 2):
            if len(a) == 1 and len(b) == 1:
                continue
            out.append((a, b))
    return out


def make_mechanism(ns: int, nr: int, seed: int,
                   attempts: Optional[Sequence[int]] = None) -> Mechanism:
    """Draw a synthetic reversible mechanism with ``ns`` species and ``nr`` reactions.

    Distributions (the workload recipe): per-species constant c_p ~ U[20, 40]
    J/mol/K; formation enthalpy h_f ~ U[-300, 300] kJ/mol (0 for the fuel, the
    oxidiser and the bath gas); standard entropy s0 = 100 + 30 n_atoms + U[0, 40]
    J/mol/K (so that association reactions lose about one molecule's translational
    entropy); per reaction A log-uniform in [1e8, 1e14] (cm-mol-s units, converted
    to SI by multiplying with 1e-6^(order-1)), b ~ U[-1, 1], E_a ~ U[0, 40]
    kcal/mol.  Species 0 is the fuel, species 1 the oxidiser and species ns-1 the
    bath gas, which is an inert N2-like molecule when ns >= 9 (with fewer species
    every species has to react for ns-1 distinct reactions to exist, so the bath gas
    is then drawn like the others).  Every reaction is element-balanced and written in its
    exothermic direction (sum of nu * h_f <= 0).

    ``attempts[j]`` selects which of reaction j's independent (A, b, E_a) draws is
    used; 0 everywhere is the plain draw.  A workload may store other attempt
    numbers to drop draws that are too stiff for the explicit time step.
    """
    if ns < 4 or nr < 1:
        raise ValueError("need ns >= 4 and nr >= 1")
    pool = _species_pool(4 if ns < 12 else 6)
    inert_bath = ns >= 9
    for tries in range(10000):
        rng = np.random.default_rng([seed, 1, tries])
        # fuel: hydrogen-rich; oxidiser: O2-like; bath: N2-like (inert)
        fuel = (2, 0, 0, 0) if ns < 12 else tuple(int(v) for v in rng.choice([(2, 0, 0, 0), (4, 1, 0, 0)]))
        ox = (0, 0, 2, 0)
        others = [c for c in pool if c not in (fuel, ox)]
        if ns < 12:
            others = [c for c in others if c[1] == 0]
        if inert_bath:
            pick = rng.choice(len(others), size=ns - 3, replace=False)
            comp = np.array([fuel, ox] + [others[i] for i in pick] + [(0, 0, 0, 2)],
                            dtype=np.int64)
            reactive = list(range(ns - 1))
        else:
            pick = rng.choice(len(others), size=ns - 2, replace=False)
            comp = np.array([fuel, ox] + [others[i] for i in pick], dtype=np.int64)
            reactive = list(range(ns))
        cands = _candidate_reactions(comp, reactive)
        if len(cands) < nr:
            continue
        order = rng.permutation(len(cands))
        chosen = [cands[i] for i in order[:nr]]
        used = set()
        for l, r in chosen:
            used.update(l)
            used.update(r)
        if 0 not in used or 1 not in used:
            continue
        break
    else:  # pragma: no cover
        raise RuntimeError("could not draw a mechanism")

    W = comp @ ELEMENT_MASS
    cp = rng.uniform(20.0, 40.0, size=ns)
    h_f = rng.uniform(-300e3, 300e3, size=ns)
    h_f[[0, 1, ns - 1]] = 0.0
    n_atoms = comp.sum(axis=1)
    s0 = 100.0 + 30.0 * n_atoms + rng.uniform(0.0, 40.0, size=ns)

    nu_f = np.zeros((nr, ns), dtype=np.int8)
    nu_r = np.zeros((nr, ns), dtype=np.int8)
    A = np.zeros(nr)
    b = np.zeros(nr)
    Ea = np.zeros(nr)
    for j, (lhs, rhs) in enumerate(chosen):
        dh = sum(h_f[i] for i in rhs) - sum(h_f[i] for i in lhs)
        if dh > 0.0:
            lhs, rhs = rhs, lhs
        for i in lhs:
            nu_f[j, i] += 1
        for i in rhs:
            nu_r[j, i] += 1
        att = 0 if attempts is None else int(attempts[j])
        prng = np.random.default_rng([seed, 2, j, att])
        order_f = int(nu_f[j].sum())
        A_cgs = 10.0 ** prng.uniform(8.0, 14.0)
        A[j] = A_cgs * (1e-6) ** (order_f - 1)
        b[j] = prng.uniform(-1.0, 1.0)
        Ea[j] = prng.uniform(0.0, 40.0) * KCAL
    names = ["fuel", "oxid"] + ["s%d" % i for i in range(2, ns - 1)] + ["bath"]
    return Mechanism(W=W, cp=cp, h_f=h_f, s0=s0, nu_f=nu_f, nu_r=nu_r, A=A, b=b,
                     Ea=Ea, comp=comp, names=names, Le=lewis_numbers(W))


def lewis_numbers(W: np.ndarray) -> np.ndarray:
    """Synthetic Lewis numbers (the paper's mixture-averaged transport comes from
    Cantera, not available): Le_i = sqrt(W_i / 0.029), which puts a light fuel
    near 0.26, water-like species near 0.8 and the bath gas near 1."""
    return np.sqrt(np.asarray(W, dtype=np.float64) / 0.029)


def gauss_points(q: int) -> np.ndarray:
    """Gauss-Legendre points on [-1, 1] (numpy's library routine), used only to
    place the initial-condition samples."""
    x, _ = np.polynomial.legendre.leggauss(q)
    return x


@dataclasses.dataclass
class Workload:
    """One configuration of the hot path (the fields of ``adg_config``)."""
    name: str
    n_elem: int
    p: int
    n_pe: int
    length: float
    dt: float
    bc_left: int
    bc_right: int
    flux: int
    limiter: int
    at_order: int
    delay_mode: int
    max_delay: int
    delay_probs: tuple
    seed: int
    ns: int
    nr: int
    mech_seed: int
    ic_seed: int
    ic_kind: str
    ic_params: dict
    n_steps: int
    tvb_M: float = 0.0
    x0: float = 0.0
    attempts: Optional[list] = None
    integrator: int = RK_SSP3
    # diffusive flux of Sec. 2 (LDG), with the synthetic transport model
    # mu = mu_ref (T / T_mu)^mu_exp, k = mu cp / Pr, D_i = k / (rho cp Le_i)
    viscous: int = 0
    mu_ref: float = 1.85e-5
    T_mu: float = 300.0
    mu_exp: float = 0.7
    prandtl: float = 0.7
    # subdomain of PEs [pe_begin, pe_end) of the domain above (pe_end = 0: whole)
    pe_begin: int = 0
    pe_end: int = 0

    def mechanism(self) -> Mechanism:
        return make_mechanism(self.ns, self.nr, self.mech_seed, self.attempts)

    def nodes_x(self) -> np.ndarray:
        """Physical x of every Gauss point, [n_elem, p+1]."""
        dx = self.length / self.n_elem
        xi = gauss_points(self.p + 1)
        xc = self.x0 + (np.arange(self.n_elem) + 0.5) * dx
        return xc[:, None] + 0.5 * dx * xi[None, :]

    def primitive(self, mech: Optional[Mechanism] = None) -> np.ndarray:
        return primitive_ic(self, mech or self.mechanism())


def composition(mech: Mechanism, y_fuel: float, y_ox: float = 0.2) -> np.ndarray:
    """Premixed composition: fuel, oxidiser, the rest bath gas."""
    Y = np.zeros(mech.ns)
    Y[0] = y_fuel
    Y[1] = y_ox
    Y[-1] = 1.0 - y_fuel - y_ox
    return Y


def primitive_ic(wl: Workload, mech: Mechanism) -> np.ndarray:
    """Initial primitive fields at the Gauss points, layout [ns+3][n_elem][p+1]:
    rows T (K), P (Pa), u (m/s), Y_1..Y_ns.

    ``ignition_gauss``: uniform T0 and P with a Gaussian hot spot of +dT at a seeded
    centre, width sigma = 5 % of the domain (Sec. 5.1 shape).
    ``ignition_sine``: T = T0 (1 + amp sin(2 pi x / L + phi)) with a seeded phase.
    ``detonation``: a driver region x < frac L at (P_hi, T_hi) next to an ambient
    (P_lo, T_lo) mixture, at rest (Sec. 5.2 shape).
    ``advection``: reactions frozen in practice (the caller passes an inert
    mechanism); density wave rho = rho0 (1 + amp sin(2 pi x / L)) at uniform P, u.
    """
    rng = np.random.default_rng([wl.ic_seed, 3])
    x = wl.nodes_x()
    L = wl.length
    prm = wl.ic_params
    out = np.zeros((mech.ns + 3, wl.n_elem, wl.p + 1))
    y_fuel = prm.get("y_fuel", 0.02)
    Y = composition(mech, y_fuel, prm.get("y_ox", 0.2))
    kind = wl.ic_kind
    if kind == "ignition_gauss":
        xc = wl.x0 + L * rng.uniform(0.35, 0.65)
        sig = 0.05 * L
        T = prm["T0"] + prm.get("dT", 300.0) * np.exp(-((x - xc) ** 2) / (2 * sig * sig))
        P = np.full_like(x, prm.get("P0", P_ATM))
        u = np.full_like(x, prm.get("u0", 0.0))
    elif kind == "ignition_sine":
        phi = rng.uniform(0.0, 2 * np.pi)
        T = prm["T0"] * (1.0 + prm.get("amp", 0.02) * np.sin(2 * np.pi * (x - wl.x0) / L + phi))
        P = np.full_like(x, prm.get("P0", P_ATM))
        u = np.full_like(x, prm.get("u0", 0.0))
    elif kind == "detonation":
        hi = (x - wl.x0) < prm.get("frac", 0.05) * L
        T = np.where(hi, prm.get("T_hi", 3000.0), prm.get("T_lo", 300.0))
        P = np.where(hi, prm.get("P_hi", 30 * P_ATM), prm.get("P_lo", P_ATM))
        u = np.zeros_like(x)
    elif kind == "advection":
        # T chosen so that P is uniform while the density varies: T ~ 1/rho.
        amp = prm.get("amp", 0.2)
        T = prm["T0"] / (1.0 + amp * np.sin(2 * np.pi * (x - wl.x0) / L))
        P = np.full_like(x, prm.get("P0", P_ATM))
        u = np.full_like(x, prm.get("u0", 50.0))
    else:
        raise ValueError(kind)
    out[0] = T
    out[1] = P
    out[2] = u
    out[3:] = Y[:, None, None]
    return out


# --------------------------------------------------------------------------
# Named workloads.  dt and the per-reaction attempt numbers are stored inputs,
# written by oracle/make_workloads.py (which evaluates stability with the
# oracle) into workloads.json beside this file.
# --------------------------------------------------------------------------

_HERE = os.path.dirname(os.path.abspath(__file__))
WORKLOADS_JSON = os.path.join(_HERE, "workloads.json")

SEED_MECH, SEED_IC, SEED_DELAY = 2501017470, 2501017480, 2501017490


def base_workloads() -> dict:
    """The five configurations of the hot path, before dt is fixed.

    ignition-5sp-200x3: 5 species / 4 reactions, 200 elements, p=3, 4 PEs, max delay 2.
    ignition-9sp-4096x4: 9 / 21, 4096 elements, p=4, 64 PEs, max delay 4.
    detonation-9sp-16384x3: 9 / 21, 16384 elements, p=3, 256 PEs, max delay 3, WENO.
    ensemble-9sp-512: 512 ignition instances, sizes U[256, 8192], p in {2, 3, 4}.
    detonation-53sp-65536x3: 53 / 325, 65536 elements, p=3, 1024 PEs, max delay 4.
    """
    u3 = lambda d: tuple([1.0 / (d + 1)] * (d + 1))
    w = {}
    w["ignition-5sp-200x3"] = Workload(
        name="ignition-5sp-200x3", n_elem=200, p=3, n_pe=4, length=0.01, dt=0.0,
        bc_left=BC_PERIODIC, bc_right=BC_PERIODIC, flux=FLUX_LF, limiter=LIM_WENO,
        at_order=4, delay_mode=DELAY_SAA, max_delay=2, delay_probs=SAA_SETS[1],
        seed=SEED_DELAY + 0, ns=5, nr=4, mech_seed=SEED_MECH + 0, ic_seed=SEED_IC + 0,
        ic_kind="ignition_gauss", ic_params={"T0": 900.0, "dT": 300.0, "y_fuel": 0.02},
        n_steps=500)
    w["ignition-9sp-4096x4"] = Workload(
        name="ignition-9sp-4096x4", n_elem=4096, p=4, n_pe=64, length=0.01, dt=0.0,
        bc_left=BC_PERIODIC, bc_right=BC_PERIODIC, flux=FLUX_LF, limiter=LIM_WENO,
        at_order=5, delay_mode=DELAY_SAA, max_delay=4, delay_probs=u3(4),
        seed=SEED_DELAY + 1, ns=9, nr=21, mech_seed=SEED_MECH + 1, ic_seed=SEED_IC + 1,
        ic_kind="ignition_sine", ic_params={"T0": 1000.0, "amp": 0.02, "y_fuel": 0.015},
        n_steps=500)
    w["detonation-9sp-16384x3"] = Workload(
        name="detonation-9sp-16384x3", n_elem=16384, p=3, n_pe=256, length=0.2, dt=0.0,
        bc_left=BC_REFLECT, bc_right=BC_OUTFLOW, flux=FLUX_HLLC, limiter=LIM_WENO,
        at_order=4, delay_mode=DELAY_SAA, max_delay=3, delay_probs=u3(3),
        seed=SEED_DELAY + 2, ns=9, nr=21, mech_seed=SEED_MECH + 2, ic_seed=SEED_IC + 2,
        ic_kind="detonation", ic_params={"frac": 0.05, "P_hi": 30 * P_ATM, "T_hi": 3000.0,
                                         "P_lo": P_ATM, "T_lo": 300.0, "y_fuel": 0.02},
        n_steps=500)
    w["detonation-53sp-65536x3"] = Workload(
        name="detonation-53sp-65536x3", n_elem=65536, p=3, n_pe=1024, length=0.2, dt=0.0,
        bc_left=BC_REFLECT, bc_right=BC_OUTFLOW, flux=FLUX_HLLC, limiter=LIM_WENO,
        at_order=4, delay_mode=DELAY_SAA, max_delay=4, delay_probs=u3(4),
        seed=SEED_DELAY + 4, ns=53, nr=325, mech_seed=SEED_MECH + 4, ic_seed=SEED_IC + 4,
        ic_kind="detonation", ic_params={"frac": 0.05, "P_hi": 30 * P_ATM, "T_hi": 3000.0,
                                         "P_lo": P_ATM, "T_lo": 300.0, "y_fuel": 0.02},
        n_steps=500)
    return w


def ensemble_workloads(n_instances: int = 512, seed: int = SEED_IC + 3,
                       path: str = WORKLOADS_JSON) -> list:
    """The batched ensemble: independent ignition instances sharing one 9-species
    mechanism, N_E ~ U[256, 8192], p ~ U{2, 3, 4}, T0 ~ U[900, 1200] K,
    Y_fuel ~ U[0.008, 0.025]; 64 elements per PE, max delay 3."""
    rng = np.random.default_rng([seed, 4])
    out = []
    for i in range(n_instances):
        ne = int(rng.integers(256, 8193))
        p = int(rng.integers(2, 5))
        T0 = float(rng.uniform(900.0, 1200.0))
        yf = float(rng.uniform(0.008, 0.025))
        npe = max(1, ne // 64)
        out.append(Workload(
            name="ensemble-%d" % i, n_elem=ne, p=p, n_pe=npe, length=0.01, dt=0.0,
            bc_left=BC_PERIODIC, bc_right=BC_PERIODIC, flux=FLUX_LF, limiter=LIM_WENO,
            at_order=p + 1, delay_mode=DELAY_SAA, max_delay=3,
            delay_probs=tuple([0.25] * 4), seed=SEED_DELAY + 3 + 1000 * i, ns=9, nr=21,
            mech_seed=SEED_MECH + 3, ic_seed=SEED_IC + 3 + 1000 * i,
            ic_kind="ignition_gauss", ic_params={"T0": T0, "dT": 300.0, "y_fuel": yf},
            n_steps=500))
    if os.path.exists(path):
        with open(path) as f:
            stored = json.load(f).get("ensemble")
        if stored:
            for i, wl in enumerate(out):
                if i < len(stored["dt"]):
                    wl.dt = float(stored["dt"][i])
                wl.attempts = stored["attempts"]
    return out


def load_workloads(path: str = WORKLOADS_JSON) -> dict:
    """Base workloads with the stored dt and attempt numbers applied."""
    w = base_workloads()
    if os.path.exists(path):
        with open(path) as f:
            stored = json.load(f)
        for name, rec in stored.get("workloads", {}).items():
            if name in w:
                w[name].dt = float(rec["dt"])
                w[name].attempts = rec.get("attempts")
    return w


def viscous(wl: Workload, **kw) -> Workload:
    """The viscous variant of a workload (the diffusive flux with the synthetic
    transport model). The explicit diffusive limit of DG scales like
    dx^2 / (nu (p+1)^4): on the ignition meshes (dx = 2.4 um) the workload's dt
    is stable for p <= 3, and p = 4 needs dt/8 (found with the oracle: dt and
    dt/2 blow up, dt/4 grows slowly, dt/8 stays flat over 2000 steps)."""
    w = dataclasses.replace(wl, viscous=1, **kw)
    if w.p >= 4 and "dt" not in kw:
        w.dt = wl.dt / 8
    return w


def scaled(wl: Workload, n_elem: int, n_pe: int, name: Optional[str] = None) -> Workload:
    """The same workload on fewer elements (for tests): the element size and dt
    are kept and the domain shrinks in proportion."""
    w = dataclasses.replace(wl)
    w.length = wl.length * n_elem / wl.n_elem
    w.n_elem = n_elem
    w.n_pe = n_pe
    w.name = name or (wl.name + "-%d" % n_elem)
    return w
