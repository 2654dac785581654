"""ctypes binding of the FP64 CPU oracle (adg_oracle.c).

TEST INFRASTRUCTURE ONLY: the test suite, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` use it to check and time the CUDA path.  The
product library never imports it.  ``build()`` compiles the C source with plain
gcc (-O2 -ffp-contract=off) into ``oracle/_build/libadg_oracle.so``.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "adg_oracle.c")
LIB = os.path.join(HERE, "_build", "libadg_oracle.so")


def build(force: bool = False) -> str:
    """Compile the oracle (a second or two) unless an up-to-date build exists."""
    os.makedirs(os.path.dirname(LIB), exist_ok=True)
    hdr = os.path.join(HERE, "adg_oracle.h")
    if (not force and os.path.exists(LIB)
            and os.path.getmtime(LIB) >= max(os.path.getmtime(SRC), os.path.getmtime(hdr))):
        return LIB
    tmp = LIB + ".tmp%d" % os.getpid()
    subprocess.check_call(["gcc", "-O2", "-ffp-contract=off", "-fPIC", "-shared",
                           "-std=c11", "-D_DEFAULT_SOURCE", "-o", tmp, SRC, "-lm"])
    os.replace(tmp, LIB)
    return LIB


class Mech(C.Structure):
    _fields_ = [("ns", C.c_int), ("nr", C.c_int),
                ("W", C.POINTER(C.c_double)), ("cp", C.POINTER(C.c_double)),
                ("hf", C.POINTER(C.c_double)), ("s0", C.POINTER(C.c_double)),
                ("nu_f", C.POINTER(C.c_byte)), ("nu_r", C.POINTER(C.c_byte)),
                ("A", C.POINTER(C.c_double)), ("b", C.POINTER(C.c_double)),
                ("Ea", C.POINTER(C.c_double)), ("Le", C.POINTER(C.c_double))]


class Cfg(C.Structure):
    _fields_ = [("n_elem", C.c_int), ("p", C.c_int), ("n_pe", C.c_int),
                ("x0", C.c_double), ("length", C.c_double), ("dt", C.c_double),
                ("bc_left", C.c_int), ("bc_right", C.c_int), ("flux", C.c_int),
                ("limiter", C.c_int), ("at_order", C.c_int), ("delay_mode", C.c_int),
                ("max_delay", C.c_int), ("delay_probs", C.POINTER(C.c_double)),
                ("seed", C.c_uint64), ("tvb_M", C.c_double), ("integrator", C.c_int),
                ("viscous", C.c_int), ("mu_ref", C.c_double), ("T_mu", C.c_double),
                ("mu_exp", C.c_double), ("prandtl", C.c_double), ("face0", C.c_int),
                ("pe_begin", C.c_int), ("pe_end", C.c_int)]


_lib = None


def lib():
    global _lib
    if _lib is None:
        _lib = C.CDLL(build())
        d = C.POINTER(C.c_double)
        _lib.or_create.restype = C.c_void_p
        _lib.or_create.argtypes = [C.POINTER(Cfg), C.POINTER(Mech)]
        _lib.or_destroy.argtypes = [C.c_void_p]
        for name in ("or_set_primitive", "or_set_state", "or_get_state", "or_get_temperature"):
            getattr(_lib, name).argtypes = [C.c_void_p, d]
        _lib.or_step.argtypes = [C.c_void_p, C.c_int]
        _lib.or_stage.argtypes = [C.c_void_p, C.c_int, C.c_int]
        ip = C.POINTER(C.c_int)
        _lib.or_part_layout.argtypes = [C.c_void_p, ip, ip, ip, ip]
        _lib.or_part_block.argtypes = [C.c_void_p, C.c_int, C.c_int, C.c_int, d, C.c_int]
        _lib.or_steps_done.restype = C.c_int64
        _lib.or_steps_done.argtypes = [C.c_void_p]
        _lib.or_get_flags.argtypes = [C.c_void_p, C.POINTER(C.c_uint8), C.POINTER(C.c_int32)]
        _lib.or_legendre.argtypes = [C.c_int, C.c_double, d, d]
        _lib.or_gauss.argtypes = [C.c_int, d, d]
        _lib.or_at_coeffs.argtypes = [C.c_int, C.c_int, d]
        _lib.or_rk_stages.argtypes = [C.c_int]
        _lib.or_lserk_coeffs.argtypes = [C.c_int, d, d, d]
        _lib.or_delay.argtypes = [C.POINTER(Cfg), C.c_int64, C.c_int]
        _lib.or_splitmix64.restype = C.c_uint64
        _lib.or_splitmix64.argtypes = [C.c_uint64]
        _lib.or_temperature.argtypes = [C.POINTER(Mech), d, C.c_double, C.c_double, d]
        _lib.or_state.argtypes = [C.POINTER(Mech), d, d, d, d, d, d]
        _lib.or_cons_from_prim.argtypes = [C.POINTER(Mech), C.c_double, C.c_double,
                                           C.c_double, d, d]
        _lib.or_rates.argtypes = [C.POINTER(Mech), C.c_double, C.c_int, d, d]
        _lib.or_wdot.argtypes = [C.POINTER(Mech), C.c_double, d, d]
        _lib.or_phys_flux.argtypes = [C.POINTER(Mech), d, d]
        _lib.or_num_flux.argtypes = [C.POINTER(Mech), C.c_int, d, d, d]
        _lib.or_eigen.argtypes = [C.POINTER(Mech), d, d, d, d]
        _lib.or_beta_matrix.argtypes = [C.c_int, d]
        _lib.or_shift_matrix.argtypes = [C.c_int, C.c_int, d]
        _lib.or_rhs_sync.argtypes = [C.POINTER(Cfg), C.POINTER(Mech), d, d]
        _lib.or_aux_sync.argtypes = [C.POINTER(Cfg), C.POINTER(Mech), d, d]
        _lib.or_limit_sync.argtypes = [C.POINTER(Cfg), C.POINTER(Mech), d, d,
                                       C.POINTER(C.c_uint8)]
        _lib.or_transport.argtypes = [C.POINTER(Mech), C.POINTER(Cfg), C.c_double, C.c_double,
                                      d, d, d, d]
        _lib.or_visc_flux.argtypes = [C.POINTER(Mech), C.POINTER(Cfg), d, d, d]
        _lib.or_reactor0d.argtypes = [C.POINTER(Mech), d, C.c_double, C.c_double, C.c_int]
    return _lib


def _dp(a: np.ndarray):
    return a.ctypes.data_as(C.POINTER(C.c_double))


class MechHandle:
    """Keeps the numpy arrays behind an ``or_mech`` alive."""

    def __init__(self, mech):
        self.arrays = [np.ascontiguousarray(x, dtype=np.float64) for x in
                       (mech.W, mech.cp, mech.h_f, mech.s0, mech.A, mech.b, mech.Ea)]
        self.nu_f = np.ascontiguousarray(mech.nu_f, dtype=np.int8)
        self.nu_r = np.ascontiguousarray(mech.nu_r, dtype=np.int8)
        W, cp, hf, s0, A, b, Ea = self.arrays
        self.ns, self.nr = int(W.shape[0]), int(A.shape[0])
        le = getattr(mech, "Le", None)
        self.Le = None if le is None else np.ascontiguousarray(le, dtype=np.float64)
        self.s = Mech(self.ns, self.nr, _dp(W), _dp(cp), _dp(hf), _dp(s0),
                      self.nu_f.ctypes.data_as(C.POINTER(C.c_byte)),
                      self.nu_r.ctypes.data_as(C.POINTER(C.c_byte)),
                      _dp(A), _dp(b), _dp(Ea),
                      _dp(self.Le) if self.Le is not None else C.POINTER(C.c_double)())

    @property
    def ref(self):
        return C.byref(self.s)


def make_cfg(wl, dt=None):
    probs = np.ascontiguousarray(np.array(wl.delay_probs if wl.delay_probs else [1.0],
                                          dtype=np.float64))
    cfg = Cfg(wl.n_elem, wl.p, wl.n_pe, wl.x0, wl.length, wl.dt if dt is None else dt,
              wl.bc_left, wl.bc_right, wl.flux, wl.limiter, wl.at_order, wl.delay_mode,
              wl.max_delay, _dp(probs), wl.seed & ((1 << 64) - 1), wl.tvb_M,
              getattr(wl, "integrator", 0), getattr(wl, "viscous", 0),
              getattr(wl, "mu_ref", 0.0), getattr(wl, "T_mu", 300.0),
              getattr(wl, "mu_exp", 0.7), getattr(wl, "prandtl", 0.7),
              int(getattr(wl, "face0", 0)), int(getattr(wl, "pe_begin", 0)),
              int(getattr(wl, "pe_end", 0)))
    return cfg, probs


def visc_flux(wl, mech, w, q):
    """f^d(w, q) at one point (w, q: [nv])."""
    cfg, probs = make_cfg(wl)
    mh = MechHandle(mech)
    w = np.ascontiguousarray(w, dtype=np.float64)
    q = np.ascontiguousarray(q, dtype=np.float64)
    fd = np.zeros_like(w)
    lib().or_visc_flux(mh.ref, C.byref(cfg), _dp(w), _dp(q), _dp(fd))
    return fd


def transport(wl, mech, rho, T, Y):
    """(mu, k, D[ns]) of the synthetic transport model."""
    cfg, probs = make_cfg(wl)
    mh = MechHandle(mech)
    Y = np.ascontiguousarray(Y, dtype=np.float64)
    mu, kc, D = np.zeros(1), np.zeros(1), np.zeros(mh.ns)
    lib().or_transport(mh.ref, C.byref(cfg), float(rho), float(T), _dp(Y), _dp(mu), _dp(kc),
                       _dp(D))
    return float(mu[0]), float(kc[0]), D


def aux_sync(wl, mech, w):
    """The LDG auxiliary variable q = dw/dx of a modal state (no delays)."""
    cfg, probs = make_cfg(wl)
    mh = MechHandle(mech)
    w = np.ascontiguousarray(w, dtype=np.float64)
    q = np.zeros_like(w)
    rc = lib().or_aux_sync(C.byref(cfg), mh.ref, _dp(w), _dp(q))
    if rc != 0:
        raise RuntimeError("or_aux_sync failed (%d)" % rc)
    return q


def limit_sync(wl, mech, w):
    """The troubled-cell indicator and WENO limiter applied once to a modal state
    (no delays): (flags [n_elem] uint8, limited state)."""
    cfg, probs = make_cfg(wl)
    mh = MechHandle(mech)
    w = np.ascontiguousarray(w, dtype=np.float64)
    out = np.zeros_like(w)
    flags = np.zeros(wl.n_elem, dtype=np.uint8)
    rc = lib().or_limit_sync(C.byref(cfg), mh.ref, _dp(w), _dp(out),
                             flags.ctypes.data_as(C.POINTER(C.c_uint8)))
    if rc != 0:
        raise RuntimeError("or_limit_sync failed (%d)" % rc)
    return flags, out


def rk_stages(integrator):
    return int(lib().or_rk_stages(int(integrator)))


def lserk_coeffs(integrator):
    """(A, B, C) of the 2N-storage LSERK scheme `integrator` (1 or 2)."""
    a, b, c = np.zeros(5), np.zeros(5), np.zeros(5)
    n = lib().or_lserk_coeffs(int(integrator), _dp(a), _dp(b), _dp(c))
    return a[:n], b[:n], c[:n]


class Oracle:
    """One instance of the scheme on the CPU."""

    def __init__(self, wl, mech=None):
        self.wl = wl
        self.mech = mech if mech is not None else wl.mechanism()
        self.mh = MechHandle(self.mech)
        self.cfg, self._probs = make_cfg(wl)
        self.nv = self.mh.ns + 2
        self.h = lib().or_create(C.byref(self.cfg), self.mh.ref)
        if not self.h:
            raise ValueError("oracle rejected the configuration")
        lay = [C.c_int(0) for _ in range(4)]
        lib().or_part_layout(self.h, *[C.byref(x) for x in lay])
        self.n_local, self.elem0 = lay[0].value, lay[1].value
        self.cut = (bool(lay[2].value), bool(lay[3].value))
        self.shape = (self.nv, self.n_local, wl.p + 1)

    def __del__(self):
        if getattr(self, "h", None):
            lib().or_destroy(self.h)
            self.h = None

    def set_primitive(self, prim):
        prim = np.ascontiguousarray(prim, dtype=np.float64)
        lib().or_set_primitive(self.h, _dp(prim))

    def set_state(self, w):
        w = np.ascontiguousarray(w, dtype=np.float64)
        lib().or_set_state(self.h, _dp(w))

    def state(self):
        w = np.zeros(self.shape)
        lib().or_get_state(self.h, _dp(w))
        return w

    def step(self, n=1):
        rc = lib().or_step(self.h, int(n))
        if rc != 0:
            raise RuntimeError("oracle step failed (%d) at step %d" % (rc, self.steps_done))

    def stage(self, s, half):
        """One half of RK stage s (or_stage): 0 the right-hand side and pre-limit
        output, 1 the limiter (and the end of the step after the last stage)."""
        rc = lib().or_stage(self.h, int(s), int(half))
        if rc != 0:
            raise RuntimeError("oracle stage failed (%d) at step %d" % (rc, self.steps_done))

    def export(self, what, side, s):
        """The owned boundary block [nv, p+1] at `side` (or_part_block)."""
        blk = np.zeros((self.nv, self.wl.p + 1))
        if lib().or_part_block(self.h, int(what), int(side), int(s), _dp(blk), 0) != 0:
            raise ValueError("no cut at side %d" % side)
        return blk

    def import_(self, what, side, s, blk):
        """Write a neighbour's block into the buffer element at `side`."""
        blk = np.ascontiguousarray(blk, dtype=np.float64)
        if lib().or_part_block(self.h, int(what), int(side), int(s), _dp(blk), 1) != 0:
            raise ValueError("no cut at side %d" % side)

    @property
    def steps_done(self):
        return int(lib().or_steps_done(self.h))

    def flags(self):
        last = np.zeros((rk_stages(self.cfg.integrator), self.n_local), dtype=np.uint8)
        cnt = np.zeros(self.n_local, dtype=np.int32)
        lib().or_get_flags(self.h, last.ctypes.data_as(C.POINTER(C.c_uint8)),
                           cnt.ctypes.data_as(C.POINTER(C.c_int32)))
        return last, cnt

    def temperature(self):
        T = np.zeros((self.n_local, self.wl.p + 1))
        lib().or_get_temperature(self.h, _dp(T))
        return T


# ---- thin wrappers of the single routines, for the pins ----

def legendre(n, x):
    P = np.zeros(n + 1)
    dP = np.zeros(n + 1)
    lib().or_legendre(n, float(x), _dp(P), _dp(dP))
    return P, dP


def gauss(q):
    x = np.zeros(q)
    w = np.zeros(q)
    assert lib().or_gauss(q, _dp(x), _dp(w)) == 0
    return x, w


def at_coeffs(order, k):
    c = np.zeros(order)
    lib().or_at_coeffs(order, k, _dp(c))
    return c


def splitmix64(x):
    return int(lib().or_splitmix64(C.c_uint64(x & ((1 << 64) - 1))))


def delay(wl, step, face):
    cfg, probs = make_cfg(wl)
    return int(lib().or_delay(C.byref(cfg), int(step), int(face)))


def temperature(mech, r, rhoe, guess=1000.0):
    mh = MechHandle(mech)
    r = np.ascontiguousarray(r, dtype=np.float64)
    T = np.zeros(1)
    it = lib().or_temperature(mh.ref, _dp(r), float(rhoe), float(guess), _dp(T))
    return float(T[0]), int(it)


def state(mech, w):
    mh = MechHandle(mech)
    w = np.ascontiguousarray(w, dtype=np.float64)
    out = [np.zeros(1) for _ in range(5)]
    lib().or_state(mh.ref, _dp(w), *[_dp(o) for o in out])
    return tuple(float(o[0]) for o in out)  # rho, u, T, P, a


def cons_from_prim(mech, T, P, u, Y):
    mh = MechHandle(mech)
    Y = np.ascontiguousarray(Y, dtype=np.float64)
    w = np.zeros(mh.ns + 2)
    lib().or_cons_from_prim(mh.ref, float(T), float(P), float(u), _dp(Y), _dp(w))
    return w


def rates(mech, T, j):
    mh = MechHandle(mech)
    kf = np.zeros(1)
    Kc = np.zeros(1)
    lib().or_rates(mh.ref, float(T), int(j), _dp(kf), _dp(Kc))
    return float(kf[0]), float(Kc[0])


def wdot(mech, T, conc):
    mh = MechHandle(mech)
    conc = np.ascontiguousarray(conc, dtype=np.float64)
    out = np.zeros(mh.ns)
    lib().or_wdot(mh.ref, float(T), _dp(conc), _dp(out))
    return out


def phys_flux(mech, w):
    mh = MechHandle(mech)
    w = np.ascontiguousarray(w, dtype=np.float64)
    f = np.zeros_like(w)
    lib().or_phys_flux(mh.ref, _dp(w), _dp(f))
    return f


def num_flux(mech, kind, wl, wr):
    mh = MechHandle(mech)
    wl = np.ascontiguousarray(wl, dtype=np.float64)
    wr = np.ascontiguousarray(wr, dtype=np.float64)
    f = np.zeros_like(wl)
    lib().or_num_flux(mh.ref, int(kind), _dp(wl), _dp(wr), _dp(f))
    return f


def eigen(mech, wbar):
    mh = MechHandle(mech)
    nv = mh.ns + 2
    wbar = np.ascontiguousarray(wbar, dtype=np.float64)
    R = np.zeros((nv, nv))
    L = np.zeros((nv, nv))
    lam = np.zeros(nv)
    lib().or_eigen(mh.ref, _dp(wbar), _dp(R), _dp(L), _dp(lam))
    return R, L, lam


def beta_matrix(p):
    B = np.zeros((p + 1, p + 1))
    lib().or_beta_matrix(p, _dp(B))
    return B


def shift_matrix(p, direction):
    S = np.zeros((p + 1, p + 1))
    lib().or_shift_matrix(p, int(direction), _dp(S))
    return S


def rhs_sync(wl, mech, w):
    mh = MechHandle(mech)
    cfg, probs = make_cfg(wl)
    w = np.ascontiguousarray(w, dtype=np.float64)
    out = np.zeros_like(w)
    rc = lib().or_rhs_sync(C.byref(cfg), mh.ref, _dp(w), _dp(out))
    if rc:
        raise RuntimeError("rhs failed %d" % rc)
    return out


def reactor0d(mech, r, rhoe, dt, n_steps):
    mh = MechHandle(mech)
    r = np.array(r, dtype=np.float64)
    rc = lib().or_reactor0d(mh.ref, _dp(r), float(rhoe), float(dt), int(n_steps))
    if rc:
        raise RuntimeError("reactor failed")
    return r
