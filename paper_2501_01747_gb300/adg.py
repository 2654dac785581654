"""Python binding of the CUDA library (include/adg.h): argument marshalling only.

Every step of the method runs in the CUDA kernels of ``csrc/``; this module builds
the shared library, converts numpy inputs to the C structs, hands PyTorch-owned
device memory and the current PyTorch stream to the library, and raises on error
codes. There is no CPU fallback: without the built library or a GPU every call
raises.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
from concurrent.futures import ThreadPoolExecutor

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
BUILD = os.path.join(HERE, "_build")
LIB = os.path.join(BUILD, "libadg.so")
SOURCES = ["adg_k64.cu", "adg_k32.cu", "adg_u64.cu", "adg_u32.cu", "adg_v64.cu",
           "adg_v32.cu", "adg_k32f.cu", "adg_kernels.cu", "adg_api.cu", "adg_static.cu"]
ARCH = "-gencode=arch=compute_103a,code=sm_103a"
NVCC_FLAGS = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", ARCH]

ADG_OK = 0
ERRORS = {-1: "ADG_ERR_ARG", -2: "ADG_ERR_CUDA", -3: "ADG_ERR_NOMEM",
          -4: "ADG_ERR_NONPHYSICAL", -5: "ADG_ERR_HISTORY", -6: "ADG_ERR_NOLIB",
          -7: "ADG_ERR_TIMEOUT"}
MAX_DELAY = 7  # ADG_MAX_DELAY
MAX_GROUPS = 24  # ADG_MAX_GROUPS
TUNING_FIELDS = 7  # ADG_TUNING_FIELDS


class AdgError(RuntimeError):
    def __init__(self, code, what=""):
        msg = "%s (%d)" % (ERRORS.get(code, "unknown"), code)
        try:
            msg += ": " + lib().adg_error_string(code).decode()
        except Exception:  # pragma: no cover
            pass
        super().__init__((what + ": " if what else "") + msg)
        self.code = code


def _nvcc():
    cand = [os.environ.get("NVCC", ""), "/usr/local/cuda/bin/nvcc", "nvcc"]
    for c in cand:
        if c and (os.path.isabs(c) and os.path.exists(c) or not os.path.isabs(c)):
            return c
    return "nvcc"


def build(force: bool = False, verbose: bool = False) -> str:
    """Compile csrc/*.cu for sm_103a into _build/libadg.so (objects in parallel)."""
    os.makedirs(BUILD, exist_ok=True)
    deps = [os.path.join(CSRC, f) for f in os.listdir(CSRC)]
    deps.append(os.path.join(os.path.dirname(HERE), "include", "adg.h"))
    newest = max(os.path.getmtime(d) for d in deps)
    if not force and os.path.exists(LIB) and os.path.getmtime(LIB) >= newest:
        return LIB
    nvcc = _nvcc()
    objs = []

    def compile_one(src):
        obj = os.path.join(BUILD, src.replace(".cu", ".o"))
        cmd = [nvcc, *NVCC_FLAGS, "-c", os.path.join(CSRC, src), "-o", obj]
        if verbose:
            print(" ".join(cmd))
        subprocess.check_call(cmd)
        return obj

    with ThreadPoolExecutor(len(SOURCES)) as ex:
        objs = list(ex.map(compile_one, SOURCES))
    tmp = LIB + ".tmp%d" % os.getpid()
    subprocess.check_call([nvcc, ARCH, "-shared", "-o", tmp, *objs, "-lcudart"])
    os.replace(tmp, LIB)
    return LIB


class Mechanism_(C.Structure):
    _fields_ = [("n_species", C.c_int), ("n_reactions", C.c_int),
                ("W", C.POINTER(C.c_double)), ("cp", C.POINTER(C.c_double)),
                ("h_f", C.POINTER(C.c_double)), ("s0", C.POINTER(C.c_double)),
                ("nu_f", C.POINTER(C.c_byte)), ("nu_r", C.POINTER(C.c_byte)),
                ("A", C.POINTER(C.c_double)), ("b", C.POINTER(C.c_double)),
                ("Ea", C.POINTER(C.c_double)), ("Le", C.POINTER(C.c_double))]


class Config_(C.Structure):
    _fields_ = [("n_elem", C.c_int), ("p", C.c_int), ("n_pe", C.c_int),
                ("x0", C.c_double), ("length", C.c_double), ("dt", C.c_double),
                ("bc_left", C.c_int), ("bc_right", C.c_int), ("flux", C.c_int),
                ("limiter", C.c_int), ("at_order", C.c_int), ("delay_mode", C.c_int),
                ("max_delay", C.c_int), ("delay_probs", C.POINTER(C.c_double)),
                ("seed", C.c_uint64), ("tvb_M", C.c_double), ("precision", C.c_int),
                ("integrator", C.c_int), ("viscous", C.c_int), ("mu_ref", C.c_double),
                ("T_mu", C.c_double), ("mu_exp", C.c_double), ("prandtl", C.c_double),
                ("pe_begin", C.c_int), ("pe_end", C.c_int)]


_lib = None
EXPORTS = ["adg_workspace_bytes", "adg_create", "adg_destroy", "adg_set_primitive",
           "adg_set_state", "adg_set_state_device", "adg_get_state", "adg_get_state_device",
           "adg_step", "adg_status", "adg_get_flags", "adg_get_temperature", "adg_steps_done",
           "adg_delay_table", "adg_launches_per_step", "adg_error_string",
           "adg_write_state", "adg_read_state", "adg_enable_kernel_timing",
           "adg_kernel_times", "adg_step_noalloc", "adg_autotune", "adg_get_tuning",
           "adg_set_tuning", "adg_step_unsync", "adg_unsync_delays",
           "adg_set_unsync_wait", "adg_set_unsync_imbalance", "adg_get_aux",
           "adg_part_layout", "adg_step_stage", "adg_part_block", "adg_set_limiter_tuning",
           "adg_write_states", "adg_read_states", "adg_states_doubles", "adg_step_io"]


def lib(path: str | None = None):
    """Load the library (building it first if needed)."""
    global _lib
    if _lib is not None:
        return _lib
    path = path or build()
    L = C.CDLL(path)
    vp, d = C.c_void_p, C.POINTER(C.c_double)
    L.adg_workspace_bytes.argtypes = [C.POINTER(Mechanism_), C.POINTER(Config_), C.c_int,
                                      C.POINTER(C.c_size_t)]
    L.adg_create.argtypes = [C.POINTER(Mechanism_), C.POINTER(Config_), C.c_int, vp,
                             C.c_size_t, C.POINTER(vp)]
    L.adg_destroy.argtypes = [vp]
    L.adg_destroy.restype = None
    L.adg_set_primitive.argtypes = [vp, C.c_int, d]
    L.adg_set_state.argtypes = [vp, C.c_int, d]
    L.adg_set_state_device.argtypes = [vp, C.c_int, vp, vp]
    L.adg_get_state.argtypes = [vp, C.c_int, d]
    L.adg_get_state_device.argtypes = [vp, C.c_int, vp, vp]
    L.adg_step.argtypes = [vp, C.c_int, vp]
    L.adg_status.argtypes = [vp, C.POINTER(C.c_int), C.POINTER(C.c_int),
                             C.POINTER(C.c_int64), C.POINTER(C.c_int)]
    L.adg_get_flags.argtypes = [vp, C.c_int, C.POINTER(C.c_uint8), C.POINTER(C.c_int32)]
    L.adg_get_temperature.argtypes = [vp, C.c_int, d]
    L.adg_get_aux.argtypes = [vp, C.c_int, C.c_int, vp]
    L.adg_steps_done.argtypes = [vp, C.c_int]
    L.adg_steps_done.restype = C.c_int64
    L.adg_delay_table.argtypes = [C.POINTER(Config_), C.c_int64, C.c_int, C.POINTER(C.c_uint8)]
    L.adg_launches_per_step.argtypes = [vp]
    L.adg_write_state.argtypes = [vp, C.c_int, d, vp]
    L.adg_read_state.argtypes = [vp, C.c_int, d, vp]
    L.adg_write_states.argtypes = [vp, d, vp]
    L.adg_read_states.argtypes = [vp, d, vp]
    L.adg_states_doubles.argtypes = [vp]
    L.adg_step_io.argtypes = [vp, d, d, vp]
    L.adg_states_doubles.restype = C.c_int64
    L.adg_enable_kernel_timing.argtypes = [vp, C.c_int]
    L.adg_kernel_times.argtypes = [vp, d, C.POINTER(C.c_int64)]
    L.adg_step_noalloc.argtypes = [C.POINTER(Mechanism_), C.POINTER(Config_), vp, vp, C.c_int,
                                   vp]
    L.adg_autotune.argtypes = [vp, vp]
    L.adg_get_tuning.argtypes = [vp, C.POINTER(C.c_int), C.POINTER(C.c_int)]
    L.adg_set_tuning.argtypes = [vp, C.c_int, C.c_int, C.c_int]
    L.adg_set_limiter_tuning.argtypes = [vp, C.c_int, C.c_int]
    L.adg_step_unsync.argtypes = [vp, C.c_int, C.c_int, vp]
    L.adg_unsync_delays.argtypes = [vp, C.POINTER(C.c_uint64)]
    L.adg_set_unsync_wait.argtypes = [vp, C.c_longlong, C.c_int]
    L.adg_set_unsync_imbalance.argtypes = [vp, C.c_int, C.c_int]
    ip = C.POINTER(C.c_int)
    L.adg_part_layout.argtypes = [C.POINTER(Config_), ip, ip, ip, ip]
    L.adg_step_stage.argtypes = [vp, C.c_int, C.c_int, vp]
    L.adg_part_block.argtypes = [vp, C.c_int, C.c_int, C.c_int, C.c_int, vp, C.c_int, vp]
    L.adg_error_string.restype = C.c_char_p
    L.adg_error_string.argtypes = [C.c_int]
    _lib = L
    return L


def _dp(a):
    return a.ctypes.data_as(C.POINTER(C.c_double))


def _check(rc, what=""):
    if rc != ADG_OK:
        raise AdgError(rc, what)


class _MechArgs:
    def __init__(self, mech):
        self.keep = [np.ascontiguousarray(x, dtype=np.float64) for x in
                     (mech.W, mech.cp, mech.h_f, mech.s0, mech.A, mech.b, mech.Ea)]
        self.nu_f = np.ascontiguousarray(mech.nu_f, dtype=np.int8)
        self.nu_r = np.ascontiguousarray(mech.nu_r, dtype=np.int8)
        W, cp, hf, s0, A, b, Ea = self.keep
        le = getattr(mech, "Le", None)
        self.Le = None if le is None else np.ascontiguousarray(le, dtype=np.float64)
        self.s = Mechanism_(W.shape[0], A.shape[0], _dp(W), _dp(cp), _dp(hf), _dp(s0),
                            self.nu_f.ctypes.data_as(C.POINTER(C.c_byte)),
                            self.nu_r.ctypes.data_as(C.POINTER(C.c_byte)),
                            _dp(A), _dp(b), _dp(Ea),
                            _dp(self.Le) if self.Le is not None else C.POINTER(C.c_double)())


FP64, MIXED, MIXED_F32CHEM = 0, 1, 2
PRECISIONS = {"fp64": FP64, "mixed": MIXED, "mixed_f32chem": MIXED_F32CHEM}
PRECISION_NAMES = {v: k for k, v in PRECISIONS.items()}


def _precision(x):
    if isinstance(x, str):
        if x not in PRECISIONS:
            raise AdgError(-1, "precision must be one of %s" % sorted(PRECISIONS))
        return PRECISIONS[x]
    if int(x) not in PRECISION_NAMES:
        raise AdgError(-1, "precision must be ADG_FP64, ADG_MIXED or ADG_MIXED_F32CHEM")
    return int(x)


def config_struct(wl, precision=FP64):
    probs = np.ascontiguousarray(np.array(wl.delay_probs or [1.0], dtype=np.float64))
    c = Config_(wl.n_elem, wl.p, wl.n_pe, wl.x0, wl.length, wl.dt, wl.bc_left, wl.bc_right,
                wl.flux, wl.limiter, wl.at_order, wl.delay_mode, wl.max_delay, _dp(probs),
                wl.seed & ((1 << 64) - 1), wl.tvb_M, _precision(precision),
                int(getattr(wl, "integrator", 0)), int(getattr(wl, "viscous", 0)),
                float(getattr(wl, "mu_ref", 0.0)), float(getattr(wl, "T_mu", 300.0)),
                float(getattr(wl, "mu_exp", 0.7)), float(getattr(wl, "prandtl", 0.7)),
                int(getattr(wl, "pe_begin", 0)), int(getattr(wl, "pe_end", 0)))
    return c, probs


PART_INPUT, PART_PRELIMIT = 0, 1


def part_layout(wl):
    """adg_part_layout: (n_local, elem0, cut_left, cut_right) of a (sub)domain."""
    cfg, probs = config_struct(wl)
    out = [C.c_int(0) for _ in range(4)]
    _check(lib().adg_part_layout(C.byref(cfg), *[C.byref(o) for o in out]), "adg_part_layout")
    return tuple(int(o.value) for o in out)


def rk_stages(wl):
    """RK stages per step of a workload's integrator (5 for LSERK4, else 3)."""
    return 5 if int(getattr(wl, "integrator", 0)) == 2 else 3


def delay_table(wl, step0, n_steps):
    """Delays [n_steps][n_pe_faces] as the library draws them."""
    cfg, probs = config_struct(wl)
    npf = 0 if wl.n_pe <= 1 else (wl.n_pe if wl.bc_left == 0 else wl.n_pe - 1)
    pb, pe = int(getattr(wl, "pe_begin", 0)), int(getattr(wl, "pe_end", 0))
    if pe > 0 and not (pb == 0 and pe == wl.n_pe):
        _, _, cut_l, cut_r = part_layout(wl)
        npf = cut_l + (pe - pb - 1) + cut_r
    out = np.zeros((n_steps, max(npf, 0)), dtype=np.uint8)
    _check(lib().adg_delay_table(C.byref(cfg), int(step0), int(n_steps),
                                 out.ctypes.data_as(C.POINTER(C.c_uint8))), "adg_delay_table")
    return out


def step_noalloc(mech, wl, w_in_dev, w_out_dev, n_steps, stream=None, precision="fp64"):
    """adg_step_noalloc: advance one instance from the device tensor w_in_dev to
    w_out_dev without any allocation (scratch in the library's static array)."""
    m = _MechArgs(mech)
    cfg, probs = config_struct(wl, precision)
    if stream is None:
        import torch
        stream = torch.cuda.current_stream(w_out_dev.device)
    st = C.c_void_p(stream.cuda_stream if hasattr(stream, "cuda_stream") else int(stream))
    _check(lib().adg_step_noalloc(C.byref(m.s), C.byref(cfg), C.c_void_p(w_in_dev.data_ptr()),
                                  C.c_void_p(w_out_dev.data_ptr()), int(n_steps), st),
           "adg_step_noalloc")


def _torch():
    import torch
    return torch


class ADG:
    """A context of one or more instances sharing one mechanism.

    Device memory is one PyTorch uint8 tensor handed to ``adg_create`` (the
    library carves its buffers out of it); kernels run on PyTorch's current CUDA
    stream unless a stream is given. ``precision`` is "fp64", "mixed" (FP32 flux,
    DG operator and limiter, FP64 chemistry) or "mixed_f32chem" (the chemistry in
    float too) for all instances, or a list with one entry per instance."""

    def __init__(self, mech, workloads, device=None, precision="fp64"):
        torch = _torch()
        if not torch.cuda.is_available():
            raise AdgError(-6, "ADG needs a CUDA device")
        self.L = lib()
        self.workloads = list(workloads)
        self._m = _MechArgs(mech)
        self.ns = int(self._m.keep[0].shape[0])
        self.nv = self.ns + 2
        prec = precision if isinstance(precision, (list, tuple)) else \
            [precision] * len(self.workloads)
        if len(prec) != len(self.workloads):
            raise AdgError(-1, "one precision per instance")
        self.precision = [_precision(x) for x in prec]
        cfgs = [config_struct(w, x) for w, x in zip(self.workloads, self.precision)]
        self._probs = [c[1] for c in cfgs]
        arr = (Config_ * len(cfgs))(*[c[0] for c in cfgs])
        self._cfgs = arr
        nbytes = C.c_size_t(0)
        _check(self.L.adg_workspace_bytes(C.byref(self._m.s), arr, len(cfgs), C.byref(nbytes)),
               "adg_workspace_bytes")
        self.device = torch.device(device or "cuda")
        self.workspace = torch.empty(int(nbytes.value) + 256, dtype=torch.uint8,
                                     device=self.device)
        base = self.workspace.data_ptr()
        aligned = (base + 255) & ~255
        h = C.c_void_p(0)
        _check(self.L.adg_create(C.byref(self._m.s), arr, len(cfgs), C.c_void_p(aligned),
                                 C.c_size_t(int(nbytes.value)), C.byref(h)), "adg_create")
        self.h = h
        # elements of each instance's arrays (a subdomain's include its buffers)
        self.n_local = [part_layout(w)[0] for w in self.workloads]

    def close(self):
        if getattr(self, "h", None) and self.h.value:
            self.L.adg_destroy(self.h)
            self.h = C.c_void_p(0)

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _k(self, k):
        if not (0 <= int(k) < len(self.workloads)):
            raise AdgError(-1, "instance %r out of range" % (k,))
        return int(k)

    def shape(self, k=0):
        wl = self.workloads[self._k(k)]
        return (self.nv, self.n_local[self._k(k)], wl.p + 1)

    def _stream(self, stream):
        if stream is None:
            return C.c_void_p(_torch().cuda.current_stream(self.device).cuda_stream)
        if hasattr(stream, "cuda_stream"):
            return C.c_void_p(stream.cuda_stream)
        return C.c_void_p(int(stream))

    def set_primitive(self, prim, k=0):
        prim = np.ascontiguousarray(prim, dtype=np.float64)
        _check(self.L.adg_set_primitive(self.h, k, _dp(prim)), "adg_set_primitive")

    def set_state(self, w, k=0):
        w = np.ascontiguousarray(w, dtype=np.float64)
        _check(self.L.adg_set_state(self.h, k, _dp(w)), "adg_set_state")

    def set_state_device(self, w_dev, k=0, stream=None):
        _check(self.L.adg_set_state_device(self.h, k, C.c_void_p(w_dev.data_ptr()),
                                           self._stream(stream)), "adg_set_state_device")

    def get_state(self, k=0, out=None):
        w = out if out is not None else np.zeros(self.shape(k))
        _check(self.L.adg_get_state(self.h, k, _dp(w)), "adg_get_state")
        return w

    def get_state_device(self, w_dev, k=0, stream=None):
        _check(self.L.adg_get_state_device(self.h, k, C.c_void_p(w_dev.data_ptr()),
                                           self._stream(stream)), "adg_get_state_device")

    def step(self, n=1, stream=None):
        _check(self.L.adg_step(self.h, int(n), self._stream(stream)), "adg_step")


    def step_stage(self, stage, half, stream=None):
        """adg_step_stage: half 0 (stage kernels) or 1 (limiters, and after the
        last stage the step counters) of RK stage `stage` of every instance."""
        _check(self.L.adg_step_stage(self.h, int(stage), int(half), self._stream(stream)),
               "adg_step_stage")

    def part_block(self, k, what, side, stage, blk_dev, import_, stream=None):
        """adg_part_block: export (import_ False) the owned boundary block of
        instance k at `side` into the device tensor blk_dev [nv, p+1], or import
        blk_dev into that side's buffer element."""
        _check(self.L.adg_part_block(self.h, self._k(k), int(what), int(side), int(stage),
                                     C.c_void_p(blk_dev.data_ptr()), 1 if import_ else 0,
                                     self._stream(stream)), "adg_part_block")
    def status(self):
        inst, el, st, sg = C.c_int(-1), C.c_int(-1), C.c_int64(-1), C.c_int(-1)
        rc = self.L.adg_status(self.h, C.byref(inst), C.byref(el), C.byref(st), C.byref(sg))
        return rc, (inst.value, el.value, st.value, sg.value)

    def check(self):
        rc, where = self.status()
        if rc != ADG_OK:
            raise AdgError(rc, "device error at instance/element/step/stage %s" % (where,))

    def flags(self, k=0):
        wl = self.workloads[self._k(k)]
        n = self.n_local[k]
        last = np.zeros((rk_stages(wl), n), dtype=np.uint8)
        cnt = np.zeros(n, dtype=np.int32)
        _check(self.L.adg_get_flags(self.h, k, last.ctypes.data_as(C.POINTER(C.c_uint8)),
                                    cnt.ctypes.data_as(C.POINTER(C.c_int32))), "adg_get_flags")
        return last, cnt

    def temperature(self, k=0):
        wl = self.workloads[self._k(k)]
        T = np.zeros((self.n_local[k], wl.p + 1))
        _check(self.L.adg_get_temperature(self.h, k, _dp(T)), "adg_get_temperature")
        return T

    def steps_done(self, k=0):
        return int(self.L.adg_steps_done(self.h, k))

    def write_state(self, w_host, k=0, stream=None):
        """Async H2D overwrite of the running state (history kept)."""
        _check(self.L.adg_write_state(self.h, k, _dp(w_host), self._stream(stream)),
               "adg_write_state")

    def read_state(self, w_host, k=0, stream=None):
        """Async D2H read of the state (valid after the stream passes it)."""
        _check(self.L.adg_read_state(self.h, k, _dp(w_host), self._stream(stream)),
               "adg_read_state")

    def states_doubles(self):
        """Length of the buffer that write_states / read_states use."""
        return int(self.L.adg_states_doubles(self.h))

    def write_states(self, w_host, stream=None):
        """adg_write_states: every instance's state from one host buffer (the
        states in instance order), asynchronously on the stream."""
        _check(self.L.adg_write_states(self.h, _dp(w_host), self._stream(stream)),
               "adg_write_states")

    def read_states(self, w_host, stream=None):
        """adg_read_states: every instance's state into one host buffer."""
        _check(self.L.adg_read_states(self.h, _dp(w_host), self._stream(stream)),
               "adg_read_states")

    def step_io(self, w_in_host, w_out_host, stream=None):
        """adg_step_io: every instance's state from w_in_host, one step, the
        results into w_out_host (both in write_states' layout), with each
        group's copies overlapped with the other groups' stages when the
        buffers are mapped pinned memory."""
        _check(self.L.adg_step_io(self.h, _dp(w_in_host), _dp(w_out_host), self._stream(stream)),
               "adg_step_io")

    def enable_kernel_timing(self, on=True):
        _check(self.L.adg_enable_kernel_timing(self.h, 1 if on else 0), "timing")

    def kernel_times(self):
        """(ms, counts) per kind: stage kernel, limiter kernel, whole step."""
        ms = np.zeros(3)
        n = np.zeros(3, dtype=np.int64)
        _check(self.L.adg_kernel_times(self.h, _dp(ms), n.ctypes.data_as(C.POINTER(C.c_int64))),
               "adg_kernel_times")
        return ms, n

    def autotune(self, stream=None):
        """Pick elements per tile and threads per CTA by timing the stage kernel."""
        _check(self.L.adg_autotune(self.h, self._stream(stream)), "adg_autotune")
        return self.tuning()

    def tuning(self):
        n = C.c_int(0)
        F = TUNING_FIELDS
        t = (C.c_int * (F * MAX_GROUPS))()
        _check(self.L.adg_get_tuning(self.h, C.byref(n), t), "adg_get_tuning")
        return [{"p": t[F * g], "precision": PRECISION_NAMES[t[F * g + 1]],
                 "elements_per_tile": t[F * g + 2], "threads_per_cta": t[F * g + 3],
                 "tiles": t[F * g + 4], "stages": t[F * g + 5],
                 "limiter_elements_per_cta": t[F * g + 6]} for g in range(n.value)]

    def set_tuning(self, group, elements_per_tile, threads_per_cta):
        """Set the stage launch configuration of a group (e.g. a stored autotune result)."""
        _check(self.L.adg_set_tuning(self.h, int(group), int(elements_per_tile),
                                     int(threads_per_cta)), "adg_set_tuning")
        return self.tuning()


    def set_limiter_tuning(self, group, elements_per_cta):
        """Set a group's limiter elements per CTA (adg_set_limiter_tuning)."""
        _check(self.L.adg_set_limiter_tuning(self.h, int(group), int(elements_per_cta)),
               "adg_set_limiter_tuning")
        return self.tuning()
    def step_unsync(self, n=1, k=0, stream=None):
        """n steps of instance k in the truly unsynchronised mode (one CTA per PE,
        each PE using the newest level its neighbours have published)."""
        _check(self.L.adg_step_unsync(self.h, self._k(k), int(n), self._stream(stream)),
               "adg_step_unsync")

    def set_unsync_wait(self, max_polls=1 << 22, withheld_pe=-1):
        """Bound of the unsynchronised mode's waits (polls of a counter), and a PE
        that never publishes (to exercise the timeout), -1 for none."""
        _check(self.L.adg_set_unsync_wait(self.h, int(max_polls), int(withheld_pe)),
               "adg_set_unsync_wait")

    def set_unsync_imbalance(self, slow_pe=-1, slow_us=0):
        """PE slow_pe idles about slow_us microseconds per stage in the
        unsynchronised mode (emulated load imbalance); -1 for none."""
        _check(self.L.adg_set_unsync_imbalance(self.h, int(slow_pe), int(slow_us)),
               "adg_set_unsync_imbalance")

    def unsync_delays(self):
        """Delays used by the unsynchronised mode since the last call: array
        [2][MAX_DELAY + 1] (row 0: flux, row 1: limiter)."""
        h = np.zeros(2 * (MAX_DELAY + 1), dtype=np.uint64)
        _check(self.L.adg_unsync_delays(self.h, h.ctypes.data_as(C.POINTER(C.c_uint64))),
               "adg_unsync_delays")
        return h.reshape(2, MAX_DELAY + 1)

    def pressure(self, k=0):
        """Pressure at every Gauss point of instance k, [n_elem, p+1]."""
        wl = self.workloads[self._k(k)]
        P = np.zeros((self.n_local[k], wl.p + 1))
        _check(self.L.adg_get_aux(self.h, k, 1, P.ctypes.data_as(C.c_void_p)), "adg_get_aux")
        return P

    def launches_per_step(self):
        return int(self.L.adg_launches_per_step(self.h))
