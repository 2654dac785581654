"""The C ABI without a GPU: the library builds, loads and exports every function
include/adg.h declares; host-side logic (delay tables, validation, workspace
sizing) agrees with the oracle's definitions."""
import ctypes as C
import os
import re

import numpy as np
import pytest

import oracle as O
from paper_2501_01747_gb300 import adg
from paper_2501_01747_gb300 import inputs as I
from tests import helpers as H

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    src = open(os.path.join(ROOT, "include", "adg.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(adg_[a-z_]+)\s*\(", src)))


def test_library_exports_every_declared_function():
    path = adg.build()
    L = C.CDLL(path)
    names = declared_functions()
    assert len(names) >= 15
    for n in names:
        assert hasattr(L, n), n
    assert set(names) == set(adg.EXPORTS)


def test_error_strings():
    L = adg.lib()
    for code in (0, -1, -2, -3, -4, -5, -6, -99):
        assert isinstance(L.adg_error_string(code), bytes)


@pytest.mark.parametrize("mode", [I.DELAY_SYNC, I.DELAY_CAA, I.DELAY_SAA])
@pytest.mark.parametrize("bc", [I.BC_PERIODIC, I.BC_OUTFLOW])
def test_delay_table_matches_oracle(mode, bc):
    wl = H.workload(64, 2, n_pe=8, delay_mode=mode, max_delay=3, bc=(bc, bc),
                    probs=(0.4, 0.3, 0.2, 0.1), seed=987654321987)
    tab = adg.delay_table(wl, 5, 40)
    npf = 8 if bc == I.BC_PERIODIC else 7
    assert tab.shape == (40, npf)
    ref = np.array([[O.delay(wl, 5 + s, f) for f in range(npf)] for s in range(40)])
    assert np.array_equal(tab, ref)


def test_delay_table_single_pe_is_empty():
    wl = H.workload(16, 2, n_pe=1, delay_mode=I.DELAY_SAA, max_delay=2)
    assert adg.delay_table(wl, 0, 10).shape == (10, 0)


def _ws(mech, wls):
    m = adg._MechArgs(mech)
    cfgs = [adg.config_struct(w) for w in wls]
    arr = (adg.Config_ * len(cfgs))(*[c[0] for c in cfgs])
    n = C.c_size_t(0)
    rc = adg.lib().adg_workspace_bytes(C.byref(m.s), arr, len(cfgs), C.byref(n))
    return rc, n.value


def test_workspace_grows_with_mesh_and_history():
    mech = I.make_mechanism(9, 21, 1)
    small = H.workload(64, 2, n_pe=4, ns=9, nr=21, delay_mode=I.DELAY_SAA, max_delay=2)
    big = H.workload(128, 2, n_pe=4, ns=9, nr=21, delay_mode=I.DELAY_SAA, max_delay=2)
    rc1, b1 = _ws(mech, [small])
    rc2, b2 = _ws(mech, [big])
    rc3, b3 = _ws(mech, [small, big])
    assert rc1 == rc2 == rc3 == 0
    nv = 11
    assert b2 - b1 >= 3 * 8 * nv * 64 * 3  # three state buffers of the extra elements
    assert b3 > b2


@pytest.mark.parametrize("field,value", [("p", 0), ("p", 5), ("n_pe", 0), ("at_order", 0),
                                         ("at_order", 7), ("max_delay", 8), ("dt", 0.0),
                                         ("flux", 3), ("limiter", 2), ("delay_mode", 5)])
def test_invalid_configurations_are_rejected(field, value):
    mech = I.make_mechanism(5, 4, 1)
    wl = H.workload(32, 2, n_pe=2, ns=5, nr=4)
    setattr(wl, field, value)
    rc, _ = _ws(mech, [wl])
    assert rc == -1


def test_mixed_periodic_boundaries_rejected():
    mech = I.make_mechanism(5, 4, 1)
    wl = H.workload(32, 2, n_pe=2, ns=5, nr=4, bc=(I.BC_PERIODIC, I.BC_OUTFLOW))
    assert _ws(mech, [wl])[0] == -1


def test_create_without_gpu_fails_cleanly():
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    mech = I.make_mechanism(5, 4, 1)
    wl = H.workload(32, 2, n_pe=2, ns=5, nr=4)
    m = adg._MechArgs(mech)
    cfg, probs = adg.config_struct(wl)
    h = C.c_void_p(0)
    rc = adg.lib().adg_create(C.byref(m.s), C.byref(cfg), 1, None, 0, C.byref(h))
    assert rc == -6 and not h.value
    with pytest.raises(adg.AdgError):
        adg.ADG(mech, [wl])
