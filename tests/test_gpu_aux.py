"""The auxiliary-field getter of the C ABI (adg_get_aux): temperature, pressure
and troubled-cell flags of the current state. The pressure is checked against
the ideal-gas definition P = rho R_u T sum_i Y_i / W_i (Sec. 2) evaluated from the
oracle's state and temperature at the Gauss points."""
import ctypes as C

import numpy as np
import pytest

import oracle as O
from paper_2501_01747_gb300 import adg
from paper_2501_01747_gb300 import inputs as I
from tests import helpers as H

pytestmark = pytest.mark.gpu

RU = 8.314462618


def test_aux_fields_match_the_oracle():
    wl = I.load_workloads()["ignition-5sp-200x3"]
    mech = wl.mechanism()
    prim = wl.primitive(mech)
    g = adg.ADG(mech, [wl])
    g.set_primitive(prim)
    o = O.Oracle(wl, mech)
    o.set_primitive(prim)
    g.step(20)
    o.step(20)
    g.check()
    To = o.temperature()
    r = H.modal_to_nodal(o.state()[2:], wl.p)  # [ns][N][Q] partial densities
    Po = RU * To * np.einsum("i,ieq->eq", 1.0 / mech.W, r)
    P = g.pressure()
    assert np.abs(P - Po).max() <= 1e-10 * Po.max()
    T = np.zeros_like(To)
    rc = g.L.adg_get_aux(g.h, 0, 0, T.ctypes.data_as(C.c_void_p))
    assert rc == 0 and np.abs(T - To).max() <= 1e-9 * To.max()
    flags = np.zeros((3, wl.n_elem), dtype=np.uint8)
    assert g.L.adg_get_aux(g.h, 0, 2, flags.ctypes.data_as(C.c_void_p)) == 0
    assert np.array_equal(flags, g.flags()[0])
    assert g.L.adg_get_aux(g.h, 0, 7, T.ctypes.data_as(C.c_void_p)) == -1
