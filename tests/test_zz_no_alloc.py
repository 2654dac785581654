"""adg_step_noalloc, the time step for callers that cannot allocate device memory
(it keeps all scratch in a static device array), against the regular context
path: the same state after the same steps, on calls in a row. The cases cover
every precision variant, an output buffer that is the input itself, and a
9-species problem right after 5-species ones (the scratch and the per-device
set-up are reused with another mechanism size). This file is collected last so
that a stop at the first failure has run every other test."""
import numpy as np
import pytest

from paper_2501_01747_gb300 import adg
from paper_2501_01747_gb300 import inputs as I
from tests import helpers as H

pytestmark = pytest.mark.gpu

TOL = 1e-10


def _context_result(wl, mech, n, prec):
    g = adg.ADG(mech, [wl], precision=prec)
    g.set_primitive(wl.primitive(mech))
    w0 = g.get_state()
    g.set_state(w0)
    g.step(n)
    g.check()
    ref = g.get_state()
    g.close()
    return w0, ref


def _noalloc(mech, wl, w0, n, prec, in_place):
    import torch
    w_in = torch.from_numpy(w0).cuda()
    w_out = w_in if in_place else torch.full_like(w_in, float("nan"))
    adg.step_noalloc(mech, wl, w_in, w_out, n, precision=prec)
    torch.cuda.synchronize()
    return w_out.cpu().numpy()


@pytest.mark.parametrize("prec", ["fp64", "mixed", "mixed_f32chem"])
@pytest.mark.parametrize("in_place", [False, True])
def test_noalloc_step_matches_context_path_twice(prec, in_place):
    wl = I.load_workloads()["ignition-5sp-200x3"]
    mech = wl.mechanism()
    w0, ref = _context_result(wl, mech, 25, prec)
    for call in range(2):
        got = _noalloc(mech, wl, w0, 25, prec, in_place)
        assert np.all(np.isfinite(got))
        err = H.parity_error(got, ref, mech)
        assert err.max() <= TOL, (call, err)


def test_noalloc_larger_mechanism_after_a_smaller_one():
    """A 9-species, 21-reaction problem (97 x p3, 7 PEs with SAA delays) right
    after two 5-species calls, then the 5-species problem again."""
    small = I.load_workloads()["ignition-5sp-200x3"]
    sm = small.mechanism()
    base = I.load_workloads()["ignition-9sp-4096x4"]
    big = I.scaled(base, 97, 7)
    big.p, big.at_order = 3, 4
    bm = big.mechanism()
    w0s, refs = _context_result(small, sm, 10, "fp64")
    w0b, refb = _context_result(big, bm, 12, "fp64")
    for _ in range(2):
        assert H.parity_error(_noalloc(sm, small, w0s, 10, "fp64", False), refs, sm).max() <= TOL
    got = _noalloc(bm, big, w0b, 12, "fp64", False)
    assert H.parity_error(got, refb, bm).max() <= TOL
    assert H.parity_error(_noalloc(sm, small, w0s, 10, "fp64", True), refs, sm).max() <= TOL


def test_noalloc_rejects_problems_beyond_the_static_scratch():
    import torch
    wl = I.load_workloads()["ignition-9sp-4096x4"]
    big = I.scaled(wl, 65536, 64)
    mech = wl.mechanism()
    w = torch.zeros(8, dtype=torch.float64, device="cuda")
    with pytest.raises(adg.AdgError) as ei:
        adg.step_noalloc(mech, big, w, w, 1)
    assert ei.value.code == -3
