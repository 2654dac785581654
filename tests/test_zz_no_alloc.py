"""adg_step_noalloc, the time step for callers that cannot allocate device memory
(it keeps all scratch in a static device array), against the regular context
path: the same state after the same steps, on two calls in a row. This file is
collected last so that a stop at the first failure has run every other test."""
import numpy as np
import pytest

from paper_2501_01747_gb300 import adg
from paper_2501_01747_gb300 import inputs as I
from tests import helpers as H

pytestmark = pytest.mark.gpu

TOL = 1e-10


def test_noalloc_step_matches_context_path_twice():
    import torch
    wl = I.load_workloads()["ignition-5sp-200x3"]
    mech = wl.mechanism()
    g = adg.ADG(mech, [wl])
    g.set_primitive(wl.primitive(mech))
    w0 = g.get_state()
    g.set_state(w0)
    g.step(25)
    g.check()
    ref = g.get_state()
    w_in = torch.from_numpy(w0).cuda()
    for call in range(2):
        w_out = torch.full_like(w_in, float("nan"))
        adg.step_noalloc(mech, wl, w_in, w_out, 25)
        torch.cuda.synchronize()
        got = w_out.cpu().numpy()
        assert np.all(np.isfinite(got))
        err = H.parity_error(got, ref, mech)
        assert err.max() <= TOL, (call, err)


def test_noalloc_rejects_problems_beyond_the_static_scratch():
    import torch
    wl = I.load_workloads()["ignition-9sp-4096x4"]
    big = I.scaled(wl, 65536, 64)
    mech = wl.mechanism()
    w = torch.zeros(8, dtype=torch.float64, device="cuda")
    with pytest.raises(adg.AdgError) as ei:
        adg.step_noalloc(mech, big, w, w, 1)
    assert ei.value.code == -3
