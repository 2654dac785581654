"""The truly unsynchronised mode (one cooperative launch, one CTA per PE, each PE
using the newest level its neighbours have published; Sec. 3.2).

Its result depends on timing, so it is pinned by what does not:
* with maximum delay 0 every PE waits for the current level, and the result is
  bit for bit the synchronous adg_step's (FP64 and mixed, with the troubled-cell
  flags), which the FP64 parity tests tie to the oracle;
* with delays (one PE made slower so that its neighbours run ahead), every
  delay used lies in [0, d], some are positive, the scheme stays conservative to
  round-off (both sides of a PE face use the common level of Sec. 3.2), and the
  error against the synchronous oracle is of the size the seeded-delay oracle
  run shows for the same maximum delay;
* a wait that cannot end reports ADG_ERR_TIMEOUT and leaves the CUDA context
  usable; more PEs than fit on the GPU at once are rejected on the host."""
import dataclasses

import numpy as np
import pytest

import oracle as O
from paper_2501_01747_gb300 import adg
from paper_2501_01747_gb300 import inputs as I
from tests import helpers as H

pytestmark = pytest.mark.gpu


def W():
    return I.load_workloads()


def no_delay(wl):
    return dataclasses.replace(wl, max_delay=0, delay_probs=(1.0,))


def totals(w, wl):
    """Domain integrals of momentum, energy and total density of a modal state."""
    dx = wl.length / wl.n_elem
    return np.array([w[0, :, 0].sum() * dx, w[1, :, 0].sum() * dx,
                     w[2:, :, 0].sum() * dx])


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_unsync_without_delay_equals_sync_bitwise(precision):
    """The 5-species ignition workload (200 x p3, 4 PEs, WENO) with maximum delay
    0, 30 steps in three calls."""
    wl = no_delay(W()["ignition-5sp-200x3"])
    mech = wl.mechanism()
    prim = wl.primitive(mech)
    a = adg.ADG(mech, [wl], precision=precision)
    b = adg.ADG(mech, [wl], precision=precision)
    a.set_primitive(prim)
    b.set_primitive(prim)
    for _ in range(3):
        a.step(10)
        b.step_unsync(10)
    a.check()
    b.check()
    assert np.array_equal(a.get_state(), b.get_state())
    fa, ca = a.flags()
    fb, cb = b.flags()
    assert np.array_equal(fa, fb) and np.array_equal(ca, cb)
    h = b.unsync_delays()
    sides = 2 * wl.n_pe  # periodic: n_pe faces, two sides each
    assert h[0, 0] == 30 * 3 * sides and h[0, 1:].sum() == 0
    assert h[1, 0] == 30 * 3 * sides and h[1, 1:].sum() == 0


def test_unsync_without_delay_full_size():
    """4096 x p4, 9 species / 21 reactions, 64 PEs (64 co-resident CTAs), maximum
    delay 0, 3 steps: bit for bit the synchronous result."""
    wl = no_delay(W()["ignition-9sp-4096x4"])
    mech = wl.mechanism()
    prim = wl.primitive(mech)
    a = adg.ADG(mech, [wl])
    b = adg.ADG(mech, [wl])
    a.set_primitive(prim)
    b.set_primitive(prim)
    a.step(3)
    b.step_unsync(3)
    a.check()
    b.check()
    assert np.array_equal(a.get_state(), b.get_state())
    assert np.array_equal(a.flags()[0], b.flags()[0])


def test_unsync_with_delays_conservative_and_accurate():
    """The 5-species ignition workload with its maximum delay 2 and AT order 4; PE
    1 idles 300 us per stage, so PEs 0 and 2 run ahead of it."""
    wl = W()["ignition-5sp-200x3"]
    n = 60
    mech = wl.mechanism()
    prim = wl.primitive(mech)
    g = adg.ADG(mech, [wl])
    g.set_primitive(prim)
    g.set_unsync_imbalance(1, 300)
    t0 = totals(g.get_state(), wl)
    g.step_unsync(n)
    g.check()
    w = g.get_state()
    assert np.all(np.isfinite(w))
    h = g.unsync_delays()
    assert h[:, wl.max_delay + 1:].sum() == 0
    assert h[0, 1:].sum() > 0, h  # the common flux level was delayed at some faces
    assert h[0].sum() == n * 3 * 2 * wl.n_pe and h[1].sum() == n * 3 * 2 * wl.n_pe
    # conservation to round-off; momentum relative to the acoustic momentum scale
    # max rho (|u| + a) over the domain
    t1 = totals(w, wl)
    scale = np.array([H.parity_scales(w, mech)[0] * wl.length, abs(t0[1]), abs(t0[2])])
    assert np.all(np.abs(t1 - t0) <= 1e-12 * scale), (t1 - t0) / scale
    # accuracy: against the synchronous oracle, as the seeded-delay oracle run
    sync = O.Oracle(dataclasses.replace(wl, delay_mode=I.DELAY_SYNC), mech)
    sync.set_primitive(prim)
    sync.step(n)
    seeded = O.Oracle(wl, mech)
    seeded.set_primitive(prim)
    seeded.step(n)
    e_seeded = H.parity_error(seeded.state(), sync.state(), mech).max()
    e_unsync = H.parity_error(w, sync.state(), mech).max()
    print("unsync error %.3e, seeded-delay error %.3e, delays %s" % (e_unsync, e_seeded, h))
    assert e_unsync <= 10 * e_seeded + 1e-10, (e_unsync, e_seeded)


def test_unsync_timeout_reports_and_context_recovers():
    """PE 1 never publishes: its neighbours give up after 2^14 polls and the
    launch reports ADG_ERR_TIMEOUT; the same context then runs normally."""
    wl = no_delay(W()["ignition-5sp-200x3"])
    mech = wl.mechanism()
    prim = wl.primitive(mech)
    g = adg.ADG(mech, [wl])
    g.set_primitive(prim)
    g.set_unsync_wait(1 << 14, 1)
    g.step_unsync(3)
    with pytest.raises(adg.AdgError) as ex:
        g.check()
    assert ex.value.code == -7
    g.set_unsync_wait()
    g.set_primitive(prim)
    g.step_unsync(10)
    g.check()
    ref = adg.ADG(mech, [wl])
    ref.set_primitive(prim)
    ref.step(10)
    ref.check()
    assert np.array_equal(g.get_state(), ref.get_state())


def test_unsync_rejects_more_pes_than_fit():
    wl = I.scaled(W()["ignition-9sp-4096x4"], 4096, 2048)
    mech = wl.mechanism()
    g = adg.ADG(mech, [wl])
    g.set_primitive(wl.primitive(mech))
    with pytest.raises(adg.AdgError) as ex:
        g.step_unsync(1)
    assert ex.value.code == -1
    g.step(1)
    g.check()
