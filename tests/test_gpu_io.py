"""adg_step_io, the step with its host copies overlapped group by group,
against adg_write_states + adg_step + adg_read_states on the same inputs: the
host results, the device states and the troubled-cell counts are the same to
the bit, step after step, with each step's input taken from the previous
step's output (a host-side time loop). The instances span three degrees and
two precisions (six groups; groups of two or more instances are cut into
parts, stepped one after the other while the other parts' copies run). A
second pair of buffers makes the call capture its graph again; pageable
buffers and a one-group context take the sequential path."""
import numpy as np
import pytest

from paper_2501_01747_gb300 import adg
from paper_2501_01747_gb300 import inputs as I

pytestmark = pytest.mark.gpu


def ensemble_case():
    """The first ten ensemble instances (degrees 2-4, their own temperatures,
    fuel fractions, delays and dt) on 40 + 8 i elements in 2 PEs; even
    instances in ADG_MIXED, odd ones in FP64."""
    wls = [I.scaled(w, 40 + 8 * i, 2) for i, w in enumerate(I.ensemble_workloads(10))]
    prec = ["mixed" if i % 2 == 0 else "fp64" for i in range(len(wls))]
    return wls, prec


def make(wls, prec, mech):
    g = adg.ADG(mech, wls, precision=prec)
    for k, w in enumerate(wls):
        g.set_primitive(w.primitive(mech), k)
    return g


def flags(g, n):
    return [g.flags(k)[1].copy() for k in range(n)]


def test_step_io_equals_write_step_read_to_the_bit():
    import torch
    wls, prec = ensemble_case()
    mech = wls[0].mechanism()
    assert len({(w.p, x) for w, x in zip(wls, prec)}) >= 4
    a, b = make(wls, prec, mech), make(wls, prec, mech)
    n = a.states_doubles()
    pin = lambda: torch.empty(n, dtype=torch.float64, pin_memory=True)
    a_in, a_out, b_in, b_out = pin(), pin(), pin(), pin()
    a.read_states(a_in.numpy())
    b.read_states(b_in.numpy())
    torch.cuda.synchronize()
    assert np.array_equal(a_in.numpy(), b_in.numpy())
    for it in range(6):
        a.write_states(a_in.numpy())
        a.step(1)
        a.read_states(a_out.numpy())
        b.step_io(b_in.numpy(), b_out.numpy())
        torch.cuda.synchronize()
        assert np.array_equal(a_out.numpy(), b_out.numpy()), it
        assert not np.array_equal(a_out.numpy(), a_in.numpy())
        # the next step starts from this one's result, perturbed on the host
        nxt = a_out.numpy() * (1.0 + 1e-9 * (it + 1))
        a_in.numpy()[:] = nxt
        b_in.numpy()[:] = nxt
    for k in range(len(wls)):
        assert np.array_equal(a.get_state(k), b.get_state(k)), k
        assert a.steps_done(k) == b.steps_done(k) == 6
    for fa, fb in zip(flags(a, len(wls)), flags(b, len(wls))):
        assert np.array_equal(fa, fb)
    # a second pair of buffers (a new capture), then pageable buffers
    c_in, c_out = pin(), pin()
    c_in.numpy()[:] = b_out.numpy()
    a_in.numpy()[:] = b_out.numpy()
    a.write_states(a_in.numpy())
    a.step(1)
    a.read_states(a_out.numpy())
    b.step_io(c_in.numpy(), c_out.numpy())
    torch.cuda.synchronize()
    assert np.array_equal(a_out.numpy(), c_out.numpy())
    page_in, page_out = c_out.numpy().copy(), np.zeros(n)
    a_in.numpy()[:] = page_in
    a.write_states(a_in.numpy())
    a.step(1)
    a.read_states(a_out.numpy())
    b.step_io(page_in, page_out)
    torch.cuda.synchronize()
    assert np.array_equal(a_out.numpy(), page_out)
    a.check()
    b.check()
    a.close()
    b.close()


def test_step_io_with_one_group_runs_the_calls_in_sequence():
    import torch
    base = I.load_workloads()["ignition-5sp-200x3"]
    wls = [base, I.scaled(base, 97, 7)]
    mech = base.mechanism()
    a, b = make(wls, ["fp64"] * 2, mech), make(wls, ["fp64"] * 2, mech)
    n = a.states_doubles()
    buf = [torch.empty(n, dtype=torch.float64, pin_memory=True) for _ in range(3)]
    a.read_states(buf[0].numpy())
    torch.cuda.synchronize()
    a.write_states(buf[0].numpy())
    a.step(1)
    a.read_states(buf[1].numpy())
    b.step_io(buf[0].numpy(), buf[2].numpy())
    torch.cuda.synchronize()
    assert np.array_equal(buf[1].numpy(), buf[2].numpy())
    a.close()
    b.close()
