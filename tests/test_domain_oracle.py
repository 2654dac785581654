"""Domain decomposition on the CPU: subdomains of the oracle, exchanging their
boundary blocks through `domain.LocalExchange` (one process) or
`domain.DistExchange` (gloo ranks, spawned processes, rendezvous on 127.0.0.1),
advance exactly as the whole-domain oracle does: the assembled owned elements
and their troubled-cell counts are bit-identical after many steps. The cases
cover periodic and bounded domains, SAA and CAA delays, WENO on a shock that
crosses the cut faces, LSERK4, ragged PE splits and one PE per subdomain. A
planted mistake (one exchange left out) must break the identity. The layouts
are pinned by hand and against the library's host-side layout."""
import dataclasses
import os
import socket
import sys

import numpy as np
import pytest

import oracle as O
from paper_2501_01747_gb300 import domain as D
from paper_2501_01747_gb300 import inputs as I

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def W():
    return I.load_workloads()


def shock_case(n_pe=32):
    """The 9-species detonation shape on 97 elements (ragged PEs: PE k owns
    [floor(97 k / n_pe), ...)), p = 2, HLLC, reflecting wall and outflow, SAA
    delays up to 3, WENO. With 32 PEs of 3 elements the hot gas fills elements
    0-4, so the faces at elements 3 and 6 are limited at nearly every stage."""
    base = W()["detonation-9sp-16384x3"]
    wl = I.scaled(base, 97, n_pe)
    wl.p, wl.at_order = 2, 3
    wl.dt = base.dt * 0.2
    return wl


def cases():
    ign = W()["ignition-5sp-200x3"]
    caa = dataclasses.replace(ign, delay_mode=I.DELAY_CAA, max_delay=3)
    ls4 = dataclasses.replace(ign, integrator=I.RK_LS4)
    return {
        "periodic-saa-2": (ign, [(0, 2), (2, 4)], 40),
        "periodic-one-pe-each": (ign, [(0, 1), (1, 2), (2, 3), (3, 4)], 40),
        "periodic-caa-3": (caa, D.split_pes(4, 3), 40),
        "periodic-lserk4-2": (ls4, [(0, 1), (1, 4)], 30),
        "bounded-shock-3": (shock_case(), [(0, 1), (1, 2), (2, 32)], 60),
    }


def whole_run(wl, mech, prim, steps):
    o = O.Oracle(wl, mech)
    o.set_primitive(prim)
    o.step(steps)
    return o.state(), o.flags()[1]


def make_parts(wl, mech, prim, ranges):
    parts = []
    for pb, pe in ranges:
        o = O.Oracle(D.subdomain(wl, pb, pe), mech)
        o.set_primitive(D.local_slice(prim, wl.n_elem, o.elem0, o.n_local, axis=1))
        parts.append(o)
    return parts


def run_local(wl, mech, prim, ranges, steps, skip=None):
    parts = make_parts(wl, mech, prim, ranges)
    ex = D.LocalExchange(parts)

    def exchange(what, s):
        if what != skip:
            ex(what, s)

    def stage(s, half):
        for o in parts:
            o.stage(s, half)

    D.advance(steps, O.rk_stages(wl.integrator), stage, exchange)
    w = np.concatenate([D.owned(o.state(), *o.cut, axis=1) for o in parts], axis=1)
    cnt = np.concatenate([D.owned(o.flags()[1], *o.cut, axis=0) for o in parts])
    return w, cnt


def cut_elements(wl, ranges):
    """Whole-domain indices of the elements on both sides of every cut face."""
    out = set()
    for pb, _ in ranges:
        if pb > 0 or wl.bc_left == I.BC_PERIODIC:
            e0 = pb * wl.n_elem // wl.n_pe
            out.update({e0, (e0 - 1) % wl.n_elem})
    return sorted(out)


@pytest.mark.parametrize("name", list(cases()))
def test_decomposed_run_is_bit_identical_to_the_whole_domain(name):
    wl, ranges, steps = cases()[name]
    mech = wl.mechanism()
    prim = wl.primitive(mech)
    ref, ref_cnt = whole_run(wl, mech, prim, steps)
    got, cnt = run_local(wl, mech, prim, ranges, steps)
    assert got.shape == ref.shape
    assert np.array_equal(got, ref), np.abs(got - ref).max()
    assert np.array_equal(cnt, ref_cnt)
    # the run used delayed levels at the cut faces (whole-domain face numbers)
    npf = wl.n_pe if wl.bc_left == I.BC_PERIODIC else wl.n_pe - 1
    cuts = [(pb - 1) % wl.n_pe for pb, _ in ranges if pb > 0 or wl.bc_left == I.BC_PERIODIC]
    assert all(0 <= f < npf for f in cuts) and cuts
    delays = [O.delay(wl, n, f) for n in range(wl.at_order + 3, steps) for f in cuts]
    assert max(delays) > 0


def test_shock_case_limits_elements_beside_a_cut():
    """The bounded case exercises the limiter's exchange: elements beside a cut
    face are flagged troubled in the whole-domain run."""
    wl, ranges, steps = cases()["bounded-shock-3"]
    mech = wl.mechanism()
    _, cnt = whole_run(wl, mech, wl.primitive(mech), steps)
    assert cut_elements(wl, ranges) == [2, 3, 5, 6]
    assert (cnt[[2, 3, 5, 6]] > steps).all()


@pytest.mark.parametrize("skip", [D.PART_INPUT, D.PART_PRELIMIT])
def test_leaving_out_an_exchange_breaks_the_identity(skip):
    wl, ranges, steps = cases()["bounded-shock-3"]
    mech = wl.mechanism()
    prim = wl.primitive(mech)
    ref, _ = whole_run(wl, mech, prim, steps)
    got, _ = run_local(wl, mech, prim, ranges, steps, skip=skip)
    assert not np.array_equal(got, ref)


def test_layouts_by_hand():
    ign = W()["ignition-5sp-200x3"]  # 200 elements, 4 PEs of 50, periodic
    mech = ign.mechanism()

    def lay(wl, pb, pe):
        o = O.Oracle(D.subdomain(wl, pb, pe), mech)
        return o.n_local, o.elem0, o.cut

    assert lay(ign, 0, 1) == (52, -1, (True, True))      # buffers: elements 199 and 50
    assert lay(ign, 1, 3) == (102, 49, (True, True))     # 49 | 50..149 | 150
    assert lay(ign, 0, 4) == (200, 0, (False, False))    # the whole domain
    shock = shock_case(7)  # 97 elements, 7 PEs: PE k owns [floor(97 k / 7), ...)
    sm = shock.mechanism()
    o = O.Oracle(D.subdomain(shock, 0, 3), sm)           # owns 0..40, buffer 41
    assert (o.n_local, o.elem0, o.cut) == (42, 0, (False, True))
    o = O.Oracle(D.subdomain(shock, 3, 7), sm)           # buffer 40, owns 41..96
    assert (o.n_local, o.elem0, o.cut) == (57, 40, (True, False))
    assert D.split_pes(7, 3) == [(0, 2), (2, 4), (4, 7)]
    assert D.neighbours(0, 2, True) == (1, 1) and D.neighbours(0, 3, False) == (None, 1)


def test_library_layout_agrees_with_the_oracle():
    from paper_2501_01747_gb300 import adg
    for wl in (W()["ignition-5sp-200x3"], shock_case(7)):
        mech = wl.mechanism()
        for pb in range(wl.n_pe):
            for pe in range(pb + 1, wl.n_pe + 1):
                sub = D.subdomain(wl, pb, pe)
                o = O.Oracle(sub, mech)
                assert adg.part_layout(sub) == (o.n_local, o.elem0, int(o.cut[0]),
                                                int(o.cut[1]))
                # the delays of the subdomain's faces are the whole domain's
                tab = adg.delay_table(sub, 3, 4)
                npf_w = wl.n_pe if wl.bc_left == I.BC_PERIODIC else wl.n_pe - 1
                first = pb - int(o.cut[0])
                ref = np.array([[O.delay(wl, 3 + s, (first + f) % npf_w)
                                 for f in range(tab.shape[1])] for s in range(4)])
                assert np.array_equal(tab, ref)


def test_bad_subdomains_are_rejected():
    ign = W()["ignition-5sp-200x3"]
    mech = ign.mechanism()
    for pb, pe in [(2, 2), (3, 1), (0, 5), (-1, 2)]:
        with pytest.raises(ValueError):
            O.Oracle(D.subdomain(ign, pb, pe), mech)
    with pytest.raises(ValueError):
        D.split_pes(3, 4)


# ---- gloo ranks ----

def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, name, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    sys.path.insert(0, ROOT)
    import torch
    import torch.distributed as dist
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        wl, ranges, steps = _gloo_cases()[name]
        mech = wl.mechanism()
        prim = wl.primitive(mech)
        part = make_parts(wl, mech, prim, [ranges[rank]])[0]
        shape = (part.nv, wl.p + 1)
        ex = D.DistExchange(dist, part, rank, world, wl.bc_left == I.BC_PERIODIC,
                            to_wire=lambda b: torch.from_numpy(np.ascontiguousarray(b)),
                            empty=lambda: torch.zeros(shape, dtype=torch.float64),
                            from_wire=lambda t: t.numpy())
        D.advance(steps, O.rk_stages(wl.integrator), part.stage, ex)
        q.put((rank, D.owned(part.state(), *part.cut, axis=1),
               D.owned(part.flags()[1], *part.cut, axis=0)))
    finally:
        dist.destroy_process_group()


def _gloo_cases():
    ign = W()["ignition-5sp-200x3"]
    return {"periodic-2": (ign, [(0, 1), (1, 4)], 30),
            "bounded-3": (shock_case(), [(0, 1), (1, 2), (2, 32)], 40)}


@pytest.mark.parametrize("name,world", [("periodic-2", 2), ("bounded-3", 3)])
def test_gloo_ranks_match_the_whole_domain(name, world):
    import torch.multiprocessing as mp
    wl, ranges, steps = _gloo_cases()[name]
    mech = wl.mechanism()
    ref, ref_cnt = whole_run(wl, mech, wl.primitive(mech), steps)
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, world, port, name, q)) for r in range(world)]
    for p in procs:
        p.start()
    res = {}
    for _ in range(world):
        r, w, cnt = q.get(timeout=300)
        res[r] = (w, cnt)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    got = np.concatenate([res[r][0] for r in range(world)], axis=1)
    cnt = np.concatenate([res[r][1] for r in range(world)])
    assert np.array_equal(got, ref)
    assert np.array_equal(cnt, ref_cnt)
