"""Domain decomposition through the CUDA library: the subdomains of one problem,
held as instances of one context (or one context each, as ranks would hold
them), step by adg_step_stage and swap their boundary blocks by
adg_part_block between the halves of every stage. The assembled owned
elements equal the whole-domain CUDA run bit for bit, and the FP64 oracle's
whole-domain run within the parity bar. One GPU: the subdomains never wait on
one another inside a kernel; the host orders the halves and the copies on one
stream."""
import dataclasses

import numpy as np
import pytest

import oracle as O
from paper_2501_01747_gb300 import adg
from paper_2501_01747_gb300 import domain as D
from paper_2501_01747_gb300 import inputs as I
from tests import helpers as H

pytestmark = pytest.mark.gpu

TOL = 1e-10


def W():
    return I.load_workloads()


def shock_case():
    """97 elements of the 9-species detonation shape in 32 ragged PEs, p = 2,
    HLLC, wall and outflow, SAA delays, WENO limiting at the cut faces."""
    base = W()["detonation-9sp-16384x3"]
    wl = I.scaled(base, 97, 32)
    wl.p, wl.at_order = 2, 3
    wl.dt = base.dt * 0.2
    return wl


def cases():
    ign = W()["ignition-5sp-200x3"]
    return {
        "periodic-2": (ign, [(0, 2), (2, 4)], 40, "fp64"),
        "periodic-one-pe-each": (ign, [(0, 1), (1, 2), (2, 3), (3, 4)], 40, "fp64"),
        "periodic-lserk4": (dataclasses.replace(ign, integrator=I.RK_LS4), [(0, 1), (1, 4)],
                            30, "fp64"),
        "bounded-shock-3": (shock_case(), [(0, 1), (1, 2), (2, 32)], 60, "fp64"),
        "bounded-shock-3-mixed": (shock_case(), [(0, 1), (1, 2), (2, 32)], 60, "mixed"),
        "periodic-2-f32chem": (ign, [(0, 2), (2, 4)], 40, "mixed_f32chem"),
    }


def whole_cuda(wl, mech, prim, steps, precision):
    g = adg.ADG(mech, [wl], precision=precision)
    g.set_primitive(prim)
    g.step(steps)
    g.check()
    w, cnt = g.get_state(), g.flags()[1]
    g.close()
    return w, cnt


def parts_in_one_context(wl, mech, prim, ranges, steps, precision):
    subs = [D.subdomain(wl, pb, pe) for pb, pe in ranges]
    g = adg.ADG(mech, subs, precision=precision)
    parts = [D.AdgPart(g, k) for k in range(len(subs))]
    for k, p in enumerate(parts):
        g.set_primitive(D.local_slice(prim, wl.n_elem, p.elem0, p.n_local, axis=1), k)
    D.advance(steps, adg.rk_stages(wl), g.step_stage, D.LocalExchange(parts))
    g.check()
    w = np.concatenate([D.owned(g.get_state(k), *p.cut, axis=1)
                        for k, p in enumerate(parts)], axis=1)
    cnt = np.concatenate([D.owned(g.flags(k)[1], *p.cut, axis=0)
                          for k, p in enumerate(parts)])
    g.close()
    return w, cnt


@pytest.mark.parametrize("name", list(cases()))
def test_subdomains_match_the_whole_domain_bit_for_bit(name):
    wl, ranges, steps, prec = cases()[name]
    mech = wl.mechanism()
    prim = wl.primitive(mech)
    ref, ref_cnt = whole_cuda(wl, mech, prim, steps, prec)
    got, cnt = parts_in_one_context(wl, mech, prim, ranges, steps, prec)
    assert np.array_equal(got, ref), np.abs(got - ref).max()
    assert np.array_equal(cnt, ref_cnt)
    if prec == "fp64":
        o = O.Oracle(wl, mech)
        o.set_primitive(prim)
        o.step(steps)
        assert H.parity_error(got, o.state(), mech).max() <= TOL


def test_one_context_per_subdomain():
    """Each subdomain in a context of its own (what one rank holds), stepped
    half-stage by half-stage on one stream."""
    wl, ranges, steps, _ = cases()["bounded-shock-3"]
    mech = wl.mechanism()
    prim = wl.primitive(mech)
    ref, _ = whole_cuda(wl, mech, prim, steps, "fp64")
    ctxs, parts = [], []
    for pb, pe in ranges:
        g = adg.ADG(mech, [D.subdomain(wl, pb, pe)])
        p = D.AdgPart(g, 0)
        g.set_primitive(D.local_slice(prim, wl.n_elem, p.elem0, p.n_local, axis=1))
        ctxs.append(g)
        parts.append(p)

    def stage(s, half):
        for g in ctxs:
            g.step_stage(s, half)

    D.advance(steps, 3, stage, D.LocalExchange(parts))
    got = np.concatenate([D.owned(g.get_state(), *p.cut, axis=1)
                          for g, p in zip(ctxs, parts)], axis=1)
    for g in ctxs:
        g.check()
        g.close()
    assert np.array_equal(got, ref)


def test_decomposed_step_captured_as_a_graph():
    """The per-stage exchange only enqueues kernels and device copies (the
    pre-limit history slot comes from the device step counter), so one step
    captured as a CUDA graph and replayed gives the whole-domain result too."""
    import torch
    wl, ranges, steps, _ = cases()["bounded-shock-3"]
    mech = wl.mechanism()
    prim = wl.primitive(mech)
    ref, ref_cnt = whole_cuda(wl, mech, prim, steps, "fp64")
    subs = [D.subdomain(wl, pb, pe) for pb, pe in ranges]
    g = adg.ADG(mech, subs)
    parts = [D.AdgPart(g, k) for k in range(len(subs))]
    for k, p in enumerate(parts):
        g.set_primitive(D.local_slice(prim, wl.n_elem, p.elem0, p.n_local, axis=1), k)
    ex = D.LocalExchange(parts)
    D.advance(5, 3, g.step_stage, ex)  # plain launches first
    graph = D.capture_step(3, g.step_stage, ex)
    for _ in range(steps - 5):
        graph.replay()
    torch.cuda.synchronize()
    g.check()
    got = np.concatenate([D.owned(g.get_state(k), *p.cut, axis=1)
                          for k, p in enumerate(parts)], axis=1)
    cnt = np.concatenate([D.owned(g.flags(k)[1], *p.cut, axis=0)
                          for k, p in enumerate(parts)])
    g.close()
    assert np.array_equal(got, ref)
    assert np.array_equal(cnt, ref_cnt)


def test_full_size_ignition_in_four_subdomains():
    """The 9-species ignition shape at full size (4096 x p4, 64 PEs, SAA delays up
    to 4, AT order 5) in four subdomains of 16 PEs, mixed precision."""
    wl = W()["ignition-9sp-4096x4"]
    mech = wl.mechanism()
    prim = wl.primitive(mech)
    ranges = D.split_pes(wl.n_pe, 4)
    ref, ref_cnt = whole_cuda(wl, mech, prim, 24, "mixed")
    got, cnt = parts_in_one_context(wl, mech, prim, ranges, 24, "mixed")
    assert np.array_equal(got, ref)
    assert np.array_equal(cnt, ref_cnt)


def test_subdomain_calls_reject_bad_arguments():
    import torch
    wl = W()["ignition-5sp-200x3"]
    mech = wl.mechanism()
    bounded = shock_case()
    g = adg.ADG(mech, [D.subdomain(wl, 0, 4), D.subdomain(wl, 1, 2)])
    blk = torch.zeros((g.nv, wl.p + 1), dtype=torch.float64, device="cuda")
    with pytest.raises(adg.AdgError):
        g.part_block(0, D.PART_INPUT, 0, 0, blk, False)   # the whole domain has no cut
    with pytest.raises(adg.AdgError):
        g.part_block(1, 2, 0, 0, blk, False)              # no such block
    with pytest.raises(adg.AdgError):
        g.part_block(1, D.PART_INPUT, 0, 3, blk, True)    # stage 3 of SSP-RK3
    with pytest.raises(adg.AdgError):
        g.step_stage(3, 0)
    with pytest.raises(adg.AdgError):
        g.step_unsync(1, k=1)                             # whole domains only
    g.close()
    bm = bounded.mechanism()
    b = adg.ADG(bm, [D.subdomain(bounded, 0, 4)])
    bblk = torch.zeros((b.nv, bounded.p + 1), dtype=torch.float64, device="cuda")
    with pytest.raises(adg.AdgError):
        b.part_block(0, D.PART_PRELIMIT, 0, 0, bblk, True)  # left side is the wall
    b.close()
    with pytest.raises(adg.AdgError):
        adg.ADG(mech, [dataclasses.replace(wl, pe_begin=2, pe_end=1)])
    with pytest.raises(adg.AdgError):
        adg.ADG(mech, [I.viscous(D.subdomain(wl, 0, 2))])
