"""Batches of independent runs (pic_batch_*) against the FP64 oracle.

One batched step advances every run with one plan, one persistent
particle-step launch over the work items of all runs and one launch per field
kernel.  Each run must give what it gives alone: the oracle's fields and
particles within the single-run tolerances, whatever the mix (patch shapes,
periodic and open boundaries, laser, filter, moving window), with and
without graph replay, after runs join, leave or step alone in between.
"""
import math

import numpy as np
import pytest

from paper_1912_04064_gb300 import pic
from paper_1912_04064_gb300 import workloads as W

from parity_utils import field_errors, match_particles, pair, particle_errors

pytestmark = pytest.mark.gpu

TOL64 = 1e-12
EB = ("Ex", "Ey", "Ez", "Bx", "By", "Bz", "Bmx", "Bmy", "Bmz")


def _open_run(nx=128, ny=64, patch=(16, 16), laser=True, filter_passes=0):
    run, _ = W.lwfa_2d(n=(nx, ny), d=(0.125, 0.5), patch=patch, ppc=(2, 2), ramp=4.0)
    run["moving_window"] = None
    run["laser"] = ({"a0": 2.0, "waist": 6.0, "tau": 4.0, "t_peak": 0.5, "y_center": ny * 0.25}
                    if laser else None)
    run["filter_passes"] = filter_passes
    return run


def _window_run():
    run, parts = W.lwfa_2d(n=(128, 64), d=(0.125, 0.5), patch=(16, 16), ppc=(2, 2),
                           ramp=6.0, t_mw=0.3, a0=1.0, waist=5.0, tau=3.0)
    run["laser"]["t_peak"] = 6.0
    rng = np.random.default_rng(9)
    parts["ux"] = rng.normal(0, 0.3, parts["x"].size)
    parts["uy"] = rng.normal(0, 0.3, parts["x"].size)
    return run, parts


def _case(kind, seed, prec="fp64", **kw):
    """(oracle, context, tolerance) of one run of the mix."""
    if kind == "window":
        run, parts = _window_run()
        o, g = pair(run, parts, prec=prec, background=("neutralising", 0.0), **kw)
        return o, g, 1e-12
    if kind == "periodic16":
        run = W.periodic_run((64, 48), (0.1, 0.1), (16, 16))
    elif kind == "periodic8":
        run = W.periodic_run((64, 64), (0.1, 0.1), (8, 8))
    elif kind == "periodic_rect":
        run = W.periodic_run((96, 32), (0.1, 0.1), (32, 16))
    elif kind == "open_laser":
        run = _open_run()
    elif kind == "open_filter":
        run = _open_run(laser=False, filter_passes=2)
    else:
        raise ValueError(kind)
    parts = W.small_random_particles(run, 12000, seed=seed, uth=0.6)
    fields = W.random_fields(W.field_shape(run), seed=seed + 1, amp=0.1)
    o, g = pair(run, parts, fields, prec=prec, **kw)
    return o, g, TOL64


def _check(o, g, tol):
    errs = field_errors(o, g)
    bad = {k: v for k, v in errs.items() if not v <= tol}
    assert not bad, bad
    perr = particle_errors(o, g)
    assert max(perr.values()) <= tol, perr
    do, dg = o.diag(), g.pic_diag()
    assert dg["np"] == do["np"] and dg["step"] == do["step"] and dg["shifts"] == do["shifts"]


@pytest.mark.parametrize("use_graph", [True, False])
@pytest.mark.parametrize("mix", ["mixed", "uniform16"])
def test_batch_matches_oracle_per_run(mix, use_graph):
    kinds = (["periodic16", "periodic8", "periodic_rect", "open_laser", "open_filter"]
             if mix == "mixed" else ["periodic16", "open_laser", "open_filter"])
    cases = [_case(k, 100 + 7 * i) for i, k in enumerate(kinds)]
    b = pic.Batch(use_graph=use_graph)
    b.pic_batch_set([g for _, g, _ in cases])
    for _ in range(3):
        for o, _, _ in cases:
            o.step(1)
        b.pic_batch_step(1)
    for o, g, tol in cases:
        _check(o, g, tol)
    d = b.pic_batch_get_diag()
    assert d["steps"] == 3 and d["nruns"] == len(cases) and d["builds"] == 1
    # plan + particle step + E + B + SM (open runs) + filter (one run): one
    # launch each per step for the whole batch
    assert d["launches"] == 3 * 6
    b.close()


def test_batch_moving_window_and_many_steps():
    """A moving-window run (shifts fall due inside the batched loop) next to
    a periodic run, stepped through several shifts."""
    cases = [_case("window", 0), _case("periodic16", 5)]
    run_w, _ = _window_run()
    b = pic.Batch()
    b.pic_batch_set([g for _, g, _ in cases])
    nsteps = 2 * math.ceil(16 * 0.125 / run_w["dt"]) + 12
    for _ in range(nsteps):
        for o, _, _ in cases:
            o.step(1)
    b.pic_batch_step(nsteps)
    assert cases[0][1].pic_diag()["shifts"] >= 2
    for o, g, tol in cases:
        _check(o, g, 1e-12)
    b.close()


def test_runs_join_leave_and_step_alone():
    """Membership changes and single-run steps between batched steps (the
    batch rebuilds its device arguments when a run's parity moved)."""
    A = _case("periodic16", 11)
    B = _case("open_laser", 12)
    C = _case("periodic8", 13)
    b = pic.Batch()
    b.pic_batch_set([A[1], B[1]])
    for o in (A[0], B[0]):
        o.step(2)
    b.pic_batch_step(2)
    # C joins; B steps alone once first (parity now differs from A's)
    B[0].step(1)
    B[1].pic_step(1)
    b.pic_batch_set([A[1], B[1], C[1]])
    for o in (A[0], B[0], C[0]):
        o.step(3)
    b.pic_batch_step(3)
    # A leaves
    b.pic_batch_set([B[1], C[1]])
    for o in (B[0], C[0]):
        o.step(1)
    b.pic_batch_step(1)
    A[0].step(1)
    A[1].pic_step(1)
    for o, g, tol in (A, B, C):
        _check(o, g, tol)
    assert b.pic_batch_get_diag()["builds"] == 3
    b.close()


def test_batch_fp32_equals_runs_alone_within_fp32_bounds():
    """FP32 batch against the same runs stepped alone in FP32: both are FP32
    roundings of the oracle's step (single step from an FP64 state)."""
    kinds = ["periodic16", "open_laser", "periodic8"]
    batched = [_case(k, 40 + i, prec="fp32") for i, k in enumerate(kinds)]
    alone = [_case(k, 40 + i, prec="fp32") for i, k in enumerate(kinds)]
    b = pic.Batch()
    b.pic_batch_set([g for _, g, _ in batched])
    b.pic_batch_step(1)
    for (o, gb, _), (_, ga, _) in zip(batched, alone):
        o.step(1)
        ga.pic_step(1)
        for k in EB + ("Jx", "Jy", "Jz"):
            ref = o.field(k)
            scale = max(np.max(np.abs(ref)), 1e-30)
            eb = np.max(np.abs(gb.pic_get_field(k) - ref)) / scale
            ea = np.max(np.abs(ga.pic_get_field(k) - ref)) / scale
            tol = 2e-5 if k.startswith("J") else 2e-6
            assert eb <= tol and ea <= tol, (k, eb, ea)
        pb, pa = gb.pic_get_particles(), ga.pic_get_particles()
        pa = match_particles(pb, pa)
        for k in pb:
            assert np.max(np.abs(pb[k] - pa[k])) <= 1e-5 * max(np.max(np.abs(pa[k])), 1.0), k
    b.close()


def test_faulted_run_leaves_batch_others_continue():
    """A run whose patch capacity overflows inside the batch (no auto-grow
    replay in batches) holds PIC_EOVERFLOW and leaves; the others keep
    matching the oracle."""
    run = W.periodic_run((64, 64), (0.1, 0.1), (16, 16))
    rng = np.random.default_rng(5)
    n = 20000
    x = rng.uniform(0, 6.4, n)
    y = rng.uniform(0, 6.4, n)
    conv = {"x": x, "y": y, "ux": -2.0 * np.sign(x - 3.2), "uy": -2.0 * np.sign(y - 3.2),
            "uz": np.zeros(n), "w": np.full(n, 0.01)}
    bad = pic.Pic(pic.config_from_run(run, "fp64", capacity_factor=1.0, capacity_min=32))
    bad.pic_load_particles(conv)
    good = _case("periodic16", 21)
    b = pic.Batch()
    b.pic_batch_set([bad, good[1]])
    status = None
    steps = 0
    for _ in range(40):
        good[0].step(1)
        steps += 1
        try:
            b.pic_batch_step(1)
        except pic.PicError as e:
            status = e.status
            break
    assert status == pic.PIC_EOVERFLOW
    assert b.pic_batch_size() == 1
    with pytest.raises(pic.PicError) as e:
        bad.pic_step(1)
    assert e.value.status == pic.PIC_ESTATE
    good[0].step(2)
    b.pic_batch_step(2)
    _check(good[0], good[1], TOL64)
    b.close()


def test_batch_rules():
    A = _case("periodic16", 1)
    B32 = _case("periodic16", 2, prec="fp32")
    empty = pic.Pic(pic.config_from_run(W.periodic_run((64, 64), (0.1, 0.1), (16, 16)), "fp64"))
    b = pic.Batch()
    for runs, status in (([A[1], B32[1]], pic.PIC_EINVAL), ([A[1], A[1]], pic.PIC_EINVAL),
                         ([A[1], empty], pic.PIC_ESTATE)):
        with pytest.raises(pic.PicError) as e:
            b.pic_batch_set(runs)
        assert e.value.status == status
    assert b.pic_batch_size() == 0
    arr = (pic.C.c_void_p * 65)(*([A[1].h.value] * 65))
    assert pic.lib().pic_batch_set(b.h, arr, 65) == pic.PIC_EINVAL
    b.pic_batch_step(1)  # empty batch: nothing to do
    b.pic_batch_set([A[1]])
    A[0].step(1)
    b.pic_batch_step(1)
    _check(A[0], A[1], TOL64)
    b.close()
