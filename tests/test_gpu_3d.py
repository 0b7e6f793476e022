"""3D3V path (dims = 3) against the 3D FP64 oracle, through the C-ABI.

Single steps from identical states (FP64 1e-12 relative max-norm per
component, J, E, B, Bm and particles), periodic and open boundaries with the
laser, reflection and removal, patch shapes, empty and corner cases, the
moving window with the upper-half plasma filled on the device, FP32 bounds,
and the full 1024 x 256 x 256 config in the benchmark's launch
configuration checked through its invariants.
"""
import math

import numpy as np
import pytest

from oracle.oracle import Oracle3
from paper_1912_04064_gb300 import pic
from paper_1912_04064_gb300 import workloads as W

from parity_utils import match_particles

pytestmark = pytest.mark.gpu

NAMES = ("Ex", "Ey", "Ez", "Bx", "By", "Bz", "Bmx", "Bmy", "Bmz", "Jx", "Jy", "Jz")
EB = NAMES[:9]
TOL64 = 1e-12
KEYS = ("x", "y", "z", "ux", "uy", "uz", "w")


def rel(a, b):
    s = np.max(np.abs(b))
    return float(np.max(np.abs(a - b)) / s) if s > 0 else float(np.max(np.abs(a)))


def pair3(run, parts=None, fields=None, prec="fp64", background=None, fill=False, **kw):
    o = Oracle3(run, track_continuity=True)
    g = pic.Pic(pic.config_from_run(run, prec, **kw))
    if fill:
        o.fill_plasma()
        g.pic_load_plasma()
    if parts is not None:
        o.load(parts)
        g.pic_load_particles(parts)
    if fields:
        for k, v in fields.items():
            o.set_field(k, v)
            g.pic_set_field(k, v)
    if background is not None:
        o.set_background(*background)
        g.pic_set_background(*background)
    return o, g


def field_errs(o, g, names=NAMES):
    return {k: rel(g.pic_get_field(k), o.field(k)) for k in names}


def particle_errs(o, g):
    a, b = g.pic_get_particles(), o.particles()
    assert a["x"].size == b["x"].size, (a["x"].size, b["x"].size)
    if a["x"].size == 0:
        return {k: 0.0 for k in KEYS}
    b = match_particles3(a, b)
    return {k: rel(a[k], b[k]) for k in KEYS}


def match_particles3(a, b):
    from scipy.spatial import cKDTree
    A = np.stack([a[k] for k in KEYS], 1)
    B = np.stack([b[k] for k in KEYS], 1)
    scale = np.maximum(np.max(np.abs(B), 0), 1e-30)
    _, idx = cKDTree(B / scale).query(A / scale, k=1)
    assert np.unique(idx).size == idx.size, "particle pairing is not one-to-one"
    return {k: b[k][idx] for k in KEYS}


def _assert(errs, tol):
    bad = {k: v for k, v in errs.items() if not v <= tol}
    assert not bad, bad


@pytest.mark.parametrize("patch", [(8, 8, 8), (16, 8, 4), (4, 8, 16), (16, 16, 16)])
def test_single_step_fp64_periodic(patch):
    """Patches whose E and Bm tile fits in shared memory stage it by TMA;
    16^3 (a 208 KB FP32 tile) gathers from HBM through L1."""
    run = W.periodic_run3((32, 16, 16), (0.1, 0.12, 0.15), patch)
    parts = W.small_random_particles3(run, 30000, seed=1, uth=0.5)
    fields = W.random_fields(W.field_shape3(run), seed=2, amp=0.1)
    o, g = pair3(run, parts, fields)
    for _ in range(2):
        o.step(1)
        g.pic_step(1)
        _assert(field_errs(o, g), TOL64)
    _assert(particle_errs(o, g), TOL64)
    d, do = g.pic_diag(), o.diag()
    assert d["np"] == do["np"]
    assert d["continuity"] < 1e-9 * max(1.0, abs(do["charge"]))


def _open3(laser=True):
    run = W.lwfa_3d(n=(64, 32, 32), d=(0.125, 0.5, 0.5), patch=(16, 8, 8), a0=2.0, waist=5.0,
                    tau=3.0, upper_half=False)
    run["moving_window"] = None
    run["laser"]["t_peak"] = 0.5
    if not laser:
        run["laser"] = None
    return run


@pytest.mark.parametrize("graph", [True, False])
def test_open_laser_reflect_remove_fp64(graph):
    run = _open3()
    parts = W.small_random_particles3(run, 40000, seed=5, uth=0.6)
    fields = W.random_fields(W.field_shape3(run), seed=6, amp=0.1)
    o, g = pair3(run, parts, fields, use_graph=graph)
    for _ in range(3):
        o.step(1)
        g.pic_step(1)
        _assert(field_errs(o, g), TOL64)
    _assert(particle_errs(o, g), TOL64)


@pytest.mark.parametrize("case", ["empty_patches", "corners"])
def test_edge_cases_fp64(case):
    run = W.periodic_run3((32, 16, 16), (0.1, 0.1, 0.1), (8, 8, 8))
    rng = np.random.default_rng(7)
    n = 4000
    if case == "empty_patches":
        x = rng.uniform(0.8, 1.6, n)       # patch column 1 only
        y = rng.uniform(0.0, 1.6, n)
        z = rng.uniform(0.0, 0.8, n)       # patch layer 0 only
    else:
        # on patch corners and edges, moving across them
        c = rng.integers(0, 4, n) * 0.8
        x = np.mod(c + rng.choice([-1e-9, 0.0, 1e-9], n), 3.2)
        y = np.mod(rng.integers(0, 2, n) * 0.8 + rng.choice([-1e-9, 0.0], n), 1.6)
        z = np.mod(rng.integers(0, 2, n) * 0.8 + rng.choice([0.0, 1e-9], n), 1.6)
    u = rng.normal(0, 0.5, (3, n))
    parts = {"x": x, "y": y, "z": z, "ux": u[0], "uy": u[1], "uz": u[2], "w": rng.uniform(0.5, 1.5, n)}
    fields = W.random_fields(W.field_shape3(run), seed=8, amp=0.05)
    o, g = pair3(run, parts, fields)
    for _ in range(3):
        o.step(1)
        g.pic_step(1)
    _assert(field_errs(o, g), 1e-11)
    _assert(particle_errs(o, g), 1e-11)


def test_moving_window_upper_half_plasma_fp64():
    run = W.lwfa_3d(n=(64, 32, 16), d=(0.125, 0.5, 0.5), patch=(16, 8, 8), ppc=(2, 1, 1),
                    n0=0.01, ramp=3.0, a0=1.0, waist=4.0, tau=3.0, t_mw=0.5)
    run["laser"]["t_peak"] = 4.0
    o, g = pair3(run, fill=True)
    a, b = g.pic_get_particles(), o.particles()
    assert a["x"].size == b["x"].size == 64 * 16 * 16 * 2
    bm = match_particles3(a, b)
    for k in KEYS:
        assert rel(a[k], bm[k]) <= 1e-12, k
    assert rel(g.pic_get_field("rho_bg"), o.field("rho_bg")) <= 1e-12
    nsteps = 2 * math.ceil(16 * 0.125 / run["dt"]) + 6
    for _ in range(nsteps):
        o.step(1)
        g.pic_step(1)
    do, dg = o.diag(), g.pic_diag()
    assert do["shifts"] >= 2 and dg["shifts"] == do["shifts"] and dg["np"] == do["np"]
    _assert(field_errs(o, g, EB), 1e-12)
    _assert(particle_errs(o, g), 1e-12)
    assert dg["gauss"] <= 1e-9 + 1e-9 * do["gauss"]


def test_window_step_decoupled_from_patch_size():
    """GPU patches of 8^3 with a 16-cell window step equal the oracle run
    with 16^3 patches (whose window steps one 16-cell patch column)."""
    run = W.lwfa_3d(n=(64, 32, 16), d=(0.125, 0.5, 0.5), patch=(16, 16, 16), ppc=(2, 1, 1),
                    n0=0.01, ramp=3.0, a0=1.0, waist=4.0, tau=3.0, t_mw=0.5)
    run["laser"]["t_peak"] = 4.0
    o = Oracle3(run, track_continuity=True)
    o.fill_plasma()
    g = pic.Pic(pic.config_from_run(run, "fp64", patch=(8, 8, 8)))
    assert g.cfg.window_cells == 16
    g.pic_load_plasma()
    nsteps = 2 * math.ceil(16 * 0.125 / run["dt"]) + 6
    for _ in range(nsteps):
        o.step(1)
        g.pic_step(1)
    do, dg = o.diag(), g.pic_diag()
    assert do["shifts"] >= 2 and dg["shifts"] == do["shifts"] and dg["np"] == do["np"]
    _assert(field_errs(o, g, EB), 1e-12)
    _assert(particle_errs(o, g), 1e-12)


@pytest.mark.parametrize("patch,tma,cfloat", [((16, 8, 8), True, False), ((8, 8, 8), True, False),
                                              ((16, 8, 8), False, False), ((16, 16, 16), False, False),
                                              ((8, 16, 8), True, False), ((8, 8, 8), True, True)])
def test_fp32_single_step_bounds(patch, tma, cfloat):
    """FP32 step from an FP64 state, for the compile-time patch shapes
    (16x8x8, 8x8x8 staged or gathered from HBM, 16^3 gathered) and a
    runtime-shaped one (8x16x8), the current tile in fixed point; and 8^3
    with float shared atomics."""
    run = _open3()
    parts = W.small_random_particles3(run, 40000, seed=9, uth=0.6)
    fields = W.random_fields(W.field_shape3(run), seed=10, amp=0.1)
    o = Oracle3(run)
    o.load(parts)
    g = pic.Pic(pic.config_from_run(run, "fp32", patch=patch, tma=tma, current_float=cfloat))
    g.pic_load_particles(parts)
    for k, v in fields.items():
        o.set_field(k, v)
        g.pic_set_field(k, v)
    o.step(1)
    g.pic_step(1)
    errs = field_errs(o, g)
    print("3D fp32", errs)
    _assert({k: v for k, v in errs.items() if k.startswith("J")}, 2e-5)
    _assert({k: v for k, v in errs.items() if not k.startswith("J")}, 2e-6)


def test_thermal_energy_history_fp64():
    run = W.periodic_run3((32, 16, 16), (0.1, 0.1, 0.1), (8, 8, 8))
    parts = W.small_random_particles3(run, 32 * 16 * 16 * 2, seed=11, uth=0.05)
    parts["w"][:] = 0.5
    o, g = pair3(run, parts, background=("neutralising", 0.0))
    worst = 0.0
    for _ in range(10):
        o.step(5)
        g.pic_step(5)
        do, dg = o.diag(), g.pic_diag()
        for k in ("U_E", "U_B", "U_K"):
            worst = max(worst, abs(dg[k] - do[k]) / max(abs(do[k]), 1e-300))
    print("3D energy history worst rel", worst)
    assert worst <= 1e-3


def test_error_paths_3d():
    run = W.periodic_run3((16, 16, 16), (0.1, 0.1, 0.1), (8, 8, 8))
    g = pic.Pic(pic.config_from_run(run, "fp64"))
    bad = W.small_random_particles3(run, 10, seed=1)
    bad["z"][3] = 1e3
    with pytest.raises(pic.PicError) as e:
        g.pic_load_particles(bad)
    assert e.value.status == pic.PIC_EINVAL
    two_d = W.small_random_particles3(run, 10, seed=2)
    rc = pic.lib().pic_load_particles(g.h, *[two_d[k].ctypes.data for k in pic.KEYS2], 10, pic.PIC_HOST)
    assert rc == pic.PIC_EINVAL
    with pytest.raises(pic.PicError) as e:
        g.pic_restore(b"PICSNAP2" + bytes(256))  # a 2D snapshot's header
    assert e.value.status == pic.PIC_EINVAL
    nan = W.small_random_particles3(run, 100, seed=3)
    good = pic.Pic(pic.config_from_run(run, "fp64"))
    good.pic_load_particles(nan)
    blob = good.pic_snapshot()
    nan["uy"][5] = np.nan
    g.pic_load_particles(nan)
    with pytest.raises(pic.PicError) as e:
        g.pic_step(1)
    assert e.value.status == pic.PIC_ENONFINITE
    with pytest.raises(pic.PicError) as e:
        g.pic_step(1)
    assert e.value.status == pic.PIC_ESTATE
    # a restore clears the fault: the context steps again
    g.pic_restore(blob)
    g.pic_step(2)
    assert g.pic_diag()["np"] == 100
    with pytest.raises(pic.PicError) as e:
        g.pic_restore(blob[:-8])
    assert e.value.status == pic.PIC_EINVAL


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_staging_wait_that_runs_out_is_reported_3d(prec):
    """3D twin of the 2D test: 8^3 patches stage their tiles by TMA; with a
    poll bound that runs out at once every block drains its copy and
    returns, the step reports PIC_ETIMEOUT and the next call PIC_ESTATE."""
    run = W.periodic_run3((16, 16, 16), (0.1, 0.1, 0.1), (8, 8, 8))
    g = pic.Pic(pic.config_from_run(run, prec, staging_wait_polls=-1, auto_grow=False))
    g.pic_load_particles(W.small_random_particles3(run, 2000, seed=4))
    with pytest.raises(pic.PicError) as e:
        g.pic_step(1)
    assert e.value.status == pic.PIC_ETIMEOUT
    with pytest.raises(pic.PicError) as e:
        g.pic_step(1)
    assert e.value.status == pic.PIC_ESTATE
    g.close()


def test_full_size_config3_invariants_fp32():
    """1024 x 256 x 256 cells, 16^3 patches, upper-half plasma (0.005 n_c,
    2 ppc: 67 108 864 electrons) filled on the device, laser a0 = 3,
    moving window: a few steps in the benchmark's launch configuration;
    particle count, charge and the discrete continuity residual checked."""
    run = W.lwfa_3d()
    # the benchmark stores the 16^3 patches' particles in 8^3 sub-patches
    g = pic.Pic(pic.config_from_run(run, "fp32", capacity_factor=2.0, patch=(8, 8, 8)))
    g.pic_load_plasma()
    d0 = g.pic_diag()
    assert d0["np"] == 1024 * 128 * 256 * 2
    g.pic_step(3)
    d = g.pic_diag()
    assert d["np"] == d0["np"]
    assert abs(d["charge"] - d0["charge"]) <= 1e-9 * abs(d0["charge"])
    # FP32 positions: continuity to FP32 rounding of the per-step charge change
    rho_scale = 0.005
    assert d["continuity"] < 1e-3 * rho_scale / run["dt"], d["continuity"]
    assert d["U_E"] > 0  # the laser has entered


def test_plasma_autotuner_3d_choice_is_valid_cached_and_exact():
    """pic_autotune_plasma on a 3D LWFA-shaped run with the moving window:
    the choice is one of the candidate shapes that divide the grid and the
    16-cell window step, a second call returns it from the cache, and the
    tuned context evolves like the given one (FP64: rounding order only)."""
    run = W.lwfa_3d(n=(64, 32, 32), d=(0.125, 0.5, 0.5), patch=(16, 8, 8), a0=1.0, waist=5.0,
                    tau=3.0, t_mw=1.0)
    cfg = pic.config_from_run(run, "fp64")
    pic.lib().pic_autotune_clear_cache()
    tuned, info = pic.pic_autotune_plasma(cfg, steps=2)
    assert info["candidates"] > 1
    px, py, pz = info["patch"]
    assert px in (8, 16) and py in (8, 16) and pz in (8, 16, cfg.patch[2])
    assert 16 % px == 0 and tuned.window_cells in (0, 16)
    assert info["task_chunk"] in (1024, 2048, 4096)
    assert info["ms_per_step"] <= info["ms_given"]
    again, info2 = pic.pic_autotune_plasma(cfg, steps=2)
    assert info2["candidates"] == 0 and info2["patch"] == info["patch"]
    a, b = pic.Pic(cfg), pic.Pic(tuned)
    for g in (a, b):
        g.pic_load_plasma()
        g.pic_step(60)
    da, db = a.pic_diag(), b.pic_diag()
    assert da["np"] == db["np"] and da["shifts"] == db["shifts"] >= 2
    for k in EB:
        assert rel(b.pic_get_field(k), a.pic_get_field(k)) <= 1e-9, k


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_snapshot_round_trip_is_bytewise_3d(prec):
    """A snapshot restored into a fresh context (particle storage allocated
    from the snapshot's capacity) and snapshotted again gives the same
    bytes: fields, background charge, both particle sets, counts, scalars."""
    run = _open3()
    parts = W.small_random_particles3(run, 20000, seed=21, uth=0.4)
    g = pic.Pic(pic.config_from_run(run, prec))
    g.pic_load_particles(parts)
    g.pic_step(3)
    blob = g.pic_snapshot()
    g2 = pic.Pic(pic.config_from_run(run, prec))
    g2.pic_restore(blob)
    assert g2.pic_snapshot() == blob
    d, d2 = g.pic_diag(), g2.pic_diag()
    for k in ("step", "np", "capacity", "U_E", "U_B", "U_K", "charge"):
        assert d2[k] == d[k], k


def test_snapshot_restore_resume_3d_moving_window():
    """A 3D snapshot taken after window shifts and restored into a fresh
    context resumes the run: the resumed state equals the oracle's
    uninterrupted run; restoring into the original context, which has
    stepped past the snapshot, rewinds it to the same result."""
    run = W.lwfa_3d(n=(64, 32, 16), d=(0.125, 0.5, 0.5), patch=(16, 8, 8), ppc=(2, 1, 1),
                    n0=0.01, ramp=3.0, a0=1.0, waist=4.0, tau=3.0, t_mw=0.5)
    run["laser"]["t_peak"] = 4.0
    o, g = pair3(run, fill=True)
    n1 = math.ceil(16 * 0.125 / run["dt"]) + 5
    n2 = math.ceil(16 * 0.125 / run["dt"]) + 3
    for _ in range(n1):
        o.step(1)
        g.pic_step(1)
    assert g.pic_diag()["shifts"] >= 1
    blob = g.pic_snapshot()
    g.pic_step(4)
    g2 = pic.Pic(pic.config_from_run(run, "fp64"))
    g2.pic_restore(blob)
    assert g2.pic_diag()["step"] == n1
    for _ in range(n2):
        o.step(1)
        g2.pic_step(1)
    do, d2 = o.diag(), g2.pic_diag()
    assert d2["shifts"] == do["shifts"] >= 2 and d2["np"] == do["np"]
    _assert(field_errs(o, g2, EB), 1e-12)
    _assert(particle_errs(o, g2), 1e-12)
    g.pic_restore(blob)
    g.pic_step(n2)
    _assert(field_errs(o, g, EB), 1e-12)
    _assert(particle_errs(o, g), 1e-12)


def test_auto_grow_replays_overflowing_steps_3d():
    """Converging flows pile particles into the central patches; with a
    patch capacity sized exactly to the initial load, pic_step grows the
    capacity (and the 26 direction buckets with it) and replays from the
    state at entry: results equal a run that never overflowed."""
    run = W.periodic_run3((32, 32, 32), (0.1, 0.1, 0.1), (8, 8, 8))
    rng = np.random.default_rng(7)
    n = 40000
    pos = {k: rng.uniform(0, 3.2, n) for k in ("x", "y", "z")}
    parts = {**pos, "ux": -2.0 * np.sign(pos["x"] - 1.6), "uy": -2.0 * np.sign(pos["y"] - 1.6),
             "uz": -2.0 * np.sign(pos["z"] - 1.6), "w": np.full(n, 0.01)}
    small = pic.Pic(pic.config_from_run(run, "fp64", capacity_factor=1.0, capacity_min=32))
    big = pic.Pic(pic.config_from_run(run, "fp64", capacity_factor=8.0))
    for g in (small, big):
        g.pic_load_particles(parts)
    cap0 = small.pic_diag()["capacity"]
    small.pic_step(20)
    big.pic_step(20)
    d = small.pic_diag()
    assert d["grows"] >= 1 and d["capacity"] > cap0
    assert d["max_patch_count"] > cap0
    for k in ("Ex", "Ey", "Ez", "Jx", "Jy", "Jz", "Bx"):
        a, b = small.pic_get_field(k), big.pic_get_field(k)
        assert np.max(np.abs(a - b)) <= 1e-12 * np.max(np.abs(b)), k
    assert small.pic_diag()["np"] == big.pic_diag()["np"] == n
    _assert(particle_errs_between(small, big), 1e-12)


def particle_errs_between(g, h):
    a, b = g.pic_get_particles(), h.pic_get_particles()
    assert a["x"].size == b["x"].size
    b = match_particles3(a, b)
    return {k: rel(a[k], b[k]) for k in KEYS}
