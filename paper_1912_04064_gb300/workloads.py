"""Seeded synthetic inputs shared by the CUDA path's tests/benchmark and the
oracle.

This module only describes runs and draws their initial particles; it holds
none of the method's arithmetic (no interpolation, push, deposition or field
update).  A run is a plain dict:

    n, d          cells and cell sizes per axis (x, y)
    dt            time step
    patch         patch size in cells (px, py)
    field_bc      per axis: "periodic" | "sm" (Silver-Mueller, open)
    part_bc       per axis (lo, hi): "periodic" | "reflect" | "remove"
    q, m          charge and mass of the mobile species (electrons: -1, 1)
    laser         None or {a0, waist, tau, t_peak, y_center}
    moving_window None or {t0}
    injection     None or {n0, x0, ramp, ppc: (ppcx, ppcy)} (plasma entering
                  with the moving window)

Particles are dicts of float64 arrays x, y (global positions in c/w),
ux, uy, uz (u = p / mc) and w (weight = local density / particles per cell).
"""
import math

import numpy as np


def cfl_dt(d, frac=0.95):
    """frac x the 2D Yee stability limit 1 / sqrt(sum 1/d^2) (c = 1)."""
    return frac / math.sqrt(sum(1.0 / x ** 2 for x in d))


def periodic_run(n, d, patch, dt=None):
    return {
        "n": tuple(int(v) for v in n), "d": tuple(float(v) for v in d),
        "dt": cfl_dt(d) if dt is None else float(dt), "patch": tuple(patch),
        "field_bc": ("periodic", "periodic"),
        "part_bc": (("periodic", "periodic"), ("periodic", "periodic")),
        "q": -1.0, "m": 1.0, "laser": None, "moving_window": None, "injection": None,
    }


def thermal_particles(run, ppc=4, uth=0.05, n0=1.0, seed=1):
    """Uniform thermal plasma: ppc particles per cell at uniform random
    positions inside each cell, Maxwellian momenta N(0, uth^2) per component,
    weight n0 / ppc."""
    rng = np.random.default_rng(seed)
    nx, ny = run["n"]
    dx, dy = run["d"]
    cx, cy = np.meshgrid(np.arange(nx), np.arange(ny), indexing="xy")
    cx = np.repeat(cx.ravel(), ppc)
    cy = np.repeat(cy.ravel(), ppc)
    n = cx.size
    x = (cx + rng.random(n)) * dx
    y = (cy + rng.random(n)) * dy
    # keep positions strictly inside the box after rounding
    x = np.minimum(x, np.nextafter(nx * dx, 0.0))
    y = np.minimum(y, np.nextafter(ny * dy, 0.0))
    u = rng.normal(0.0, uth, size=(3, n))
    w = np.full(n, n0 / ppc)
    return {"x": x, "y": y, "ux": u[0], "uy": u[1], "uz": u[2], "w": w}


def thermal_2d(n=(128, 128), d=(0.1, 0.1), patch=(16, 16), ppc=4, uth=0.05, seed=1):
    """Uniform thermal plasma, periodic fields and particles, electrons on a
    uniform neutralising background (the 128x128, 4 ppc, u_th = 0.05 case)."""
    run = periodic_run(n, d, patch)
    return run, thermal_particles(run, ppc=ppc, uth=uth, seed=seed)


def density_profile(x, n0, x0, ramp):
    """Plasma density at x: linear up-ramp of length `ramp` from x0, then n0."""
    x = np.asarray(x, dtype=np.float64)
    if ramp <= 0.0:
        return np.where(x >= x0, n0, 0.0)
    return n0 * np.clip((x - x0) / ramp, 0.0, 1.0)


def regular_particles(nx, ny, dx, dy, ppc, profile, x_offset=0.0, cells_x=None):
    """Particles placed regularly (ppcx x ppcy per cell) at rest; weight is
    the profile at the particle's x divided by the particles per cell."""
    ppcx, ppcy = ppc
    i0, i1 = (0, nx) if cells_x is None else cells_x
    ii = np.arange(i0, i1)
    jj = np.arange(ny)
    a = (np.arange(ppcx) + 0.5) / ppcx
    b = (np.arange(ppcy) + 0.5) / ppcy
    # order: cell row j, cell i, sub-row b, sub-column a
    J, I, B, A = np.meshgrid(jj, ii, b, a, indexing="ij")
    x = ((I + A) * dx).ravel()
    y = ((J + B) * dy).ravel()
    w = profile(x + x_offset) / (ppcx * ppcy)
    z = np.zeros_like(x)
    return {"x": x, "y": y, "ux": z.copy(), "uy": z.copy(), "uz": z.copy(), "w": w}


def lwfa_2d(n=(2048, 512), d=(0.125, 0.5), patch=(32, 32), ppc=(2, 2), n0=0.01,
            ramp=200.0, a0=2.0, waist=20.0, tau=30.0, t_mw=None, frac=0.95):
    """2D3V LWFA-shaped run: Gaussian y-polarised laser entering at x_min,
    cold electrons on immobile ions with a linear density ramp, moving
    window at c, Silver-Mueller fields on every face, particles removed
    through the x faces and reflected at the y faces."""
    run = lwfa_run(n, d, patch, ppc, n0, ramp, a0, waist, tau, t_mw, frac)
    nx, ny = n
    dx, dy = d
    parts = regular_particles(nx, ny, dx, dy, ppc,
                              lambda x: density_profile(x, n0, 0.0, ramp))
    return run, parts


def lwfa_run(n=(2048, 512), d=(0.125, 0.5), patch=(32, 32), ppc=(2, 2), n0=0.01,
             ramp=200.0, a0=2.0, waist=20.0, tau=30.0, t_mw=None, frac=0.95):
    """The run dictionary of lwfa_2d without its particles (the plasma is
    the injection profile; a context can fill it on the device)."""
    nx, ny = n
    dx, dy = d
    Lx, Ly = nx * dx, ny * dy
    run = {
        "n": (nx, ny), "d": (dx, dy), "dt": cfl_dt(d, frac), "patch": tuple(patch),
        "field_bc": ("sm", "sm"),
        "part_bc": (("remove", "remove"), ("reflect", "reflect")),
        "q": -1.0, "m": 1.0,
        "laser": {"a0": a0, "waist": waist, "tau": tau, "t_peak": 2.0 * tau,
                  "y_center": Ly / 2.0},
        "moving_window": {"t0": Lx / 2.0 if t_mw is None else t_mw},
        "injection": {"n0": n0, "x0": 0.0, "ramp": ramp, "ppc": tuple(ppc)},
    }
    return run


def served_requests(count, seed):
    """Requests of the served ensemble: grid uniform over {256x256,
    512x256, 1024x512, 2048x512} (dx = 0.125, dy = 0.5, 32x32 patches),
    1-8 particles per cell, density 0.001-0.02 n_c uniform or ramped
    (20-200 c/w0), a Gaussian laser (a0 0.5-4, with the moving window) in
    half of them, 200-2000 steps.  Returns [(run, steps, particles)]."""
    rng = np.random.default_rng(seed)
    grids = [(256, 256), (512, 256), (1024, 512), (2048, 512)]
    out = []
    for _ in range(count):
        nx, ny = grids[int(rng.integers(len(grids)))]
        ppc_total = int(rng.integers(1, 9))
        ppc = (2, ppc_total // 2) if ppc_total % 2 == 0 and ppc_total > 2 else (ppc_total, 1)
        n0 = float(rng.uniform(0.001, 0.02))
        ramp = 0.0 if rng.random() < 0.5 else float(rng.uniform(20.0, 200.0))
        laser = rng.random() < 0.5
        a0 = float(rng.uniform(0.5, 4.0))
        steps = int(rng.integers(200, 2001))
        run = lwfa_run(n=(nx, ny), ppc=ppc, n0=n0, ramp=ramp, a0=a0)
        if not laser:
            run["laser"] = None
            run["moving_window"] = None
        out.append((run, steps, nx * ny * ppc_total))
    return out


def random_fields(shape, seed, amp=0.05, names=("Ex", "Ey", "Ez", "Bx", "By", "Bz",
                                                  "Bmx", "Bmy", "Bmz")):
    """Smooth-ish random fields for identical-state single-step tests."""
    rng = np.random.default_rng(seed)
    return {k: amp * rng.standard_normal(shape) for k in names}


def small_random_particles(run, n, seed, uth=0.3):
    """n particles uniformly over the box, momenta N(0, uth^2) (test cases)."""
    rng = np.random.default_rng(seed)
    nx, ny = run["n"]
    dx, dy = run["d"]
    x = np.minimum(rng.random(n) * nx * dx, np.nextafter(nx * dx, 0))
    y = np.minimum(rng.random(n) * ny * dy, np.nextafter(ny * dy, 0))
    u = rng.normal(0.0, uth, size=(3, n))
    w = 0.5 + rng.random(n)
    return {"x": x, "y": y, "ux": u[0], "uy": u[1], "uz": u[2], "w": w}


def field_shape(run):
    """Shape (ny_e, nx_e) of the field arrays exchanged with either side:
    per axis n (periodic, indices [0, n)) or n + 2 (open, indices [-1, n])."""
    nx, ny = run["n"]
    fx, fy = run["field_bc"]
    return (ny if fy == "periodic" else ny + 2, nx if fx == "periodic" else nx + 2)


# ------------------------------------------------------------------ 3D3V --

def periodic_run3(n, d, patch, dt=None, frac=0.95):
    """Fully periodic 3D3V run (fields and particles), electrons."""
    return {"n": tuple(n), "d": tuple(d), "dt": dt if dt is not None else cfl_dt(d, frac),
            "patch": tuple(patch), "field_bc": ("periodic",) * 3,
            "part_bc": (("periodic", "periodic"),) * 3, "q": -1.0, "m": 1.0}


def lwfa_3d(n=(1024, 256, 256), d=(0.125, 0.5, 0.5), patch=(16, 16, 16), ppc=(2, 1, 1),
            n0=0.005, ramp=0.0, a0=3.0, waist=15.0, tau=30.0, t_mw=None, frac=0.95,
            upper_half=True):
    """3D3V LWFA-shaped run: y-polarised Gaussian laser through x_min,
    cold electrons on immobile ions filling the upper half of the transverse
    box (y >= Ly/2, all x and z) when upper_half, moving window at c,
    Silver-Mueller on every face, particles removed through the x faces and
    reflected at the y and z faces.  The plasma is the injection profile
    (a context fills it on the device)."""
    nx, ny, nz = n
    dx, dy, dz = d
    Lx, Ly, Lz = nx * dx, ny * dy, nz * dz
    return {
        "n": tuple(n), "d": tuple(d), "dt": cfl_dt(d, frac), "patch": tuple(patch),
        "field_bc": ("sm", "sm", "sm"),
        "part_bc": (("remove", "remove"), ("reflect", "reflect"), ("reflect", "reflect")),
        "q": -1.0, "m": 1.0,
        "laser": {"a0": a0, "waist": waist, "tau": tau, "t_peak": 2.0 * tau,
                  "y_center": Ly / 2.0, "z_center": Lz / 2.0},
        "moving_window": {"t0": Lx / 2.0 if t_mw is None else t_mw},
        "injection": {"n0": n0, "x0": 0.0, "ramp": ramp, "ppc": tuple(ppc),
                      "ymin": Ly / 2.0 if upper_half else 0.0},
    }


def field_shape3(run):
    """(nz_e, ny_e, nx_e) of 3D field arrays: per axis n (periodic) or
    n + 2 (open)."""
    return tuple(run["n"][a] + (0 if run["field_bc"][a] == "periodic" else 2) for a in (2, 1, 0))


def small_random_particles3(run, n, seed, uth=0.3):
    """n particles uniformly over the 3D box, momenta N(0, uth^2)."""
    rng = np.random.default_rng(seed)
    out = {}
    for a, k in enumerate(("x", "y", "z")):
        L = run["n"][a] * run["d"][a]
        out[k] = np.minimum(rng.random(n) * L, np.nextafter(L, 0))
    u = rng.normal(0.0, uth, size=(3, n))
    out["ux"], out["uy"], out["uz"] = u[0], u[1], u[2]
    out["w"] = 0.5 + rng.random(n)
    return out
