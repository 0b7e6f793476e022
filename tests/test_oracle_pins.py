"""Pins of the FP64 CPU oracle against what the mathematics fixes.

Each test ties one part of the oracle to something other than itself: a
closed form (Boris gyration, discrete Yee eigenmodes), an invariant (discrete
continuity, Gauss law, div B), an exact-rational brute force on tiny inputs
(Esirkepov as the average of the two single-axis paths, interpolation with
the piecewise B-spline), or an independent physical bound (Silver-Mueller
reflection, laser amplitude).  None of these needs a GPU.
"""
import math
from fractions import Fraction as Fr

import numpy as np
import pytest

from oracle.oracle import Oracle, boris, poisson_periodic, shape2
from paper_1912_04064_gb300 import workloads as W


# ---------------------------------------------------------------- shape ----

def bspline2(t: Fr) -> Fr:
    """Quadratic B-spline, piecewise form (textbook definition)."""
    a = abs(t)
    if a <= Fr(1, 2):
        return Fr(3, 4) - a * a
    if a <= Fr(3, 2):
        return (a - Fr(3, 2)) ** 2 / 2
    return Fr(0)


def test_shape_equals_bspline_and_moments():
    rng = np.random.default_rng(0)
    for xi in list(rng.uniform(-3, 7, 200)) + [0.0, 0.5, -0.5, 1.5, 2.25]:
        i0, S = shape2(float(xi))
        X = Fr(float(xi))
        for k in range(3):
            exact = bspline2(Fr(i0 - 1 + k) - X)
            assert abs(S[k] - float(exact)) <= 2e-16
        # partition of unity, zero first moment, second moment 1/4
        d = [i0 - 1 + k - xi for k in range(3)]
        assert abs(S.sum() - 1.0) < 1e-15
        assert abs(sum(S[k] * d[k] for k in range(3))) < 1e-15
        assert abs(sum(S[k] * d[k] ** 2 for k in range(3)) - 0.25) < 1e-15
        # no weight outside the three nodes
        assert bspline2(Fr(i0 - 2) - X) == 0 and bspline2(Fr(i0 + 2) - X) == 0


# ---------------------------------------------------------------- Boris ----

def _uniform_run(n=64, d=0.1, patch=16):
    return W.periodic_run((n, n), (d, d), (patch, patch))


def test_boris_gyration_closed_form():
    """Uniform B_z, E = 0: |u| is conserved to round-off, u rotates by exactly
    theta = 2 atan(|q| dt B / (2 m gamma)) per step in the sense fixed by
    du/dt = q v x B, and the positions lie on a circle of radius
    dt |u_perp| / (2 gamma sin(theta / 2))."""
    run = _uniform_run()
    o = Oracle(run)
    B0 = 0.8
    shp = o.shape
    o.set_field("Bz", np.full(shp, B0))
    o.set_field("Bmz", np.full(shp, B0))
    u0 = np.array([0.6, 0.0, 0.3])
    o.load({"x": [3.2], "y": [3.2], "ux": [u0[0]], "uy": [u0[1]], "uz": [u0[2]], "w": [0.0]})
    g = math.sqrt(1 + u0 @ u0)
    dt = run["dt"]
    theta = 2 * math.atan(dt * B0 / (2 * g))
    R = dt * math.hypot(u0[0], u0[1]) / (2 * g * math.sin(theta / 2))
    xs, us = [], []
    for n in range(2000):
        o.step(1)
        p = o.particles()
        xs.append((p["x"][0], p["y"][0]))
        us.append((p["ux"][0], p["uy"][0], p["uz"][0]))
    xs, us = np.array(xs), np.array(us)
    norm = np.sqrt((us ** 2).sum(1))
    assert np.max(np.abs(norm - np.linalg.norm(u0))) < 1e-13
    assert np.max(np.abs(us[:, 2] - u0[2])) < 1e-15
    ang = np.arctan2(us[1:, 1] * us[:-1, 0] - us[1:, 0] * us[:-1, 1],
                     us[1:, 0] * us[:-1, 0] + us[1:, 1] * us[:-1, 1])
    # q = -1, B along +z: u rotates counter-clockwise
    assert np.max(np.abs(ang - theta)) < 1e-12
    # circle: fit centre from the mean of the points (a whole number of turns
    # is not needed: use the exact geometric centre from three points)
    (x1, y1), (x2, y2), (x3, y3) = xs[0], xs[1], xs[2]
    D = 2 * (x1 * (y2 - y3) + x2 * (y3 - y1) + x3 * (y1 - y2))
    cx = ((x1 ** 2 + y1 ** 2) * (y2 - y3) + (x2 ** 2 + y2 ** 2) * (y3 - y1) + (x3 ** 2 + y3 ** 2) * (y1 - y2)) / D
    cy = ((x1 ** 2 + y1 ** 2) * (x3 - x2) + (x2 ** 2 + y2 ** 2) * (x1 - x3) + (x3 ** 2 + y3 ** 2) * (x2 - x1)) / D
    r = np.hypot(xs[:, 0] - cx, xs[:, 1] - cy)
    assert np.max(np.abs(r - R)) / R < 1e-10


def test_boris_pure_electric_field():
    """B = 0: the push is an exact uniform acceleration u += q dt E / m."""
    rng = np.random.default_rng(3)
    for _ in range(50):
        E = rng.normal(size=3)
        u = rng.normal(size=3)
        q, m, dt = -1.0, 1.0, 0.07
        out = boris(q, m, dt, E, np.zeros(3), u)
        assert np.allclose(out, u + q * dt * E / m, rtol=0, atol=1e-15)


def test_boris_push_through_grid_uniform_E():
    run = _uniform_run()
    o = Oracle(run)
    E0 = (0.01, -0.02, 0.03)
    for k, v in zip(("Ex", "Ey", "Ez"), E0):
        o.set_field(k, np.full(o.shape, v))
    o.load({"x": [1.0], "y": [2.0], "ux": [0.1], "uy": [0.0], "uz": [0.0], "w": [0.0]})
    o.step(1)
    p = o.particles()
    dt = run["dt"]
    assert abs(p["ux"][0] - (0.1 - dt * E0[0])) < 1e-15
    assert abs(p["uy"][0] - (0.0 - dt * E0[1])) < 1e-15
    assert abs(p["uz"][0] - (0.0 - dt * E0[2])) < 1e-15


# ------------------------------------------------------------------ Yee ----

def _mode_fields(run, mx, my, t0):
    nx, ny = run["n"]
    dx, dy = run["d"]
    dt = run["dt"]
    kx, ky = 2 * math.pi * mx / (nx * dx), 2 * math.pi * my / (ny * dy)
    kxh, kyh = 2 / dx * math.sin(kx * dx / 2), 2 / dy * math.sin(ky * dy / 2)
    omega = 2 / dt * math.asin(dt / 2 * math.hypot(kxh, kyh))
    Om = 2 / dt * math.sin(omega * dt / 2)
    i = np.arange(nx)[None, :]
    j = np.arange(ny)[:, None]

    def ph(sx, sy, t):
        return kx * (i + 0.5 * sx) * dx + ky * (j + 0.5 * sy) * dy - omega * t

    tE, tB = t0, t0 + 0.5 * dt
    tm = {
        "Ez": np.cos(ph(0, 0, tE)),
        "Bx": (kyh / Om) * np.cos(ph(0, 1, tB)),
        "By": -(kxh / Om) * np.cos(ph(1, 0, tB)),
    }
    te = {
        "Bz": np.cos(ph(1, 1, tB)),
        "Ex": -(kyh / Om) * np.cos(ph(1, 0, tE)),
        "Ey": (kxh / Om) * np.cos(ph(0, 1, tE)),
    }
    return tm, te


@pytest.mark.parametrize("mx,my", [(1, 0), (0, 1), (2, 3), (3, 3), (5, 1)])
def test_yee_discrete_dispersion(mx, my):
    """A Fourier mode with omega from sin^2(w dt/2)/dt^2 = sum sin^2(k d/2)/d^2
    is an exact eigenvector of the Yee update: after N steps the fields equal
    the analytic discrete mode to round-off (both polarisations)."""
    run = W.periodic_run((32, 24), (0.1, 0.15), (8, 8))
    tm, te = _mode_fields(run, mx, my, 0.0)
    o = Oracle(run)
    for k, v in {**tm, **te}.items():
        o.set_field(k, v)
    N = 300
    o.step(N)
    tm2, te2 = _mode_fields(run, mx, my, N * run["dt"])
    for k, v in {**tm2, **te2}.items():
        err = np.max(np.abs(o.field(k) - v))
        assert err < 1e-11, (k, err)
    # Bm^N = (B^{N-1/2} + B^{N+1/2}) / 2 = cos(w dt / 2) x the mode at t_N
    tmb, teb = _mode_fields(run, mx, my, N * run["dt"] - 0.5 * run["dt"])
    nx, ny = run["n"]
    dx, dy = run["d"]
    kx, ky = 2 * math.pi * mx / (nx * dx), 2 * math.pi * my / (ny * dy)
    kxh, kyh = 2 / dx * math.sin(kx * dx / 2), 2 / dy * math.sin(ky * dy / 2)
    omega = 2 / run["dt"] * math.asin(run["dt"] / 2 * math.hypot(kxh, kyh))
    c = math.cos(omega * run["dt"] / 2)
    for k, v in (("Bmx", tmb["Bx"]), ("Bmy", tmb["By"]), ("Bmz", teb["Bz"])):
        err = np.max(np.abs(o.field(k) - c * v))
        assert err < 1e-11, (k, err)
    # discrete div B (cell-centred) stays at round-off
    dx, dy = run["d"]
    Bx, By = o.field("Bx"), o.field("By")
    divB = (np.roll(Bx, -1, axis=1) - Bx) / dx + (By - np.roll(By, 1, axis=0)) / dy
    # Bx at (i, j+1/2), By at (i+1/2, j): divergence at (i+1/2, j+1/2)
    divB = (np.roll(Bx, -1, axis=1) - Bx) / dx + (np.roll(By, -1, axis=0) - By) / dy
    assert np.max(np.abs(divB)) < 1e-10


# ------------------------------------------------------------ Esirkepov ----

def _esirkepov_exact(x0, y0, x1, y1, dx, dy, dt, q, w, vz):
    """Exact rational current of one particle as the average of the two
    single-axis paths (x then y, y then x); Jz from the exact time integral
    (Simpson, exact for the quadratic integrand) of the linearly
    interpolated shape product.  Returns dicts {(i, j): value}."""
    def shp(xi):
        base = math.floor(xi) - 2
        return {k: bspline2(Fr(k) - xi) for k in range(base, base + 6) if bspline2(Fr(k) - xi) != 0}

    X0, Y0, X1, Y1 = (Fr(v) for v in (x0, y0, x1, y1))
    S0x, S1x = shp(X0 / Fr(dx)), shp(X1 / Fr(dx))
    S0y, S1y = shp(Y0 / Fr(dy)), shp(Y1 / Fr(dy))
    ks = range(min(S0x | S1x) - 1, max(S0x | S1x) + 2)
    ls = range(min(S0y | S1y) - 1, max(S0y | S1y) + 2)
    Q, Wt, DX, DY, DT, VZ = Fr(q), Fr(w), Fr(dx), Fr(dy), Fr(dt), Fr(vz)

    def g(d, k):
        return d.get(k, Fr(0))

    Jx, Jy, Jz = {}, {}, {}
    for l in ls:
        accA = accB = Fr(0)
        for k in ks:
            dS = g(S1x, k) - g(S0x, k)
            accA += dS * g(S0y, l)       # x first, at y0
            accB += dS * g(S1y, l)       # x second, at y1
            Jx[(k, l)] = -Q * Wt * DX / DT * (accA + accB) / 2
    for k in ks:
        accA = accB = Fr(0)
        for l in ls:
            dS = g(S1y, l) - g(S0y, l)
            accA += dS * g(S1x, k)       # y second, at x1
            accB += dS * g(S0x, k)       # y first, at x0
            Jy[(k, l)] = -Q * Wt * DY / DT * (accA + accB) / 2
    for k in ks:
        for l in ls:
            f0 = g(S0x, k) * g(S0y, l)
            f1 = g(S1x, k) * g(S1y, l)
            fh = (g(S0x, k) + g(S1x, k)) / 2 * (g(S0y, l) + g(S1y, l)) / 2
            Jz[(k, l)] = Q * Wt * VZ * (f0 + 4 * fh + f1) / 6
    return Jx, Jy, Jz


def test_esirkepov_bruteforce_4x4_three_particles():
    """4x4 periodic cells, one 4x4 patch (its current halo wraps onto
    itself), three particles at dyadic positions moving along +x,
    diagonally and across the periodic corner: the oracle's domain current
    equals the exact rational current to 1e-15 relative."""
    dx, dy, dt = 0.5, 0.25, 0.125
    run = W.periodic_run((4, 4), (dx, dy), (4, 4), dt=dt)
    parts = {"x": [0.625, 1.3125, 0.015625], "y": [0.5625, 0.3125, 0.984375],
             "ux": [0.8, 0.5, -0.9], "uy": [0.0, -0.6, 0.3], "uz": [0.1, 0.2, 0.0],
             "w": [1.0, 0.75, 1.25]}
    o = Oracle(run)
    o.load(parts)
    o.step(1)
    Jn = {k: o.field(k) for k in ("Jx", "Jy", "Jz")}
    ex = {k: np.zeros((4, 4), dtype=object) for k in ("Jx", "Jy", "Jz")}
    for k in ex:
        ex[k][:, :] = Fr(0)
    for p in range(3):
        u = np.array([parts["ux"][p], parts["uy"][p], parts["uz"][p]])
        gm = math.sqrt(1.0 + u[0] * u[0] + u[1] * u[1] + u[2] * u[2])
        x0, y0 = parts["x"][p], parts["y"][p]
        x1, y1 = x0 + dt * u[0] / gm, y0 + dt * u[1] / gm
        J3 = _esirkepov_exact(x0, y0, x1, y1, dx, dy, dt, -1.0, parts["w"][p], u[2] / gm)
        for name, J in zip(("Jx", "Jy", "Jz"), J3):
            for (i, j), v in J.items():
                ex[name][j % 4, i % 4] += v
    for name in ex:
        exf = ex[name].astype(float)
        scale = np.max(np.abs(exf))
        assert scale > 0
        assert np.max(np.abs(Jn[name] - exf)) <= 1e-15 * scale * 4, name


def test_esirkepov_zero_displacement_and_continuity():
    run = W.periodic_run((16, 16), (0.2, 0.3), (8, 8))
    o = Oracle(run)
    dx, dy, dt = run["d"][0], run["d"][1], run["dt"]
    rng = np.random.default_rng(7)
    for _ in range(300):
        x0, y0 = rng.uniform(0.5, 2.5), rng.uniform(0.5, 4.0)
        still = rng.random() < 0.2
        mvx = 0.0 if still else rng.uniform(-0.99, 0.99) * dx
        mvy = 0.0 if still else rng.uniform(-0.99, 0.99) * dy
        w, vz = rng.uniform(0.1, 2), rng.uniform(-0.9, 0.9)
        J, ix, iy = o.esirkepov(x0, y0, x0 + mvx, y0 + mvy, w, vz)
        if still:
            assert np.all(J[0] == 0) and np.all(J[1] == 0)
        # charge before/after on the same 5x5 window
        def rho(x, y):
            r = np.zeros((5, 5))
            i0, Sx = shape2(x / dx)
            j0, Sy = shape2(y / dy)
            for a in range(3):
                for b in range(3):
                    r[j0 - 1 + b - iy, i0 - 1 + a - ix] += -1.0 * w * Sx[a] * Sy[b]
            return r
        r0, r1 = rho(x0, y0), rho(x0 + mvx, y0 + mvy)
        Jx = np.pad(J[0], ((0, 0), (1, 0)))   # Jx at dual index k-1 -> column k
        Jy = np.pad(J[1], ((1, 0), (0, 0)))
        div = (Jx[:, 1:] - Jx[:, :-1]) / dx + (Jy[1:, :] - Jy[:-1, :]) / dy
        res = (r1 - r0) / dt + div
        scale = max(np.max(np.abs(r0)) / dt, 1e-300)
        assert np.max(np.abs(res)) / scale < 1e-14


def test_esirkepov_contribution_bound():
    """Every current contribution of one particle of weight w moving at
    |v| < c for one step is below (3/4) |q| w per window node and component:
    the prefix sums of S1 - S0 change with position at a rate equal to a
    linear hat (at most 1), so |P| <= |displacement in cells| < dt/d, and
    the averaged transverse shape is at most 3/4 (J_z: |v_z| < 1 and
    W_z <= (3/4)^2).  The FP32 kernels' fixed-point scale, 2^K / ((3/4)^2
    |q| w_max), keeps contributions below (4/3) 2^K on this bound; the
    extreme moves below show that (3/4)^2 alone would not bound them."""
    run = W.periodic_run((16, 16), (0.2, 0.3), (8, 8))
    o = Oracle(run)
    dx, dt = run["d"][0], run["dt"]
    rng = np.random.default_rng(17)
    worst = 0.0
    for n in range(3000):
        if n % 2:
            x0, y0 = rng.uniform(0.5, 2.5), rng.uniform(0.5, 4.0)
            v = rng.normal(size=3)
            v *= rng.uniform(0.0, 0.999999) / np.linalg.norm(v)
        else:   # fast along x, centred between nodes, on a y node
            x0 = (rng.integers(3, 10) + 0.5 + rng.uniform(-0.3, 0.3)) * dx
            y0 = rng.integers(3, 10) * run["d"][1]
            v = np.array([rng.choice([-1, 1]) * rng.uniform(0.99, 0.999999), 0.0, 0.0])
        w = rng.uniform(0.1, 2.0)
        J, _, _ = o.esirkepov(x0, y0, x0 + v[0] * dt, y0 + v[1] * dt, w, v[2])
        worst = max(worst, float(np.max(np.abs(J))) / w)
    assert worst < 0.75, worst
    assert worst > 0.5625, worst


def test_gather_bruteforce():
    """Interpolation of every component equals the exact rational sum of the
    piecewise B-spline weights at the component's own stagger."""
    run = W.periodic_run((8, 8), (0.5, 0.25), (4, 4), dt=0.1)
    o = Oracle(run)
    rng = np.random.default_rng(11)
    stag = {"Ex": (1, 0), "Ey": (0, 1), "Ez": (0, 0), "Bmx": (0, 1), "Bmy": (1, 0), "Bmz": (1, 1)}
    vals = {}
    for k in stag:
        v = np.round(rng.normal(size=o.shape) * 64) / 64  # dyadic values
        o.set_field(k, v)
        vals[k] = v
    for _ in range(20):
        x, y = float(rng.uniform(0, 4)), float(rng.uniform(0, 2))
        for k, (sx, sy) in stag.items():
            xi = Fr(x) / Fr(0.5) - Fr(sx, 2)
            eta = Fr(y) / Fr(0.25) - Fr(sy, 2)
            tot = Fr(0)
            for i in range(math.floor(xi) - 2, math.floor(xi) + 3):
                for j in range(math.floor(eta) - 2, math.floor(eta) + 3):
                    wgt = bspline2(Fr(i) - xi) * bspline2(Fr(j) - eta)
                    if wgt:
                        tot += wgt * Fr(vals[k][j % 8, i % 8])
            assert abs(o.gather(k, x, y) - float(tot)) < 1e-14, k


# ---------------------------------------------------- Gauss, continuity ----

def _poisson_state(run, parts, seed_bg=1.0):
    o = Oracle(run, track_continuity=True)
    o.load(parts)
    o.set_background("uniform", seed_bg)
    rho = o.field("rho") + seed_bg
    Ex, Ey = poisson_periodic(rho, *run["d"])
    o.set_field("Ex", Ex)
    o.set_field("Ey", Ey)
    return o, rho


def test_poisson_solution_satisfies_discrete_gauss():
    run, parts = W.thermal_2d(n=(32, 48), d=(0.1, 0.07), patch=(8, 8), seed=5)
    o, rho = _poisson_state(run, parts)
    Ex, Ey = o.field("Ex"), o.field("Ey")
    dx, dy = run["d"]
    div = (Ex - np.roll(Ex, 1, axis=1)) / dx + (Ey - np.roll(Ey, 1, axis=0)) / dy
    assert np.max(np.abs(div - (rho - rho.mean()))) < 1e-11 * np.max(np.abs(rho))
    # single mode: rho = cos(kx x) -> Ex = sin(kx (x)) type closed form
    nx, ny = 32, 48
    kx = 2 * math.pi * 3 / (nx * dx)
    khx = 2 / dx * math.sin(kx * dx / 2)
    xi = np.arange(nx) * dx
    r1 = np.tile(np.cos(kx * xi), (ny, 1))
    Ex1, Ey1 = poisson_periodic(r1, dx, dy)
    # phi = cos(kx x) / khx^2 ; Ex = -(phi(i+1) - phi(i)) / dx
    phi = np.cos(kx * xi) / khx ** 2
    exp_Ex = -(np.roll(phi, -1) - phi) / dx
    assert np.max(np.abs(Ex1 - exp_Ex[None, :])) < 1e-12
    assert np.max(np.abs(Ey1)) < 1e-12


def test_gauss_and_continuity_preserved_thermal():
    """Poisson start, 20 steps of the full loop: max |div E - rho| stays at
    round-off and the discrete continuity residual of the last step is
    round-off (Esirkepov + Yee conserve charge exactly)."""
    run, parts = W.thermal_2d(n=(32, 32), patch=(8, 8), seed=2)
    o, rho = _poisson_state(run, parts)
    scale = np.max(np.abs(rho))
    d0 = o.diag()
    assert d0["gauss"] < 1e-11 * scale
    o.step(20)
    d = o.diag()
    assert d["gauss"] < 1e-10 * scale
    assert d["continuity"] < 1e-10 * scale / run["dt"]
    assert d["np"] == len(parts["x"])


# ----------------------------------------------------- invariance of SDMD ----

def test_thread_count_invariance_bitwise():
    run, parts = W.thermal_2d(n=(64, 32), patch=(8, 8), seed=4)
    outs = []
    for nt in (1, 4):
        o = Oracle(run, nthreads=nt)
        o.load(parts)
        o.set_background("uniform", 1.0)
        o.step(4)
        outs.append({k: o.field(k) for k in ("Ex", "Ey", "Ez", "Bz", "Jx", "Jy", "Jz")})
    for k in outs[0]:
        assert np.array_equal(outs[0][k], outs[1][k]), k


def test_patch_size_invariance():
    """The patch decomposition changes only the summation order of J."""
    base = None
    for patch in ((8, 8), (16, 16), (32, 16), (4, 8)):
        run, parts = W.thermal_2d(n=(64, 32), patch=patch, seed=4)
        o = Oracle(run)
        o.load(parts)
        o.step(3)
        f = {k: o.field(k) for k in ("Ex", "Ey", "Ez", "Bx", "By", "Bz", "Jx", "Jy", "Jz")}
        if base is None:
            base = f
            continue
        for k in f:
            scale = np.max(np.abs(base[k]))
            assert np.max(np.abs(f[k] - base[k])) <= 1e-13 * scale, (patch, k)


# ------------------------------------------------ open boundaries, laser ----

def _vacuum_open_run(nx, ny, dx, dy, patch=(16, 8), periodic_y=True):
    run = W.periodic_run((nx, ny), (dx, dy), patch)
    run["field_bc"] = ("sm", "periodic" if periodic_y else "sm")
    run["part_bc"] = (("remove", "remove"), ("periodic", "periodic") if periodic_y else ("reflect", "reflect"))
    return run


@pytest.mark.parametrize("direction", [+1, -1])
def test_silver_mueller_reflection_normal_incidence(direction):
    """A plane-wave packet (k = 1, i.e. the laser wavelength, 8 cells per
    c/w) hitting an open x face: the reflected energy fraction is below
    1e-4 (amplitude reflection below 1e-2)."""
    nx, ny, dx, dy = 1024, 8, 0.125, 0.5
    run = _vacuum_open_run(nx, ny, dx, dy)
    o = Oracle(run)
    dt = run["dt"]
    sig, xc = 10.0, 64.0

    def f(x, t):
        s = x - direction * t
        return np.exp(-((s - xc) / sig) ** 2) * np.cos(s)

    sh = o.shape
    xi = (np.arange(sh[1]) - 1) * dx
    ey = np.tile(f(xi, 0.0), (sh[0], 1))
    bz = direction * np.tile(f(xi + 0.5 * dx, 0.5 * dt), (sh[0], 1))
    o.set_field("Ey", ey)
    o.set_field("Bz", bz)
    o.set_field("Bmz", direction * np.tile(f(xi + 0.5 * dx, 0.0), (sh[0], 1)))
    e0 = np.sum(ey[:, 1:-1] ** 2)
    nsteps = int(100.0 / dt)
    o.step(nsteps)
    ey2 = o.field("Ey")[:, 1:-1]
    half = slice(nx // 2, nx) if direction > 0 else slice(0, nx // 2)
    refl = np.sum(ey2[:, half] ** 2) / e0
    assert refl < 1e-4, refl


def test_laser_injection_amplitude():
    """A Gaussian laser entering through x_min reaches the expected peak
    field a0 on axis near the focal plane (within 3 %)."""
    nx, ny, dx, dy = 256, 256, 0.125, 0.5
    run = _vacuum_open_run(nx, ny, dx, dy, patch=(32, 32), periodic_y=False)
    a0, tau = 2.0, 12.0
    run["laser"] = {"a0": a0, "waist": 20.0, "tau": tau, "t_peak": 2 * tau, "y_center": ny * dy / 2}
    o = Oracle(run)
    xprobe = 10.0
    ip, jc = int(round(xprobe / dx)) + 1, ny // 2 + 1   # +1: open-axis layout starts at -1
    peak = 0.0
    t_end = 2 * tau + xprobe + 2 * tau
    for _ in range(int(t_end / run["dt"])):
        o.step(1)
        peak = max(peak, abs(o.field("Ey")[jc, ip]))
    assert abs(peak / a0 - 1.0) < 0.03, peak
    # injected laser function itself
    assert abs(o.laser(ny * dy / 2, 2 * tau + math.pi / 2) - a0 * math.exp(-2 * math.log(2) * (math.pi / 2 / tau) ** 2)) < 1e-12


# -------------------------------------------------------- moving window ----

def test_moving_window_shift_is_exact():
    """The shift of a moving-window step moves every field value exactly one
    patch column down, zeroes the new column, drops the leaving particles
    and injects the profile's plasma regularly at rest."""
    run, parts = W.lwfa_2d(n=(64, 32), d=(0.125, 0.5), patch=(16, 16), ppc=(2, 2),
                           ramp=4.0, t_mw=0.0)
    run["laser"]["tau"] = 4.0
    run["laser"]["t_peak"] = 8.0
    dt, P, dx = run["dt"], 16, 0.125
    nshift_step = math.ceil(P * dx / dt)       # first step with t >= P dx
    A, B = Oracle(run), Oracle({**run, "moving_window": {"t0": 1e9}})
    rf = W.random_fields(A.shape, seed=9, amp=0.01)
    for o in (A, B):
        o.load(parts)
        o.set_background("neutralising")
        for k, v in rf.items():
            o.set_field(k, v)
        o.step(nshift_step - 1)
    assert A.diag()["shifts"] == 0
    A.step(1)
    B.step(1)
    assert A.diag()["shifts"] == 1
    nx, G = 64, 4
    for k in ("Ex", "Ey", "Ez", "Bx", "By", "Bz", "Bmx", "Bmy", "Bmz", "rho_bg"):
        a, b = A.field(k), B.field(k)
        # layout index c <-> grid index c - 1 on the open x axis; grid
        # indices [-1, nx-P] come from [P-1, nx] (the old boundary node
        # included); [nx-P+1, nx-P+G-1] come from old ghosts (not exposed);
        # [nx-P+G, nx] have no source and are vacuum
        keep = nx - P + 2
        # the new ions' stencil reaches one node below the new column
        kk = keep - 2 if k == "rho_bg" else keep
        assert np.array_equal(a[:, 0:kk], b[:, P:P + kk]), k
        assert np.any(a[:, 0:kk] != 0.0), k
        if k != "rho_bg":
            assert np.all(a[:, nx - P + G + 1:] == 0.0), k
    # the ion background keeps the whole stencil of the kept ions at the
    # seam: after the shift the neutral plasma at rest has zero net charge
    # everywhere except where the kept electrons have moved
    assert A.diag()["gauss"] < 10 * B.diag()["gauss"] + 1e-12
    pa, pb = A.particles(), B.particles()
    keep_b = pb["x"] - P * dx >= 0.0
    new = pa["x"] >= (nx - P) * dx
    assert new.sum() == P * 32 * 4
    assert (~new).sum() == keep_b.sum()
    xphys = pa["x"][new] + P * dx
    assert np.allclose(pa["w"][new], W.density_profile(xphys, 0.01, 0.0, 4.0) / 4, rtol=0, atol=1e-18)
    assert np.all(pa["ux"][new] == 0.0)


# ------------------------------------------- particle BCs, currents, energy ----

def test_reflecting_particle_boundary():
    """A particle crossing a reflecting face is mirrored and its normal
    momentum reversed (zero fields, so the free-flight move is exact)."""
    run, _ = W.lwfa_2d(n=(32, 32), d=(0.125, 0.5), patch=(16, 16))
    run["laser"] = None
    run["moving_window"] = None
    o = Oracle(run)
    dt = run["dt"]
    u = np.array([0.1, -0.9, 0.2])
    g = math.sqrt(1 + u @ u)
    y0 = 0.02
    o.load({"x": [2.0], "y": [y0], "ux": [u[0]], "uy": [u[1]], "uz": [u[2]], "w": [0.0]})
    o.step(1)
    p = o.particles()
    assert abs(p["y"][0] - (-(y0 + dt * u[1] / g))) < 1e-15
    assert p["uy"][0] == -u[1] and p["ux"][0] == u[0]
    # removal through x_max
    o2 = Oracle(run)
    o2.load({"x": [32 * 0.125 - 1e-3], "y": [3.0], "ux": [5.0], "uy": [0.0], "uz": [0.0], "w": [0.0]})
    o2.step(1)
    assert o2.diag()["np"] == 0


@pytest.mark.parametrize("vel", [(0.3, 0.0, 0.0), (0.0, -0.4, 0.0), (0.0, 0.0, 0.5), (0.2, 0.3, -0.1)])
def test_uniform_drift_current_closed_form(vel):
    """A uniform plasma drifting with momentum u carries the current
    J = q n v everywhere; from zero fields one step gives E = -dt J exactly
    (curl B = 0), which pins the deposit normalisation of every component and
    the current term of the E update."""
    run = W.periodic_run((16, 16), (0.1, 0.2), (8, 8))
    n0, ppc = 0.7, (2, 2)
    parts = W.regular_particles(16, 16, 0.1, 0.2, ppc, lambda x: np.full_like(x, n0))
    for k, v in zip(("ux", "uy", "uz"), vel):
        parts[k][:] = v
    o = Oracle(run)
    o.load(parts)
    o.step(1)
    u = np.array(vel)
    v = u / math.sqrt(1 + u @ u)
    dt = run["dt"]
    for name, vc in zip(("Ex", "Ey", "Ez"), v):
        assert np.max(np.abs(o.field(name) - (-dt * (-1.0) * n0 * vc))) < 1e-14, name
    for name, vc in zip(("Jx", "Jy", "Jz"), v):
        assert np.max(np.abs(o.field(name) - (-1.0) * n0 * vc)) < 1e-14, name


def test_silver_mueller_discrete_condition_holds():
    """On every open face the ghost B written by the oracle makes the
    discrete Silver-Mueller condition hold exactly at the half step:
    mean over (t_n, t_n+1) of E_t  -/+  mean over the two faces of B_t at
    t_n+1/2 = 2 E_inc(t_n+1/2).  Both open axes, random interior fields, the
    laser on at x_min."""
    run = _vacuum_open_run(48, 40, 0.125, 0.25, patch=(16, 8), periodic_y=False)
    run["laser"] = {"a0": 1.0, "waist": 3.0, "tau": 5.0, "t_peak": 0.5, "y_center": 5.0}
    o = Oracle(run)
    rf = W.random_fields(o.shape, seed=21, amp=0.1)
    for k, v in rf.items():
        o.set_field(k, v)
    o.step(1)
    F1 = {k: o.field(k) for k in ("Ex", "Ey", "Ez", "Bx", "By", "Bz")}
    t_half = 1.5 * run["dt"]
    o.step(1)
    F2 = {k: o.field(k) for k in ("Ex", "Ey", "Ez")}
    nx, ny = 48, 40
    dy = 0.25
    # layout index = grid index + 1 on open axes; rows/cols 1..n-1 avoid corners
    J = slice(2, ny)          # grid rows 1 .. ny-1
    I = slice(2, nx)          # grid cols 1 .. nx-1
    ez = 0.5 * (F1["Ez"] + F2["Ez"])
    ey = 0.5 * (F1["Ey"] + F2["Ey"])
    ex = 0.5 * (F1["Ex"] + F2["Ex"])
    by, bz, bx = F1["By"], F1["Bz"], F1["Bx"]
    # x_min (node 0 <-> col 1; ghost -1 <-> col 0): Ez - By = 0, Ey + Bz = 2 Einc
    assert np.max(np.abs(ez[J, 1] - 0.5 * (by[J, 0] + by[J, 1]))) < 1e-14
    yj = (np.arange(ny + 2)[J] - 1 + 0.5) * dy
    einc = np.array([o.laser(y, t_half) for y in yj])
    assert np.max(np.abs(einc)) > 1e-3
    assert np.max(np.abs(ey[J, 1] + 0.5 * (bz[J, 0] + bz[J, 1]) - 2 * einc)) < 1e-14
    # x_max (node nx <-> col nx+1; ghost dual nx <-> col nx+1): Ez + By = 0, Ey - Bz = 0
    assert np.max(np.abs(ez[J, nx + 1] + 0.5 * (by[J, nx + 1] + by[J, nx]))) < 1e-14
    assert np.max(np.abs(ey[J, nx + 1] - 0.5 * (bz[J, nx + 1] + bz[J, nx]))) < 1e-14
    # y_min: Ez + Bx = 0, Ex - Bz = 0 ; y_max: Ez - Bx = 0, Ex + Bz = 0
    assert np.max(np.abs(ez[1, I] + 0.5 * (bx[0, I] + bx[1, I]))) < 1e-14
    assert np.max(np.abs(ex[1, I] - 0.5 * (bz[0, I] + bz[1, I]))) < 1e-14
    assert np.max(np.abs(ez[ny + 1, I] - 0.5 * (bx[ny + 1, I] + bx[ny, I]))) < 1e-14
    assert np.max(np.abs(ex[ny + 1, I] + 0.5 * (bz[ny + 1, I] + bz[ny, I]))) < 1e-14


def test_energy_conservation_thermal():
    """Periodic thermal plasma from the Poisson state: total energy
    U_E + U_B + U_K stays within 1 % over 60 steps (momentum-conserving
    shape-2 PIC heats slowly at dx = 2 Debye lengths); a wrong sign in the
    field/particle coupling breaks this at once."""
    run, parts = W.thermal_2d(n=(32, 32), patch=(8, 8), seed=3)
    o, rho = _poisson_state(run, parts)
    d0 = o.diag()
    tot0 = d0["U_E"] + d0["U_B"] + d0["U_K"]
    for _ in range(6):
        o.step(10)
        d = o.diag()
        tot = d["U_E"] + d["U_B"] + d["U_K"]
        assert abs(tot / tot0 - 1) < 1e-2


def test_moving_window_keeps_neutral_plasma_neutral():
    """A neutral plasma at rest with no fields stays exactly neutral through
    window shifts: the ion background shifted with its whole stencil plus the
    ions of the injected column cancel the electrons everywhere, including
    the seam between the old domain and the new column (Gauss residual at
    round-off, far below the plateau density)."""
    run, parts = W.lwfa_2d(n=(64, 32), d=(0.125, 0.5), patch=(16, 16), ppc=(2, 2),
                           ramp=4.0, t_mw=0.0)
    run["laser"] = None
    o = Oracle(run)
    o.load(parts)
    o.set_background("neutralising")
    o.step(3 * math.ceil(16 * 0.125 / run["dt"]))
    d = o.diag()
    assert d["shifts"] >= 2
    assert d["gauss"] < 1e-15, d["gauss"]


# ------------------------------------------------------- current filter ----

@pytest.mark.parametrize("passes", [1, 2])
@pytest.mark.parametrize("mx,my", [(1, 0), (3, 2), (8, 0), (16, 5)])
def test_binomial_filter_fourier_eigenvalue(passes, mx, my):
    """(1,2,1)/4 along an axis multiplies a Fourier mode of wavenumber k by
    cos^2(k d / 2); `passes` passes along x and y give
    cos^(2 passes)(pi mx / nx) cos^(2 passes)(pi my / ny); the Nyquist mode
    (mx = nx / 2) is removed and the sum of J is conserved."""
    run = W.periodic_run((32, 24), (0.1, 0.1), (8, 8))
    run["filter_passes"] = passes
    o = Oracle(run)
    nx, ny = 32, 24
    i = np.arange(nx)[None, :]
    j = np.arange(ny)[:, None]
    J = np.cos(2 * np.pi * mx * i / nx + 0.3) * np.cos(2 * np.pi * my * j / ny - 0.7) + 0.2
    for k in ("Jx", "Jy", "Jz"):
        o.set_field(k, J)
    o.apply_filter()
    g = (math.cos(math.pi * mx / nx) ** 2 * math.cos(math.pi * my / ny) ** 2) ** passes
    expect = g * (J - 0.2) + 0.2
    for k in ("Jx", "Jy", "Jz"):
        out = o.field(k)
        assert np.max(np.abs(out - expect)) < 1e-14, k
        assert abs(out.sum() - J.sum()) < 1e-12


def test_binomial_filter_two_pass_impulse_response_open_axes():
    """On open axes, far from the edges, two passes turn a unit impulse into
    the binomial 5 x 5 stencil (1,4,6,4,1) x (1,4,6,4,1) / 256."""
    run, _ = W.lwfa_2d(n=(32, 32), d=(0.125, 0.5), patch=(16, 16))
    run["filter_passes"] = 2
    o = Oracle(run)
    J = np.zeros(o.shape)
    J[17, 15] = 1.0
    o.set_field("Jz", J)
    o.apply_filter()
    out = o.field("Jz")
    b = np.array([1, 4, 6, 4, 1]) / 16.0
    expect = np.zeros_like(J)
    expect[15:20, 13:18] = np.outer(b, b)
    assert np.max(np.abs(out - expect)) < 1e-16
