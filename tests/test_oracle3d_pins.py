"""Pins of the 3D3V FP64 oracle against what the mathematics fixes.

- Reduction to 2D: a run one cell thick along a periodic z reproduces the
  pinned 2D oracle step for step (every field, current and particle).
- Discrete Yee eigenmode with all three wave numbers nonzero.
- Esirkepov in 3D: discrete continuity to round-off for any move of less
  than a cell per axis; zero current without motion; the z-integrated
  current of a move in the (x, y) plane equals the 2D oracle's.
- Cyclic permutation of the axes (x, y, z) -> (y, z, x) commutes with a
  step (catches an asymmetric index or sign in one component).
- Gauss's law preserved over steps from a Poisson start.
- Silver-Mueller faces: a plane wave leaves through each of the six faces
  in both polarisations with reflected energy below 1e-4, and below 1e-2 at
  oblique (30 degree) incidence; the laser reaches a0 on axis.
- Moving window with the upper-half plasma: a neutral plasma stays neutral
  through shifts; the fill places exactly the upper-half cells' particles.
- Bitwise independence of the thread count.
"""
import math

import numpy as np
import pytest

from oracle.oracle import Oracle, Oracle3, poisson_periodic3
from paper_1912_04064_gb300 import workloads as W

NAMES = ("Ex", "Ey", "Ez", "Bx", "By", "Bz", "Bmx", "Bmy", "Bmz", "Jx", "Jy", "Jz")


def rel(a, b):
    s = np.max(np.abs(b))
    return float(np.max(np.abs(a - b)) / s) if s > 0 else float(np.max(np.abs(a)))


# ------------------------------------------------------ reduction to 2D ----

def test_one_cell_thick_periodic_z_reproduces_2d_oracle():
    run2 = W.periodic_run((32, 16), (0.1, 0.12), (8, 8))
    run3 = W.periodic_run3((32, 16, 1), (0.1, 0.12, 1.0), (8, 8, 1), dt=run2["dt"])
    p2 = W.small_random_particles(run2, 3000, seed=3, uth=0.4)
    rng = np.random.default_rng(4)
    p3 = dict(p2)
    p3["z"] = rng.uniform(0.0, 1.0, p2["x"].size)
    f2 = W.random_fields(W.field_shape(run2), seed=5, amp=0.1)
    o2, o3 = Oracle(run2), Oracle3(run3)
    o2.load(p2)
    o3.load(p3)
    for k, v in f2.items():
        o2.set_field(k, v)
        o3.set_field(k, v[None, :, :])
    for _ in range(3):
        o2.step(1)
        o3.step(1)
        for k in NAMES:
            assert rel(o3.field(k)[0], o2.field(k)) < 1e-12, k
    a, b = o3.particles(), o2.particles()
    ka = np.lexsort((a["y"], a["x"]))
    kb = np.lexsort((b["y"], b["x"]))
    for k in ("x", "y", "ux", "uy", "uz", "w"):
        assert rel(a[k][ka], b[k][kb]) < 1e-12, k


def test_one_cell_thick_open_laser_window_reproduces_2d_oracle():
    """Open (Silver-Mueller) x and y faces with the laser at x_min, particles
    removed in x and reflected in y, the moving window shifting twice with
    plasma injection: the one-cell periodic-z 3D run equals the 2D run (the
    3D laser's z factor is 1 at z = z_center = 0)."""
    run2, parts = W.lwfa_2d(n=(64, 32), d=(0.125, 0.5), patch=(8, 8), ppc=(2, 2), ramp=3.0,
                            a0=1.5, waist=4.0, tau=3.0, t_mw=0.5)
    run2["laser"]["t_peak"] = 4.0
    rng = np.random.default_rng(7)
    n = parts["x"].size
    for k in ("ux", "uy", "uz"):
        parts[k] = rng.normal(0.0, 0.3, n)
    run3 = {
        "n": (64, 32, 1), "d": (0.125, 0.5, 1.0), "dt": run2["dt"], "patch": (8, 8, 1),
        "field_bc": ("sm", "sm", "periodic"),
        "part_bc": (("remove", "remove"), ("reflect", "reflect"), ("periodic", "periodic")),
        "q": -1.0, "m": 1.0,
        "laser": dict(run2["laser"], z_center=0.0),
        "moving_window": dict(run2["moving_window"]),
        "injection": dict(run2["injection"], ppc=(2, 2, 1), ymin=0.0),
    }
    p3 = dict(parts)
    p3["z"] = np.full(n, 0.5)
    f2 = W.random_fields(W.field_shape(run2), seed=8, amp=0.05)
    o2, o3 = Oracle(run2), Oracle3(run3)
    o2.load(parts)
    o3.load(p3)
    o2.set_background("neutralising")
    o3.set_background("neutralising")
    for k, v in f2.items():
        o2.set_field(k, v)
        o3.set_field(k, v[None, :, :])
    nsteps = 2 * math.ceil(8 * 0.125 / run2["dt"]) + 4
    for _ in range(nsteps):
        o2.step(1)
        o3.step(1)
    d2, d3 = o2.diag(), o3.diag()
    assert d2["shifts"] >= 2 and d3["shifts"] == d2["shifts"] and d3["np"] == d2["np"]
    for k in NAMES:
        assert rel(o3.field(k)[0], o2.field(k)) < 1e-11, k
    assert rel(o3.field("rho_bg")[0], o2.field("rho_bg")) < 1e-12


def test_reflecting_and_removing_faces_3d():
    """A particle crossing a reflecting face of each axis is mirrored and its
    normal momentum reversed; one crossing x_max is removed (zero fields,
    zero weight: the free-flight move is exact)."""
    run = W.lwfa_3d(n=(32, 16, 16), d=(0.125, 0.5, 0.5), patch=(16, 8, 8))
    run["laser"] = None
    run["moving_window"] = None
    dt = run["dt"]
    for axis, pos in ((1, [2.0, 0.02, 3.0]), (2, [2.0, 3.0, 0.02])):
        u = np.array([0.1, 0.2, 0.3])
        u[axis] = -0.9
        g = math.sqrt(1 + u @ u)
        o = Oracle3(run)
        o.load({"x": [pos[0]], "y": [pos[1]], "z": [pos[2]], "ux": [u[0]], "uy": [u[1]],
                "uz": [u[2]], "w": [0.0]})
        o.step(1)
        p = o.particles()
        key = "xyz"[axis]
        assert abs(p[key][0] - (-(pos[axis] + dt * u[axis] / g))) < 1e-15
        for a in range(3):
            expect = -u[a] if a == axis else u[a]
            assert p["u" + "xyz"[a]][0] == expect
    o = Oracle3(run)
    o.load({"x": [32 * 0.125 - 1e-3], "y": [3.0], "z": [3.0], "ux": [5.0], "uy": [0.0],
            "uz": [0.0], "w": [0.0]})
    o.step(1)
    assert o.diag()["np"] == 0


# ------------------------------------------------------------ Yee 3D -------

STAG = {"Ex": (1, 0, 0), "Ey": (0, 1, 0), "Ez": (0, 0, 1),
        "Bx": (0, 1, 1), "By": (1, 0, 1), "Bz": (1, 1, 0)}


@pytest.mark.parametrize("m", [(2, 1, 1), (1, 2, 3), (3, 0, 2)])
def test_yee3d_discrete_eigenmode(m):
    n, d = (16, 12, 10), (0.1, 0.13, 0.17)
    run = W.periodic_run3(n, d, (4, 4, 5))
    dt = run["dt"]
    k = np.array([2 * np.pi * m[a] / (n[a] * d[a]) for a in range(3)])
    K = np.array([(2.0 / d[a]) * math.sin(k[a] * d[a] / 2.0) for a in range(3)])
    Kn = float(np.linalg.norm(K))
    omega = (2.0 / dt) * math.asin(Kn * dt / 2.0)
    Om = Kn
    E0 = np.cross(K, np.array([0.3, -0.7, 0.5]))
    E0 /= np.linalg.norm(E0)
    B0 = np.cross(K, E0) / Om
    amp = {"Ex": E0[0], "Ey": E0[1], "Ez": E0[2], "Bx": B0[0], "By": B0[1], "Bz": B0[2]}
    zz, yy, xx = np.meshgrid(np.arange(n[2]), np.arange(n[1]), np.arange(n[0]), indexing="ij")

    def mode(name, t):
        s = STAG[name]
        ph = (k[0] * (xx + 0.5 * s[0]) * d[0] + k[1] * (yy + 0.5 * s[1]) * d[1] +
              k[2] * (zz + 0.5 * s[2]) * d[2] - omega * t)
        return amp[name] * np.cos(ph)

    o = Oracle3(run)
    for c in ("Ex", "Ey", "Ez"):
        o.set_field(c, mode(c, 0.0))
    for c in ("Bx", "By", "Bz"):
        o.set_field(c, mode(c, 0.5 * dt))
        o.set_field("Bm" + c[1], 0.5 * (mode(c, -0.5 * dt) + mode(c, 0.5 * dt)))
    steps = 40
    o.step(steps)
    for c in ("Ex", "Ey", "Ez"):
        assert np.max(np.abs(o.field(c) - mode(c, steps * dt))) < 1e-12, c
    for c in ("Bx", "By", "Bz"):
        assert np.max(np.abs(o.field(c) - mode(c, (steps + 0.5) * dt))) < 1e-12, c
    # discrete div B stays zero
    Bx, By, Bz = o.field("Bx"), o.field("By"), o.field("Bz")
    divB = ((np.roll(Bx, -1, 2) - Bx) / d[0] + (np.roll(By, -1, 1) - By) / d[1] +
            (np.roll(Bz, -1, 0) - Bz) / d[2])
    assert np.max(np.abs(divB)) < 1e-12


# ------------------------------------------------------- Esirkepov 3D ------

def _rho_window(o, x, w, ix, d):
    """q w S(x) S(y) S(z) on the 5^3 window starting at ix (exact node
    weights from the quadratic B-spline)."""
    from oracle.oracle import shape2
    out = np.zeros((5, 5, 5))
    S = []
    for a in range(3):
        i0, s = shape2(x[a] / d[a])
        row = np.zeros(5)
        for t in range(3):
            row[i0 - 1 + t - ix[a]] = s[t]
        S.append(row)
    q = -1.0
    return q * w * S[2][:, None, None] * S[1][None, :, None] * S[0][None, None, :]


def test_esirkepov3d_continuity_and_zero_motion():
    run = W.periodic_run3((16, 16, 16), (0.1, 0.2, 0.15), (4, 4, 4))
    o = Oracle3(run)
    d, dt = run["d"], run["dt"]
    rng = np.random.default_rng(11)
    for _ in range(300):
        x0 = np.array([rng.uniform(0.5, 1.1) for _ in range(3)]) * np.array([1, 1.5, 1.2])
        dx = rng.uniform(-0.95, 0.95, 3) * np.array(d)
        x1 = x0 + dx
        w = rng.uniform(0.5, 1.5)
        J, ix = o.esirkepov(x0, x1, w)
        r0 = _rho_window(o, x0, w, ix, d)
        r1 = _rho_window(o, x1, w, ix, d)
        Jx, Jy, Jz = J
        div = np.zeros((5, 5, 5))
        div += (Jx - np.concatenate([np.zeros((5, 5, 1)), Jx[:, :, :-1]], 2)) / d[0]
        div += (Jy - np.concatenate([np.zeros((5, 1, 5)), Jy[:, :-1, :]], 1)) / d[1]
        div += (Jz - np.concatenate([np.zeros((1, 5, 5)), Jz[:-1, :, :]], 0)) / d[2]
        res = (r1 - r0) / dt + div
        scale = max(np.max(np.abs(J)) / min(d), 1e-30)
        assert np.max(np.abs(res)) <= 1e-13 * scale
        # currents leave the window empty at its far edges (sum of W = 0)
        assert np.max(np.abs(Jx[:, :, 4])) <= 1e-14 * scale
    J, _ = o.esirkepov(np.array([0.31, 0.47, 0.52]), np.array([0.31, 0.47, 0.52]), 1.0)
    assert np.all(J == 0.0)


def test_esirkepov3d_contribution_bound():
    """3D: every current contribution of one particle of weight w moving at
    |v| < c for one step is below (3/4)^2 |q| w (prefix sum of S1 - S0 at
    most the displacement, below dt/d; transverse weight at most (3/4)^2).
    The FP32 kernels' fixed-point scale, 2^K / ((3/4)^3 |q| w_max), keeps
    contributions below (4/3) 2^K on this bound; (3/4)^3 alone is exceeded."""
    run = W.periodic_run3((16, 16, 16), (0.1, 0.2, 0.15), (4, 4, 4))
    o = Oracle3(run)
    d, dt = np.array(run["d"]), run["dt"]
    rng = np.random.default_rng(19)
    worst = 0.0
    for n in range(2000):
        if n % 2:
            x0 = rng.uniform(0.5, 1.1, 3) * np.array([1.0, 1.5, 1.2])
            v = rng.normal(size=3)
            v *= rng.uniform(0.0, 0.999999) / np.linalg.norm(v)
        else:   # fast along x, centred between x nodes, on y and z nodes
            x0 = np.array([(rng.integers(3, 8) + 0.5 + rng.uniform(-0.3, 0.3)) * d[0],
                           rng.integers(3, 8) * d[1], rng.integers(3, 8) * d[2]])
            v = np.array([rng.choice([-1, 1]) * rng.uniform(0.99, 0.999999), 0.0, 0.0])
        w = rng.uniform(0.1, 2.0)
        J, _ = o.esirkepov(x0, x0 + v * dt, w)
        worst = max(worst, float(np.max(np.abs(J))) / w)
    assert worst < 0.5625, worst
    assert worst > 0.421875, worst


def test_esirkepov3d_planar_move_integrates_to_2d():
    """A move with no z displacement: summing the 3D Jx, Jy over the z
    window gives the 2D oracle's Jx, Jy of the same (x, y) move."""
    run3 = W.periodic_run3((16, 16, 16), (0.1, 0.2, 0.15), (4, 4, 4))
    run2 = W.periodic_run((16, 16), (0.1, 0.2), (4, 4), dt=run3["dt"])
    o3, o2 = Oracle3(run3), Oracle(run2)
    rng = np.random.default_rng(12)
    for _ in range(50):
        x0 = np.array([rng.uniform(0.4, 1.2), rng.uniform(0.4, 2.0), rng.uniform(0.3, 1.5)])
        x1 = x0 + np.array([rng.uniform(-0.09, 0.09), rng.uniform(-0.19, 0.19), 0.0])
        J3, ix3 = o3.esirkepov(x0, x1, 0.8)
        J2, ix2, iy2 = o2.esirkepov(x0[0], x0[1], x1[0], x1[1], 0.8, 0.0)
        assert ix3[:2] == (ix2, iy2)
        for c in (0, 1):
            assert np.max(np.abs(J3[c].sum(0) - J2[c])) <= 1e-13 * np.max(np.abs(J2[c]))
        assert np.all(J3[2] == 0.0)


# --------------------------------------------------- axis permutation ------

def _perm_field(a):
    """(z, y, x)-indexed array of the run with axes (X, Y, Z) = (y, z, x):
    new[K = x, J = z, I = y]."""
    return np.ascontiguousarray(np.transpose(a, (2, 0, 1)))


def test_cyclic_axis_permutation_commutes_with_step():
    run = W.periodic_run3((8, 8, 8), (0.1, 0.1, 0.1), (4, 4, 4))
    p = W.small_random_particles3(run, 3000, seed=21, uth=0.4)
    f = W.random_fields(W.field_shape3(run), seed=22, amp=0.1)
    a = Oracle3(run)
    a.load(p)
    pp = {"x": p["y"], "y": p["z"], "z": p["x"], "ux": p["uy"], "uy": p["uz"], "uz": p["ux"],
          "w": p["w"]}
    b = Oracle3(run)
    b.load(pp)
    # vector components rotate with the axes: new X-component = old y
    comp = {"x": "y", "y": "z", "z": "x"}
    for k, v in f.items():
        a.set_field(k, v)
    for k in f:
        base, c = k[:-1], k[-1]
        b.set_field(k, _perm_field(f[base + comp[c]]))
    for _ in range(2):
        a.step(1)
        b.step(1)
    for k in NAMES:
        base, c = k[:-1], k[-1]
        assert rel(b.field(k), _perm_field(a.field(base + comp[c]))) < 1e-12, k


# ---------------------------------------------------------------- Gauss ----

def test_gauss_preserved_from_poisson_start():
    run = W.periodic_run3((16, 8, 8), (0.1, 0.1, 0.1), (4, 4, 4))
    p = W.small_random_particles3(run, 6000, seed=31, uth=0.2)
    o = Oracle3(run, track_continuity=True)
    o.load(p)
    rho = o.field("rho")
    o.set_background("uniform", -float(rho.mean()))
    Ex, Ey, Ez = poisson_periodic3(rho, run["d"])
    for k, v in (("Ex", Ex), ("Ey", Ey), ("Ez", Ez)):
        o.set_field(k, v)
    g0 = o.diag()["gauss"]
    scale = float(np.max(np.abs(rho)))
    assert g0 < 1e-12 * scale
    o.step(6)
    d = o.diag()
    assert d["gauss"] < 1e-11 * scale, d
    assert d["continuity"] < 1e-10 * scale / run["dt"], d


# --------------------------------------------------- Silver-Mueller 3D -----

def _open_axis_run(axis, n_long=768, n_tr=4, d_long=0.125, d_tr=0.5):
    n = [n_tr] * 3
    d = [d_tr] * 3
    n[axis] = n_long
    d[axis] = d_long
    patch = [n_tr] * 3
    patch[axis] = 32
    run = W.periodic_run3(tuple(n), tuple(d), tuple(patch))
    fb = ["periodic"] * 3
    fb[axis] = "sm"
    run["field_bc"] = tuple(fb)
    pb = [("periodic", "periodic")] * 3
    pb[axis] = ("remove", "remove")
    run["part_bc"] = tuple(pb)
    return run


@pytest.mark.parametrize("axis", [0, 1, 2])
@pytest.mark.parametrize("pol", [0, 1])
@pytest.mark.parametrize("direction", [+1, -1])
def test_plane_wave_leaves_every_face(axis, pol, direction):
    """A wave packet along `axis` with E along one of the two transverse
    axes, travelling towards the lower (direction -1) or upper face: the
    energy left behind after it has crossed the face is below 1e-4."""
    run = _open_axis_run(axis)
    o = Oracle3(run)
    dt, dl = run["dt"], run["d"][axis]
    tr = [b for b in range(3) if b != axis]
    ecomp = tr[pol]
    bcomp = [b for b in range(3) if b not in (axis, ecomp)][0]
    # for propagation along +axis: B = axis_hat x E
    sign = np.cross(np.eye(3)[axis], np.eye(3)[ecomp])[bcomp]
    sig, xc = 10.0, 48.0

    def f(s):
        return np.exp(-((s - xc) / sig) ** 2) * np.cos(s)

    names = "xyz"
    shape = o.shape
    L = run["n"][axis] * dl
    if direction < 0:
        xc = L - 48.0
    ax_arr = 2 - axis  # array axis of `axis` in (z, y, x)

    def along(stag_shift, t):
        pos = (np.arange(shape[ax_arr]) - 1 + 0.5 * stag_shift) * dl
        v = f(pos - direction * t)
        sh = [1, 1, 1]
        sh[ax_arr] = -1
        return np.broadcast_to(v.reshape(sh), shape).copy()

    e = along(0, 0.0)
    o.set_field("E" + names[ecomp], e)
    o.set_field("B" + names[bcomp], direction * sign * along(1, 0.5 * dt))
    o.set_field("Bm" + names[bcomp], direction * sign * along(1, 0.0))
    e0 = np.sum(e ** 2)
    o.step(int(90.0 / dt))
    left = np.sum(o.field("E" + names[ecomp]) ** 2) + np.sum(o.field("B" + names[bcomp]) ** 2)
    assert left / e0 < 1e-4, left / e0


def test_oblique_incidence_absorbed():
    """A plane wave hitting the x_min face at 30 degrees (k_y != 0, TE and
    TM): reflected energy below 1e-2 of the incident energy."""
    nx, ny, nz = 512, 32, 2
    d = (0.125, 0.125 * 4, 0.5)
    for pol in ("Ez", "Ey"):
        run = W.periodic_run3((nx, ny, nz), d, (32, 16, 2))
        run["field_bc"] = ("sm", "periodic", "periodic")
        run["part_bc"] = (("remove", "remove"), ("periodic", "periodic"), ("periodic", "periodic"))
        o = Oracle3(run)
        dt = run["dt"]
        Ly = ny * d[1]
        ky = 2 * np.pi / Ly
        kx = -ky / math.tan(math.radians(30.0))   # travelling towards x_min
        kk = math.hypot(kx, ky)
        sig, xc = 12.0, 40.0
        shape = o.shape
        zz, yy, xx = np.meshgrid(np.arange(shape[0]), np.arange(shape[1]),
                                 np.arange(shape[2]) - 1, indexing="ij")
        khat = np.array([kx, ky, 0.0]) / kk

        def wave(sx, sy, t):
            x = (xx + 0.5 * sx) * d[0]
            y = (yy + 0.5 * sy) * d[1]
            s = x * khat[0] + y * khat[1] - t
            env = np.exp(-((x - xc - khat[0] * t) / sig) ** 2)
            return env * np.cos(kk * (s + xc * (-khat[0])))

        if pol == "Ez":   # E along z, B = khat x E in the (x, y) plane
            o.set_field("Ez", wave(0, 0, 0.0))
            b = np.cross(khat, [0, 0, 1.0])
            o.set_field("Bx", b[0] * wave(0, 1, 0.5 * dt))
            o.set_field("By", b[1] * wave(1, 0, 0.5 * dt))
            o.set_field("Bmx", b[0] * wave(0, 1, 0.0))
            o.set_field("Bmy", b[1] * wave(1, 0, 0.0))
        else:             # E in the (x, y) plane, B along z
            ev = np.cross([0, 0, 1.0], khat)
            o.set_field("Ex", ev[0] * wave(1, 0, 0.0))
            o.set_field("Ey", ev[1] * wave(0, 1, 0.0))
            o.set_field("Bz", wave(1, 1, 0.5 * dt))
            o.set_field("Bmz", wave(1, 1, 0.0))
        d0 = o.diag()
        u0 = d0["U_E"] + d0["U_B"]
        o.step(int(80.0 / dt))
        d1 = o.diag()
        assert (d1["U_E"] + d1["U_B"]) / u0 < 1e-2, (pol, (d1["U_E"] + d1["U_B"]) / u0)


def test_laser3d_amplitude():
    """The Gaussian beam entering through x_min reaches, on axis, a0 times
    the largest value of envelope x carrier, max_t exp(-2 ln2 t^2 / tau^2)
    |sin t|, times its diffraction between the focus (x_min) and the probe,
    w0 / w(x) = (1 + (x / z_R)^2)^(-1/2), z_R = w0^2 / 2 (k = 1): within
    1.5 %."""
    nx, ny, nz = 64, 96, 96
    waist, a0, tau = 12.0, 2.0, 12.0
    run = W.lwfa_3d(n=(nx, ny, nz), d=(0.125, 0.5, 0.5), patch=(32, 16, 16), a0=a0,
                    waist=waist, tau=tau, upper_half=False)
    run["moving_window"] = None
    run["injection"]["n0"] = 0.0
    o = Oracle3(run)
    xprobe = 4.0
    ip, jc, kc = int(round(xprobe / 0.125)) + 1, ny // 2 + 1, nz // 2 + 1
    peak = 0.0
    for _ in range(int((3 * tau + xprobe) / run["dt"])):
        o.step(1)
        peak = max(peak, abs(o.field("Ey")[kc, jc, ip]))
    # Ey at (x, y + dy/2, z): the profile there is exp(-(dy/2 / w)^2) of a0
    zr = waist ** 2 / 2.0
    tt = np.linspace(-3 * tau, 3 * tau, 200001)
    env = float(np.max(np.abs(np.exp(-2 * math.log(2) * tt ** 2 / tau ** 2) * np.sin(tt))))
    expect = (a0 * env * math.exp(-((0.25 / waist) ** 2)) /
              math.sqrt(1.0 + (xprobe / zr) ** 2))
    assert abs(peak / expect - 1.0) < 0.015, (peak, expect)
    # the injected beam is centred on (y_center, z_center): Ey sits at
    # y = (j + 1/2) dy, z = k dz, so the field is mirror-symmetric under
    # j -> ny - 1 - j and k -> nz - k (layout index = grid index + 1)
    ey = o.field("Ey")[:, :, ip]
    jj = np.arange(ny)
    kk = np.arange(1, nz)
    assert np.max(np.abs(ey[:, 1 + jj] - ey[:, 1 + (ny - 1 - jj)])) <= 1e-12 * np.max(np.abs(ey))
    assert np.max(np.abs(ey[1 + kk, :] - ey[1 + (nz - kk), :])) <= 1e-12 * np.max(np.abs(ey))
    t = 2 * tau + math.pi / 2
    assert abs(o.laser(ny * 0.25, nz * 0.25, t) -
               a0 * math.exp(-2 * math.log(2) * (math.pi / 2 / tau) ** 2)) < 1e-12


# ------------------------------------------------------ moving window ------

def test_fill_upper_half_and_window_keep_plasma_neutral():
    run = W.lwfa_3d(n=(32, 16, 8), d=(0.125, 0.5, 0.5), patch=(8, 8, 8), ppc=(2, 1, 2),
                    n0=0.01, ramp=2.0, t_mw=0.0)
    run["laser"] = None
    o = Oracle3(run)
    o.fill_plasma()
    p = o.particles()
    assert p["x"].size == 32 * 8 * 8 * 4          # the upper 8 of 16 rows
    assert np.all(p["y"] >= 8 * 0.5)
    assert np.all(p["ux"] == 0)
    d0 = o.diag()
    assert abs(d0["charge"] - (-np.sum(p["w"]) * 0.125 * 0.25)) < 1e-15 * p["x"].size
    assert d0["gauss"] < 1e-15
    o.step(3 * math.ceil(8 * 0.125 / run["dt"]))
    d = o.diag()
    assert d["shifts"] >= 2
    assert d["gauss"] < 1e-15, d["gauss"]
    assert d["U_E"] == 0.0 and d["U_K"] == 0.0


def test_thread_count_invariance_bitwise():
    run = W.periodic_run3((16, 8, 8), (0.1, 0.1, 0.1), (4, 4, 4))
    p = W.small_random_particles3(run, 5000, seed=41, uth=0.4)
    outs = []
    for nt in (1, 4):
        o = Oracle3(run, nthreads=nt)
        o.load(p)
        o.step(3)
        outs.append([o.field(k) for k in NAMES])
    for a, b in zip(*outs):
        assert np.array_equal(a, b)
