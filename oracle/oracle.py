"""ctypes front-end of the FP64 CPU oracle.

TEST INFRASTRUCTURE ONLY: imported by tests/, by ``__graft_entry__.smoke()``
and by the CPU-baseline leg of ``bench.py``.  The product package never
imports this module and the oracle shares no code with the CUDA path.

A run is described by the plain dictionary produced by
``paper_1912_04064_gb300.workloads`` (grid, time step, patches, boundary
conditions, laser, moving window, injected plasma); this module turns it into
the oracle's own C configuration.

The periodic Poisson solve of the initial field (discrete Gauss law
div_h E = rho - <rho>, E = -grad_h phi on the Yee lattice) is written here
with numpy's FFT as a library step: the discrete Laplacian of a Fourier mode
is -(kx_h^2 + ky_h^2) with k_h = (2/d) sin(k d / 2).
"""
import ctypes as C
import math
import os

import numpy as np

from . import build as _build

FIELDS = ["Ex", "Ey", "Ez", "Bx", "By", "Bz", "Bmx", "Bmy", "Bmz",
          "Jx", "Jy", "Jz", "rho", "rho_bg"]
FBC = {"periodic": 0, "sm": 1}
PBC = {"periodic": 0, "reflect": 1, "remove": 2}


class _Cfg(C.Structure):
    _fields_ = [("nx", C.c_int), ("ny", C.c_int),
                ("dx", C.c_double), ("dy", C.c_double), ("dt", C.c_double),
                ("px", C.c_int), ("py", C.c_int),
                ("fbc_x", C.c_int), ("fbc_y", C.c_int),
                ("pbc_x", C.c_int * 2), ("pbc_y", C.c_int * 2),
                ("q", C.c_double), ("m", C.c_double),
                ("laser_on", C.c_int),
                ("a0", C.c_double), ("waist", C.c_double), ("tau", C.c_double),
                ("t_peak", C.c_double), ("y_center", C.c_double),
                ("mw_on", C.c_int), ("mw_t0", C.c_double),
                ("inj_n0", C.c_double), ("inj_x0", C.c_double), ("inj_ramp", C.c_double),
                ("inj_ppcx", C.c_int), ("inj_ppcy", C.c_int),
                ("track_continuity", C.c_int), ("filter_passes", C.c_int),
                ("nthreads", C.c_int)]


_lib = None


def lib():
    global _lib
    if _lib is None:
        _lib = C.CDLL(_build.build())
        L = _lib
        L.orc_create.restype = C.c_void_p
        L.orc_create.argtypes = [C.POINTER(_Cfg)]
        L.orc_destroy.argtypes = [C.c_void_p]
        dp = C.POINTER(C.c_double)
        L.orc_load.argtypes = [C.c_void_p] + [dp] * 6 + [C.c_long]
        L.orc_num_particles.restype = C.c_long
        L.orc_num_particles.argtypes = [C.c_void_p]
        L.orc_get_particles.restype = C.c_long
        L.orc_get_particles.argtypes = [C.c_void_p, dp]
        L.orc_set_field.argtypes = [C.c_void_p, C.c_int, dp]
        L.orc_get_field.argtypes = [C.c_void_p, C.c_int, dp]
        L.orc_set_background.argtypes = [C.c_void_p, C.c_int, C.c_double]
        L.orc_step.argtypes = [C.c_void_p, C.c_int]
        L.orc_diag.argtypes = [C.c_void_p, dp]
        L.orc_shape2.argtypes = [C.c_double, C.POINTER(C.c_int), dp]
        L.orc_boris.argtypes = [C.c_double, C.c_double, C.c_double, dp, dp, dp]
        L.orc_esirkepov.argtypes = [C.c_void_p, C.c_double, C.c_double, C.c_double,
                                    C.c_double, C.c_double, C.c_double,
                                    C.POINTER(C.c_int), C.POINTER(C.c_int), dp]
        L.orc_apply_filter.argtypes = [C.c_void_p]
        L.orc_gather.restype = C.c_double
        L.orc_gather.argtypes = [C.c_void_p, C.c_int, C.c_double, C.c_double]
        L.orc_laser_field.argtypes = [C.c_void_p, C.c_double, C.c_double, dp]
    return _lib


def _ptr(a):
    return a.ctypes.data_as(C.POINTER(C.c_double))


def make_config(run: dict, nthreads: int = 0, track_continuity: bool = False) -> _Cfg:
    c = _Cfg()
    c.nx, c.ny = run["n"]
    c.dx, c.dy = run["d"]
    c.dt = run["dt"]
    c.px, c.py = run["patch"]
    c.fbc_x, c.fbc_y = (FBC[b] for b in run["field_bc"])
    c.pbc_x[0], c.pbc_x[1] = (PBC[b] for b in run["part_bc"][0])
    c.pbc_y[0], c.pbc_y[1] = (PBC[b] for b in run["part_bc"][1])
    c.q = run.get("q", -1.0)
    c.m = run.get("m", 1.0)
    las = run.get("laser")
    if las:
        c.laser_on = 1
        c.a0, c.waist, c.tau = las["a0"], las["waist"], las["tau"]
        c.t_peak, c.y_center = las["t_peak"], las["y_center"]
    mw = run.get("moving_window")
    if mw:
        c.mw_on = 1
        c.mw_t0 = mw["t0"]
    inj = run.get("injection")
    if inj:
        c.inj_n0, c.inj_x0, c.inj_ramp = inj["n0"], inj["x0"], inj["ramp"]
        c.inj_ppcx, c.inj_ppcy = inj["ppc"]
    else:
        c.inj_ppcx = c.inj_ppcy = 1
    c.track_continuity = int(track_continuity)
    c.filter_passes = int(run.get("filter_passes", 0))
    c.nthreads = nthreads
    return c


class Oracle:
    """One oracle run (FP64, CPU)."""

    def __init__(self, run: dict, nthreads: int = 0, track_continuity: bool = False):
        self.run = run
        self.cfg = make_config(run, nthreads, track_continuity)
        self.h = lib().orc_create(C.byref(self.cfg))
        if not self.h:
            raise ValueError("oracle rejected the configuration")
        nx, ny = run["n"]
        self.shape = (ny if run["field_bc"][1] == "periodic" else ny + 2,
                      nx if run["field_bc"][0] == "periodic" else nx + 2)

    def __del__(self):
        if getattr(self, "h", None):
            lib().orc_destroy(self.h)
            self.h = None

    def load(self, p: dict):
        arrs = [np.ascontiguousarray(p[k], dtype=np.float64) for k in ("x", "y", "ux", "uy", "uz", "w")]
        n = arrs[0].size
        if lib().orc_load(self.h, *[_ptr(a) for a in arrs], n) != 0:
            raise MemoryError("oracle load failed")

    def particles(self) -> dict:
        n = lib().orc_num_particles(self.h)
        out = np.empty((6, max(n, 1)), dtype=np.float64)
        lib().orc_get_particles(self.h, _ptr(out))
        return {k: out[i, :n].copy() for i, k in enumerate(("x", "y", "ux", "uy", "uz", "w"))}

    def set_field(self, name: str, a):
        a = np.ascontiguousarray(a, dtype=np.float64)
        if a.shape != self.shape:
            raise ValueError(f"{name}: shape {a.shape} != {self.shape}")
        if lib().orc_set_field(self.h, FIELDS.index(name), _ptr(a)) != 0:
            raise ValueError(name)

    def field(self, name: str) -> np.ndarray:
        out = np.empty(self.shape, dtype=np.float64)
        lib().orc_get_field(self.h, FIELDS.index(name), _ptr(out))
        return out

    def set_background(self, mode: str, value: float = 0.0):
        m = {"none": 0, "uniform": 1, "neutralising": 2}[mode]
        lib().orc_set_background(self.h, m, value)

    def step(self, n: int = 1):
        rc = lib().orc_step(self.h, int(n))
        if rc != 0:
            raise RuntimeError("oracle step failed: a particle moved more than one cell")

    def diag(self) -> dict:
        out = np.zeros(10)
        lib().orc_diag(self.h, _ptr(out))
        keys = ("step", "t", "np", "U_E", "U_B", "U_K", "gauss", "continuity", "shifts", "charge")
        return dict(zip(keys, out.tolist()))

    def laser(self, y: float, t: float) -> float:
        v = C.c_double()
        lib().orc_laser_field(self.h, y, t, C.byref(v))
        return v.value

    def apply_filter(self):
        lib().orc_apply_filter(self.h)

    def gather(self, name: str, x: float, y: float) -> float:
        return lib().orc_gather(self.h, FIELDS.index(name), x, y)

    def esirkepov(self, x0, y0, x1, y1, w, vz):
        """Current window (Jx, Jy, Jz) of one particle and its first node."""
        J = np.zeros((3, 5, 5))
        ix, iy = C.c_int(), C.c_int()
        rc = lib().orc_esirkepov(self.h, x0, y0, x1, y1, w, vz, C.byref(ix), C.byref(iy), _ptr(J))
        if rc != 0:
            raise ValueError("move exceeds one cell")
        return J, ix.value, iy.value


def shape2(xi: float):
    S = np.zeros(3)
    i0 = C.c_int()
    lib().orc_shape2(xi, C.byref(i0), _ptr(S))
    return i0.value, S


def boris(q, m, dt, E, B, u):
    E = np.ascontiguousarray(E, dtype=np.float64)
    B = np.ascontiguousarray(B, dtype=np.float64)
    u = np.array(u, dtype=np.float64)
    lib().orc_boris(q, m, dt, _ptr(E), _ptr(B), _ptr(u))
    return u


def poisson_periodic(rho: np.ndarray, dx: float, dy: float):
    """E = -grad_h phi with div_h E = rho - mean(rho) on a periodic Yee grid.

    rho: (ny, nx) at primal nodes.  Returns (Ex, Ey) with Ex at (i+1/2, j)
    and Ey at (i, j+1/2).
    """
    ny, nx = rho.shape
    kx = 2.0 * np.pi * np.fft.fftfreq(nx, d=dx)
    ky = 2.0 * np.pi * np.fft.fftfreq(ny, d=dy)
    khx = (2.0 / dx) * np.sin(kx * dx / 2.0)
    khy = (2.0 / dy) * np.sin(ky * dy / 2.0)
    k2 = khy[:, None] ** 2 + khx[None, :] ** 2
    rh = np.fft.fft2(rho - rho.mean())
    k2[0, 0] = 1.0
    ph = rh / k2          # -lap_h phi = rho  ->  phi_hat = rho_hat / k_h^2
    ph[0, 0] = 0.0
    phi = np.real(np.fft.ifft2(ph))
    Ex = -(np.roll(phi, -1, axis=1) - phi) / dx
    Ey = -(np.roll(phi, -1, axis=0) - phi) / dy
    return Ex, Ey


def cfl_dt(d, frac=0.95):
    return frac / math.sqrt(sum(1.0 / x ** 2 for x in d))


# ------------------------------------------------------------------ 3D3V --

class _Cfg3(C.Structure):
    _fields_ = [("n", C.c_int * 3), ("d", C.c_double * 3), ("dt", C.c_double),
                ("p", C.c_int * 3), ("fbc", C.c_int * 3), ("pbc", (C.c_int * 2) * 3),
                ("q", C.c_double), ("m", C.c_double), ("laser_on", C.c_int),
                ("a0", C.c_double), ("waist", C.c_double), ("tau", C.c_double),
                ("t_peak", C.c_double), ("y_center", C.c_double), ("z_center", C.c_double),
                ("mw_on", C.c_int), ("mw_t0", C.c_double),
                ("inj_n0", C.c_double), ("inj_x0", C.c_double), ("inj_ramp", C.c_double),
                ("inj_ymin", C.c_double), ("inj_ppc", C.c_int * 3),
                ("track_continuity", C.c_int), ("nthreads", C.c_int)]


_lib3_ready = False


def lib3():
    """The oracle library with the 3D entry points' signatures set."""
    global _lib3_ready
    L = lib()
    if not _lib3_ready:
        dp = C.POINTER(C.c_double)
        vp = C.c_void_p
        L.o3_create.restype = vp
        L.o3_create.argtypes = [C.POINTER(_Cfg3)]
        L.o3_destroy.argtypes = [vp]
        L.o3_load.argtypes = [vp] + [dp] * 7 + [C.c_long]
        L.o3_fill_plasma.argtypes = [vp]
        L.o3_num_particles.restype = C.c_long
        L.o3_num_particles.argtypes = [vp]
        L.o3_get_particles.restype = C.c_long
        L.o3_get_particles.argtypes = [vp, dp]
        L.o3_set_field.argtypes = [vp, C.c_int, dp]
        L.o3_get_field.argtypes = [vp, C.c_int, dp]
        L.o3_set_background.argtypes = [vp, C.c_int, C.c_double]
        L.o3_step.argtypes = [vp, C.c_int]
        L.o3_diag.argtypes = [vp, dp]
        L.o3_esirkepov.argtypes = [vp, dp, dp, C.c_double, C.POINTER(C.c_int), dp]
        L.o3_gather.restype = C.c_double
        L.o3_gather.argtypes = [vp, C.c_int, C.c_double, C.c_double, C.c_double]
        L.o3_laser_field.argtypes = [vp, C.c_double, C.c_double, C.c_double, dp]
        _lib3_ready = True
    return L


KEYS3 = ("x", "y", "z", "ux", "uy", "uz", "w")


def make_config3(run: dict, nthreads: int = 0, track_continuity: bool = False) -> _Cfg3:
    c = _Cfg3()
    for a in range(3):
        c.n[a] = run["n"][a]
        c.d[a] = run["d"][a]
        c.p[a] = run["patch"][a]
        c.fbc[a] = FBC[run["field_bc"][a]]
        c.pbc[a][0], c.pbc[a][1] = (PBC[b] for b in run["part_bc"][a])
    c.dt = run["dt"]
    c.q = run.get("q", -1.0)
    c.m = run.get("m", 1.0)
    las = run.get("laser")
    if las:
        c.laser_on = 1
        c.a0, c.waist, c.tau = las["a0"], las["waist"], las["tau"]
        c.t_peak, c.y_center, c.z_center = las["t_peak"], las["y_center"], las["z_center"]
    mw = run.get("moving_window")
    if mw:
        c.mw_on = 1
        c.mw_t0 = mw["t0"]
    inj = run.get("injection")
    if inj:
        c.inj_n0, c.inj_x0, c.inj_ramp = inj["n0"], inj["x0"], inj["ramp"]
        c.inj_ymin = inj.get("ymin", 0.0)
        for a in range(3):
            c.inj_ppc[a] = inj["ppc"][a]
    else:
        for a in range(3):
            c.inj_ppc[a] = 1
    c.track_continuity = int(track_continuity)
    c.nthreads = nthreads
    return c


def field_shape3(run: dict):
    """(nz_e, ny_e, nx_e): per axis n (periodic) or n + 2 (open)."""
    return tuple(run["n"][a] + (0 if run["field_bc"][a] == "periodic" else 2) for a in (2, 1, 0))


class Oracle3:
    """One 3D3V oracle run (FP64, CPU)."""

    def __init__(self, run: dict, nthreads: int = 0, track_continuity: bool = False):
        self.run = run
        self.cfg = make_config3(run, nthreads, track_continuity)
        self.h = lib3().o3_create(C.byref(self.cfg))
        if not self.h:
            raise ValueError("oracle rejected the configuration")
        self.shape = field_shape3(run)

    def __del__(self):
        if getattr(self, "h", None):
            lib3().o3_destroy(self.h)
            self.h = None

    def load(self, p: dict):
        arrs = [np.ascontiguousarray(p[k], dtype=np.float64) for k in KEYS3]
        if lib3().o3_load(self.h, *[_ptr(a) for a in arrs], arrs[0].size) != 0:
            raise MemoryError("oracle load failed")

    def fill_plasma(self):
        lib3().o3_fill_plasma(self.h)

    def particles(self) -> dict:
        n = lib3().o3_num_particles(self.h)
        out = np.empty((7, max(n, 1)), dtype=np.float64)
        lib3().o3_get_particles(self.h, _ptr(out))
        return {k: out[i, :n].copy() for i, k in enumerate(KEYS3)}

    def set_field(self, name: str, a):
        a = np.ascontiguousarray(a, dtype=np.float64)
        if a.shape != self.shape:
            raise ValueError(f"{name}: shape {a.shape} != {self.shape}")
        if lib3().o3_set_field(self.h, FIELDS.index(name), _ptr(a)) != 0:
            raise ValueError(name)

    def field(self, name: str) -> np.ndarray:
        out = np.empty(self.shape, dtype=np.float64)
        lib3().o3_get_field(self.h, FIELDS.index(name), _ptr(out))
        return out

    def set_background(self, mode: str, value: float = 0.0):
        m = {"none": 0, "uniform": 1, "neutralising": 2}[mode]
        lib3().o3_set_background(self.h, m, value)

    def step(self, n: int = 1):
        rc = lib3().o3_step(self.h, int(n))
        if rc != 0:
            raise RuntimeError("oracle step failed: a particle moved more than one cell")

    def diag(self) -> dict:
        out = np.zeros(10)
        lib3().o3_diag(self.h, _ptr(out))
        keys = ("step", "t", "np", "U_E", "U_B", "U_K", "gauss", "continuity", "shifts", "charge")
        return dict(zip(keys, out.tolist()))

    def laser(self, y: float, z: float, t: float) -> float:
        v = C.c_double()
        lib3().o3_laser_field(self.h, y, z, t, C.byref(v))
        return v.value

    def gather(self, name: str, x: float, y: float, z: float) -> float:
        return lib3().o3_gather(self.h, FIELDS.index(name), x, y, z)

    def esirkepov(self, x0, x1, w):
        """Current windows J[c][k][j][i] (5^3 per component) of one particle
        and the window's first node per axis."""
        J = np.zeros((3, 5, 5, 5))
        a0 = np.ascontiguousarray(x0, dtype=np.float64)
        a1 = np.ascontiguousarray(x1, dtype=np.float64)
        ix = (C.c_int * 3)()
        rc = lib3().o3_esirkepov(self.h, _ptr(a0), _ptr(a1), w, ix, _ptr(J))
        if rc != 0:
            raise ValueError("move exceeds one cell")
        return J, tuple(ix)


def poisson_periodic3(rho: np.ndarray, d):
    """E = -grad_h phi, div_h E = rho - mean(rho) on a periodic 3D Yee grid.
    rho: (nz, ny, nx) at nodes.  Returns (Ex, Ey, Ez) on their edges."""
    nz, ny, nx = rho.shape
    dx, dy, dz = d
    kh = [(2.0 / h) * np.sin(2.0 * np.pi * np.fft.fftfreq(n, d=h) * h / 2.0)
          for n, h in ((nx, dx), (ny, dy), (nz, dz))]
    k2 = kh[2][:, None, None] ** 2 + kh[1][None, :, None] ** 2 + kh[0][None, None, :] ** 2
    rh = np.fft.fftn(rho - rho.mean())
    k2[0, 0, 0] = 1.0
    ph = rh / k2
    ph[0, 0, 0] = 0.0
    phi = np.real(np.fft.ifftn(ph))
    Ex = -(np.roll(phi, -1, axis=2) - phi) / dx
    Ey = -(np.roll(phi, -1, axis=1) - phi) / dy
    Ez = -(np.roll(phi, -1, axis=0) - phi) / dz
    return Ex, Ey, Ez
