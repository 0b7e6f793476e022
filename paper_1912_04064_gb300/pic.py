"""Thin ctypes binding of libpic (include/pic.h).

Argument marshalling only: every step of the particle-in-cell path runs in
the library's sm_103a kernels.  The functions keep the C names
(``pic_create``, ``pic_load_particles``, ``pic_step``, ``pic_get_field``,
``pic_diag`` ...); :class:`Pic` bundles them for one context.  Host buffers
are numpy float64 arrays; device buffers are torch CUDA tensors (torch only
provides device memory and streams).

The library must be built (``paper_1912_04064_gb300.build.build()``); there
is no fallback: importing the binding without ``libpic.so`` raises.
"""
import ctypes as C
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
# PIC_CHECKED=1: the bounds-checked build (build.build(checked=True))
LIB_PATH = os.path.join(HERE, "libpic_checked.so" if os.environ.get("PIC_CHECKED") == "1"
                        else "libpic.so")

PIC_OK, PIC_EINVAL, PIC_ENOMEM, PIC_ECUDA, PIC_EOVERFLOW, PIC_ETIMEOUT, PIC_ENONFINITE, PIC_ESTATE = range(8)
STATUS = ["PIC_OK", "PIC_EINVAL", "PIC_ENOMEM", "PIC_ECUDA", "PIC_EOVERFLOW", "PIC_ETIMEOUT",
          "PIC_ENONFINITE", "PIC_ESTATE"]
PIC_FP64, PIC_FP32 = 0, 1
PIC_HOST, PIC_DEVICE = 0, 1
FIELDS = ["Ex", "Ey", "Ez", "Bx", "By", "Bz", "Bmx", "Bmy", "Bmz", "Jx", "Jy", "Jz", "rho", "rho_bg"]
FBC = {"periodic": 0, "sm": 1}
PBC = {"periodic": 0, "reflect": 1, "remove": 2}
BG = {"none": 0, "uniform": 1, "neutralising": 2}
KEYS2 = ("x", "y", "ux", "uy", "uz", "w")
KEYS3 = ("x", "y", "z", "ux", "uy", "uz", "w")


class pic_config(C.Structure):
    _fields_ = [
        ("dims", C.c_int), ("n", C.c_int * 3), ("d", C.c_double * 3), ("dt", C.c_double),
        ("patch", C.c_int * 3), ("prec", C.c_int), ("bc_field", C.c_int * 3),
        ("bc_part", (C.c_int * 2) * 3), ("q", C.c_double), ("m", C.c_double),
        ("laser_on", C.c_int), ("laser_a0", C.c_double), ("laser_waist", C.c_double),
        ("laser_tau", C.c_double), ("laser_t_peak", C.c_double), ("laser_y_center", C.c_double),
        ("moving_window", C.c_int), ("mw_t0", C.c_double),
        ("inj_n0", C.c_double), ("inj_x0", C.c_double), ("inj_ramp", C.c_double),
        ("inj_ppc", C.c_int * 3), ("capacity_factor", C.c_double), ("capacity_min", C.c_int),
        ("stream", C.c_void_p), ("device", C.c_int), ("use_graph", C.c_int), ("timing", C.c_int),
        ("tma", C.c_int), ("block", C.c_int), ("merge", C.c_int), ("auto_grow", C.c_int),
        ("sort_every", C.c_int), ("task_chunk", C.c_int), ("filter_passes", C.c_int),
        ("inj_ymin", C.c_double), ("laser_z_center", C.c_double), ("window_cells", C.c_int),
        ("dev_alloc", C.c_void_p), ("dev_free", C.c_void_p), ("alloc_user", C.c_void_p),
        ("current_float", C.c_int), ("staging_wait_polls", C.c_longlong),
        ("deterministic", C.c_int),
    ]


# the caller's device allocator (pic_config.dev_alloc / dev_free)
DEV_ALLOC = C.CFUNCTYPE(C.c_void_p, C.c_size_t, C.c_void_p)
DEV_FREE = C.CFUNCTYPE(None, C.c_void_p, C.c_void_p)


def torch_allocator(device: int = 0):
    """dev_alloc / dev_free callbacks that take the context's device memory
    from PyTorch's caching allocator; returns (alloc, free), to be kept alive
    as long as the context (``Pic(cfg, allocator=...)`` does)."""
    import torch

    def alloc(nbytes, _user):
        try:
            return torch.cuda.caching_allocator_alloc(int(nbytes), device)
        except Exception:
            return None

    def free(ptr, _user):
        torch.cuda.caching_allocator_delete(ptr)

    return DEV_ALLOC(alloc), DEV_FREE(free)


class pic_diag_t(C.Structure):
    _fields_ = [
        ("step", C.c_longlong), ("t", C.c_double), ("np", C.c_longlong),
        ("U_E", C.c_double), ("U_B", C.c_double), ("U_K", C.c_double),
        ("gauss", C.c_double), ("continuity", C.c_double), ("charge", C.c_double),
        ("shifts", C.c_int), ("max_patch_count", C.c_int), ("capacity", C.c_int),
        ("ms_particles", C.c_double), ("ms_fields", C.c_double), ("ms_window", C.c_double),
        ("launches", C.c_longlong), ("particle_step_launches", C.c_longlong),
        ("grows", C.c_int), ("sorts", C.c_longlong), ("ms_sort", C.c_double),
        ("calm_particle_steps", C.c_longlong),
    ]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class pic_tune_t(C.Structure):
    _fields_ = [("patch", C.c_int * 3), ("block", C.c_int), ("task_chunk", C.c_int),
                ("ms_per_step", C.c_double), ("ms_given", C.c_double), ("candidates", C.c_int)]


class pic_batch_config(C.Structure):
    _fields_ = [("stream", C.c_void_p), ("device", C.c_int), ("use_graph", C.c_int),
                ("task_chunk", C.c_int)]


class pic_batch_diag_t(C.Structure):
    _fields_ = [("steps", C.c_longlong), ("launches", C.c_longlong), ("builds", C.c_longlong),
                ("nruns", C.c_int), ("grid", C.c_int)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


PIC_BATCH_MAX = 64
PIC_REQ_QUEUED, PIC_REQ_RUNNING, PIC_REQ_DONE, PIC_REQ_FAILED, PIC_REQ_CANCELLED = range(5)


class pic_server_config(C.Structure):
    _fields_ = [("stream", C.c_void_p), ("device", C.c_int), ("hbm_budget", C.c_size_t),
                ("max_runs", C.c_int), ("steps_per_tick", C.c_int), ("use_graph", C.c_int)]


class pic_request_info(C.Structure):
    _fields_ = [("state", C.c_int), ("status", C.c_int), ("steps_done", C.c_longlong),
                ("steps_total", C.c_longlong), ("np0", C.c_longlong), ("np", C.c_longlong),
                ("footprint", C.c_size_t), ("t_submit", C.c_double), ("t_admit", C.c_double),
                ("t_done", C.c_double), ("U_E", C.c_double), ("U_B", C.c_double),
                ("U_K", C.c_double)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class pic_server_stats(C.Structure):
    _fields_ = [("submitted", C.c_longlong), ("done", C.c_longlong), ("failed", C.c_longlong),
                ("queued", C.c_longlong), ("running", C.c_longlong), ("ticks", C.c_longlong),
                ("batched_steps", C.c_longlong), ("particle_steps", C.c_double),
                ("hbm_in_use", C.c_size_t), ("busy_s", C.c_double), ("cancelled", C.c_longlong)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}

EXPORTS = ["pic_create", "pic_load_particles", "pic_set_field", "pic_set_background", "pic_step",
           "pic_get_field", "pic_get_particles", "pic_diag", "pic_sync", "pic_snapshot",
           "pic_restore", "pic_footprint", "pic_last_error", "pic_destroy", "pic_version",
           "pic_field_energy_noalloc", "pic_batch_create", "pic_batch_set", "pic_batch_step",
           "pic_batch_size", "pic_batch_get_diag", "pic_batch_last_error", "pic_batch_destroy",
           "pic_load_plasma", "pic_autotune", "pic_autotune_clear_cache", "pic_server_create",
           "pic_server_submit", "pic_server_tick", "pic_server_info", "pic_server_take",
           "pic_server_get_stats", "pic_server_clock", "pic_server_destroy", "pic_load_particles3",
           "pic_init_fields", "pic_server_cancel", "pic_autotune_plasma"]

_lib = None


def lib():
    """Load libpic.so (raises if it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"libpic.so not built at {LIB_PATH}: run paper_1912_04064_gb300.build.build()")
        L = C.CDLL(LIB_PATH)
        vp, dp, sz = C.c_void_p, C.c_void_p, C.c_size_t
        L.pic_create.argtypes = [C.POINTER(pic_config), C.POINTER(C.c_void_p)]
        L.pic_load_particles.argtypes = [vp] + [dp] * 6 + [sz, C.c_int]
        L.pic_set_field.argtypes = [vp, C.c_int, dp, C.c_int]
        L.pic_set_background.argtypes = [vp, C.c_int, C.c_double]
        L.pic_step.argtypes = [vp, C.c_int]
        L.pic_get_field.argtypes = [vp, C.c_int, dp, C.c_int]
        L.pic_get_particles.argtypes = [vp, dp, sz, C.POINTER(C.c_size_t), C.c_int]
        L.pic_diag.argtypes = [vp, C.POINTER(pic_diag_t)]
        L.pic_sync.argtypes = [vp]
        L.pic_snapshot.argtypes = [vp, vp, C.POINTER(C.c_size_t)]
        L.pic_restore.argtypes = [vp, vp, sz]
        L.pic_footprint.argtypes = [C.POINTER(pic_config), sz]
        L.pic_footprint.restype = sz
        L.pic_last_error.argtypes = [vp]
        L.pic_last_error.restype = C.c_char_p
        L.pic_destroy.argtypes = [vp]
        L.pic_destroy.restype = None
        L.pic_version.restype = C.c_char_p
        L.pic_field_energy_noalloc.argtypes = [vp] * 6 + [C.c_int, C.c_int, C.c_double, vp, vp]
        L.pic_field_energy_noalloc.restype = C.c_int
        L.pic_load_plasma.argtypes = [vp]
        L.pic_init_fields.argtypes = [vp, C.c_int]
        L.pic_init_fields.restype = C.c_int
        L.pic_load_particles3.argtypes = [vp] + [dp] * 7 + [sz, C.c_int]
        L.pic_load_particles3.restype = C.c_int
        L.pic_autotune.argtypes = ([C.POINTER(pic_config)] + [dp] * 6 +
                                   [sz, C.c_int, C.c_int, C.POINTER(pic_config), C.POINTER(pic_tune_t)])
        L.pic_autotune_clear_cache.restype = None
        L.pic_autotune_plasma.argtypes = [C.POINTER(pic_config), C.c_int, C.POINTER(pic_config),
                                          C.POINTER(pic_tune_t)]
        L.pic_autotune_plasma.restype = C.c_int
        L.pic_server_create.argtypes = [C.POINTER(pic_server_config), C.POINTER(C.c_void_p)]
        L.pic_server_submit.argtypes = [vp, C.POINTER(pic_config), C.c_longlong, C.c_int,
                                        C.POINTER(C.c_longlong)]
        L.pic_server_tick.argtypes = [vp, C.POINTER(C.c_int)]
        L.pic_server_info.argtypes = [vp, C.c_longlong, C.POINTER(pic_request_info)]
        L.pic_server_take.argtypes = [vp, C.c_longlong, C.POINTER(C.c_void_p)]
        L.pic_server_cancel.argtypes = [vp, C.c_longlong]
        L.pic_server_cancel.restype = C.c_int
        L.pic_server_get_stats.argtypes = [vp, C.POINTER(pic_server_stats)]
        L.pic_server_clock.argtypes = [vp]
        L.pic_server_clock.restype = C.c_double
        L.pic_server_destroy.argtypes = [vp]
        L.pic_server_destroy.restype = None
        L.pic_batch_create.argtypes = [C.POINTER(pic_batch_config), C.POINTER(C.c_void_p)]
        L.pic_batch_set.argtypes = [vp, C.POINTER(C.c_void_p), C.c_int]
        L.pic_batch_step.argtypes = [vp, C.c_int]
        L.pic_batch_size.argtypes = [vp]
        L.pic_batch_get_diag.argtypes = [vp, C.POINTER(pic_batch_diag_t)]
        L.pic_batch_last_error.argtypes = [vp]
        L.pic_batch_last_error.restype = C.c_char_p
        L.pic_batch_destroy.argtypes = [vp]
        L.pic_batch_destroy.restype = None
        for name in ("pic_create", "pic_load_particles", "pic_set_field", "pic_set_background",
                     "pic_step", "pic_get_field", "pic_get_particles", "pic_diag", "pic_sync",
                     "pic_snapshot", "pic_restore", "pic_batch_create", "pic_batch_set",
                     "pic_batch_step", "pic_batch_size", "pic_batch_get_diag", "pic_load_plasma",
                     "pic_autotune", "pic_server_create", "pic_server_submit", "pic_server_tick",
                     "pic_server_info", "pic_server_take", "pic_server_get_stats"):
            getattr(L, name).restype = C.c_int
        _lib = L
    return _lib


class PicError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{STATUS[status] if 0 <= status < len(STATUS) else status}: {msg}")
        self.status = status


def config_from_run(run: dict, prec: str = "fp64", stream=None, device: int = 0,
                    use_graph: bool = True, timing: bool = False, tma: bool = True,
                    capacity_factor: float = 0.0, capacity_min: int = 0, block: int = 0,
                    merge: int = -1, auto_grow: bool = True, sort_every: int = 0,
                    task_chunk: int = 0, patch=None, current_float: bool = False,
                    staging_wait_polls: int = 0, deterministic: bool = False) -> pic_config:
    """pic_config of a run dictionary (see ``workloads``); `patch` overrides
    the run's patch size (the window step stays the run's patch width
    unless the run names its own ``moving_window["cells"]``)."""
    c = pic_config()
    dims = len(run["n"])
    c.dims = dims
    for a in range(3):
        c.n[a] = run["n"][a] if a < dims else 1
        c.d[a] = run["d"][a] if a < dims else 1.0
        c.patch[a] = (patch or run["patch"])[a] if a < dims else 1
    c.dt = run["dt"]
    c.prec = PIC_FP32 if prec in ("fp32", PIC_FP32) else PIC_FP64
    for a in range(dims):
        c.bc_field[a] = FBC[run["field_bc"][a]]
        for f in range(2):
            c.bc_part[a][f] = PBC[run["part_bc"][a][f]]
    c.q = run.get("q", -1.0)
    c.m = run.get("m", 1.0)
    las = run.get("laser")
    if las:
        c.laser_on = 1
        c.laser_a0, c.laser_waist, c.laser_tau = las["a0"], las["waist"], las["tau"]
        c.laser_t_peak, c.laser_y_center = las["t_peak"], las["y_center"]
        c.laser_z_center = las.get("z_center", 0.0)
    mw = run.get("moving_window")
    if mw:
        c.moving_window = 1
        c.mw_t0 = mw["t0"]
        c.window_cells = int(mw.get("cells", run["patch"][0] if patch else 0))
    inj = run.get("injection")
    if inj:
        c.inj_n0, c.inj_x0, c.inj_ramp = inj["n0"], inj["x0"], inj["ramp"]
        ppc = tuple(inj["ppc"]) + (1,) * (3 - len(inj["ppc"]))
        c.inj_ppc[0], c.inj_ppc[1], c.inj_ppc[2] = ppc
        c.inj_ymin = inj.get("ymin", 0.0)
    else:
        c.inj_ppc[0] = c.inj_ppc[1] = c.inj_ppc[2] = 1
    c.capacity_factor = capacity_factor
    c.capacity_min = capacity_min
    c.stream = stream
    c.device = device
    c.use_graph = int(use_graph)
    c.timing = int(timing)
    c.tma = 1 if tma else 0
    c.block = block
    c.merge = merge
    c.auto_grow = int(auto_grow)
    c.current_float = int(current_float)
    c.staging_wait_polls = int(staging_wait_polls)
    c.deterministic = int(deterministic)
    c.sort_every = sort_every
    c.task_chunk = task_chunk
    c.filter_passes = int(run.get("filter_passes", 0))
    return c


def pic_footprint(cfg: pic_config, np_max: int) -> int:
    return lib().pic_footprint(C.byref(cfg), np_max)


def pic_version() -> str:
    return lib().pic_version().decode()


def _ptr(a):
    """Pointer and location of a host numpy array or a CUDA tensor."""
    if isinstance(a, np.ndarray):
        return a.ctypes.data, PIC_HOST
    if hasattr(a, "data_ptr"):
        return a.data_ptr(), (PIC_DEVICE if a.is_cuda else PIC_HOST)
    raise TypeError(type(a))


def _field_shape(cfg: pic_config):
    dims = 3 if cfg.dims == 3 else 2
    return tuple(cfg.n[a] + (0 if cfg.bc_field[a] == 0 else 2) for a in reversed(range(dims)))


class Pic:
    """One libpic context (C-ABI calls with argument marshalling)."""

    def __init__(self, cfg: pic_config, allocator=None):
        """allocator: optional (dev_alloc, dev_free) ctypes callbacks (e.g.
        ``torch_allocator()``) for all device memory of the context; kept
        alive with it."""
        self.cfg = cfg
        self._allocator = allocator
        if allocator is not None:
            cfg.dev_alloc = C.cast(allocator[0], C.c_void_p)
            cfg.dev_free = C.cast(allocator[1], C.c_void_p)
        self.h = C.c_void_p()
        self._check(lib().pic_create(C.byref(cfg), C.byref(self.h)), create=True)
        self.shape = _field_shape(cfg)

    @classmethod
    def adopt(cls, h, cfg: pic_config) -> "Pic":
        """Wrap a context created elsewhere (e.g. handed over by a server)."""
        self = cls.__new__(cls)
        self.cfg = cfg
        self.h = h
        self.shape = _field_shape(cfg)
        return self

    def _check(self, rc, create=False):
        if rc != PIC_OK:
            msg = "" if create or not self.h else lib().pic_last_error(self.h).decode()
            raise PicError(rc, msg or "pic_create rejected the configuration")

    def close(self):
        if self.h:
            lib().pic_destroy(self.h)
            self.h = C.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # -- C-ABI calls
    def pic_load_particles(self, p: dict):
        """Particles as a dict of float64 arrays (numpy: host, torch CUDA:
        device); 3D contexts take "z" too (pic_load_particles3)."""
        keys = KEYS3 if self.cfg.dims == 3 else KEYS2
        arrs = []
        for k in keys:
            a = p[k]
            if isinstance(a, np.ndarray) or not hasattr(a, "data_ptr"):
                a = np.ascontiguousarray(a, dtype=np.float64)
            arrs.append(a)
        ptrs = [_ptr(a) for a in arrs]
        where = ptrs[0][1]
        n = int(arrs[0].shape[0])
        fn = lib().pic_load_particles3 if self.cfg.dims == 3 else lib().pic_load_particles
        self._check(fn(self.h, *[q for q, _ in ptrs], n, where))

    def pic_load_plasma(self):
        """Fill the domain with the configuration's plasma profile on the device."""
        self._check(lib().pic_load_plasma(self.h))

    def pic_set_field(self, name: str, a):
        if isinstance(a, np.ndarray) or not hasattr(a, "data_ptr"):
            a = np.ascontiguousarray(a, dtype=np.float64)
        if tuple(a.shape) != self.shape:
            raise ValueError(f"{name}: shape {tuple(a.shape)} != {self.shape}")
        q, where = _ptr(a)
        self._check(lib().pic_set_field(self.h, FIELDS.index(name), q, where))

    def pic_init_fields(self, mode: str = "poisson"):
        """Initial fields: "zero", or "poisson" (E from Gauss's law, periodic axes)."""
        self._check(lib().pic_init_fields(self.h, {"zero": 0, "poisson": 1}[mode]))

    def pic_set_background(self, mode: str, value: float = 0.0):
        self._check(lib().pic_set_background(self.h, BG[mode], value))

    def pic_step(self, n: int = 1):
        self._check(lib().pic_step(self.h, int(n)))

    def pic_get_field(self, name: str, out=None):
        if out is None:
            out = np.empty(self.shape, dtype=np.float64)
        q, where = _ptr(out)
        self._check(lib().pic_get_field(self.h, FIELDS.index(name), q, where))
        return out

    def pic_get_particles(self, out=None) -> dict:
        """Particles as float64 arrays (global positions, u, w).  `out`: an
        optional host array of shape (6, >= count) (7 rows in 3D) to fill,
        e.g. page-locked memory, which the library writes in place; the
        returned arrays are views of it."""
        n = C.c_size_t()
        self._check(lib().pic_get_particles(self.h, None, 0, C.byref(n), PIC_HOST))
        keys = KEYS3 if self.cfg.dims == 3 else KEYS2
        if out is None or out.shape[0] != len(keys) or out.shape[1] < n.value or \
                out.dtype != np.float64 or not out.flags["C_CONTIGUOUS"]:
            out = np.empty((len(keys), max(n.value, 1)), dtype=np.float64)
        cap = out.shape[1]
        self._check(lib().pic_get_particles(self.h, out.ctypes.data, cap, C.byref(n), PIC_HOST))
        m = n.value
        return {k: out[i, :m] for i, k in enumerate(keys)}

    def pic_diag(self) -> dict:
        d = pic_diag_t()
        self._check(lib().pic_diag(self.h, C.byref(d)))
        return d.as_dict()

    def pic_sync(self):
        self._check(lib().pic_sync(self.h))

    def pic_snapshot(self) -> bytes:
        n = C.c_size_t()
        self._check(lib().pic_snapshot(self.h, None, C.byref(n)))
        buf = C.create_string_buffer(n.value)
        self._check(lib().pic_snapshot(self.h, buf, C.byref(n)))
        return buf.raw

    def pic_restore(self, blob: bytes):
        buf = C.create_string_buffer(blob, len(blob))
        self._check(lib().pic_restore(self.h, buf, len(blob)))

    def last_error(self) -> str:
        return lib().pic_last_error(self.h).decode() if self.h else ""


def pic_autotune(cfg: pic_config, parts: dict, steps: int = 5):
    """Time candidate launch shapes on `parts` (host float64 arrays); returns
    (tuned pic_config, dict of the choice and timings)."""
    arrs = [np.ascontiguousarray(parts[k], dtype=np.float64)
            for k in ("x", "y", "ux", "uy", "uz", "w")]
    tuned, res = pic_config(), pic_tune_t()
    rc = lib().pic_autotune(C.byref(cfg), *[a.ctypes.data for a in arrs], int(arrs[0].size),
                            PIC_HOST, int(steps), C.byref(tuned), C.byref(res))
    if rc != PIC_OK:
        raise PicError(rc, "pic_autotune failed")
    info = {"patch": (res.patch[0], res.patch[1]), "block": res.block,
            "task_chunk": res.task_chunk, "ms_per_step": res.ms_per_step,
            "ms_given": res.ms_given, "candidates": res.candidates}
    return tuned, info


def pic_autotune_plasma(cfg: pic_config, steps: int = 5):
    """Time candidate launch shapes on the configured plasma (filled on the
    device; 2D or 3D); returns (tuned pic_config, dict of the choice)."""
    tuned, res = pic_config(), pic_tune_t()
    rc = lib().pic_autotune_plasma(C.byref(cfg), int(steps), C.byref(tuned), C.byref(res))
    if rc != PIC_OK:
        raise PicError(rc, "pic_autotune_plasma failed")
    info = {"patch": tuple(res.patch[a] for a in range(cfg.dims)), "block": res.block,
            "task_chunk": res.task_chunk, "ms_per_step": res.ms_per_step,
            "ms_given": res.ms_given, "candidates": res.candidates}
    return tuned, info


class Batch:
    """A batch of contexts advanced together (pic_batch_* calls)."""

    def __init__(self, stream=None, device: int = 0, use_graph: bool = True, task_chunk: int = 0):
        cfg = pic_batch_config(stream, device, int(use_graph), int(task_chunk))
        self.h = C.c_void_p()
        self.runs = []
        rc = lib().pic_batch_create(C.byref(cfg), C.byref(self.h))
        if rc != PIC_OK:
            raise PicError(rc, "pic_batch_create failed")

    def _check(self, rc):
        if rc != PIC_OK:
            raise PicError(rc, lib().pic_batch_last_error(self.h).decode())

    def pic_batch_set(self, runs):
        arr = (C.c_void_p * max(len(runs), 1))(*[r.h.value for r in runs])
        self._check(lib().pic_batch_set(self.h, arr, len(runs)))
        self.runs = list(runs)

    def pic_batch_step(self, n: int = 1):
        self._check(lib().pic_batch_step(self.h, int(n)))

    def pic_batch_size(self) -> int:
        return lib().pic_batch_size(self.h)

    def pic_batch_get_diag(self) -> dict:
        d = pic_batch_diag_t()
        self._check(lib().pic_batch_get_diag(self.h, C.byref(d)))
        return d.as_dict()

    def close(self):
        if self.h:
            lib().pic_batch_destroy(self.h)
            self.h = C.c_void_p()
            self.runs = []

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Server:
    """Continuous-batching request loop (pic_server_* calls)."""

    def __init__(self, device: int = 0, hbm_budget: int = 0, max_runs: int = 0,
                 steps_per_tick: int = 0, use_graph: bool = True, stream=None):
        cfg = pic_server_config(stream, device, int(hbm_budget), int(max_runs),
                                int(steps_per_tick), int(use_graph))
        self.h = C.c_void_p()
        rc = lib().pic_server_create(C.byref(cfg), C.byref(self.h))
        if rc != PIC_OK:
            raise PicError(rc, "pic_server_create failed")

    def pic_server_submit(self, cfg: pic_config, nsteps: int, keep: bool = False) -> int:
        rid = C.c_longlong()
        rc = lib().pic_server_submit(self.h, C.byref(cfg), int(nsteps), int(keep), C.byref(rid))
        if rc != PIC_OK:
            raise PicError(rc, "pic_server_submit rejected the request")
        return rid.value

    def pic_server_tick(self) -> int:
        running = C.c_int()
        rc = lib().pic_server_tick(self.h, C.byref(running))
        if rc != PIC_OK:
            raise PicError(rc, "pic_server_tick failed")
        return running.value

    def pic_server_info(self, rid: int) -> dict:
        info = pic_request_info()
        rc = lib().pic_server_info(self.h, int(rid), C.byref(info))
        if rc != PIC_OK:
            raise PicError(rc, "unknown request")
        return info.as_dict()

    def pic_server_take(self, rid: int, cfg: pic_config) -> "Pic":
        """The finished context of a kept request, wrapped as a Pic."""
        h = C.c_void_p()
        rc = lib().pic_server_take(self.h, int(rid), C.byref(h))
        if rc != PIC_OK:
            raise PicError(rc, "request not finished or not kept")
        return Pic.adopt(h, cfg)

    def pic_server_cancel(self, rid: int):
        rc = lib().pic_server_cancel(self.h, rid)
        if rc != PIC_OK:
            raise PicError(rc, "cannot cancel request %d" % rid)

    def pic_server_get_stats(self) -> dict:
        st = pic_server_stats()
        rc = lib().pic_server_get_stats(self.h, C.byref(st))
        if rc != PIC_OK:
            raise PicError(rc, "pic_server_get_stats failed")
        return st.as_dict()

    def pic_server_clock(self) -> float:
        return lib().pic_server_clock(self.h)

    def close(self):
        if self.h:
            lib().pic_server_destroy(self.h)
            self.h = C.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
