"""Initial fields through pic_init_fields (GPU) against the oracle.

The Poisson start solves Gauss's law div_h E = rho - <rho> on the periodic
Yee lattice (Section 2.1 initialises E consistently with the charge density
so that the Yee/Esirkepov scheme keeps Gauss's law for all later steps).
The GPU solves it spectrally in FP64 (cuFFT transforms, own scaling and
gradient kernels); the oracle with numpy's FFT from its own deposited rho.
Both are the same linear map up to rounding, so FP64 agrees to ~1e-13.
"""
import numpy as np
import pytest

from oracle.oracle import Oracle3, poisson_periodic, poisson_periodic3
from paper_1912_04064_gb300 import pic
from paper_1912_04064_gb300 import workloads as W

from parity_utils import field_errors, pair, rel_err

pytestmark = pytest.mark.gpu

TOL64 = 1e-12


@pytest.mark.parametrize("n,patch", [((64, 64), (16, 16)), ((96, 48), (32, 16))])
def test_poisson_start_2d_fp64(n, patch):
    run, parts = W.thermal_2d(n=n, patch=patch, seed=5)
    o, g = pair(run, parts, background=("uniform", 1.0))
    g.pic_init_fields("poisson")
    rho = o.field("rho") + 1.0
    Ex, Ey = poisson_periodic(rho, *run["d"])
    assert rel_err(g.pic_get_field("Ex"), Ex) <= TOL64
    assert rel_err(g.pic_get_field("Ey"), Ey) <= TOL64
    for k in ("Ez", "Bx", "By", "Bz", "Bmx", "Bmy", "Bmz"):
        assert not np.any(g.pic_get_field(k)), k
    scale = float(np.max(np.abs(rho)))
    assert g.pic_diag()["gauss"] < 1e-12 * scale
    # the run continues from the GPU-initialised state exactly as the oracle's
    for k, v in (("Ex", Ex), ("Ey", Ey)):
        o.set_field(k, v)
    o.step(5)
    g.pic_step(5)
    errs = field_errors(o, g)
    assert max(errs.values()) <= 1e-10, errs
    assert g.pic_diag()["gauss"] < 1e-10 * scale


def test_poisson_start_2d_fp32():
    run, parts = W.thermal_2d(n=(64, 64), patch=(16, 16), seed=6)
    o, g = pair(run, parts, prec="fp32", background=("uniform", 1.0))
    g.pic_init_fields("poisson")
    rho = o.field("rho") + 1.0
    Ex, Ey = poisson_periodic(rho, *run["d"])
    # FP32 positions and deposit (eps 6e-8 per term, 4 ppc per node) feed an
    # FP64 solve; the result is rounded to FP32 on the grid
    assert rel_err(g.pic_get_field("Ex"), Ex) <= 1e-5
    assert rel_err(g.pic_get_field("Ey"), Ey) <= 1e-5


def test_zero_start_clears_fields():
    run = W.periodic_run((64, 32), (0.1, 0.1), (16, 16))
    parts = W.small_random_particles(run, 5000, seed=7)
    fields = W.random_fields((32, 64), seed=8, amp=0.1)
    o, g = pair(run, parts, fields)
    g.pic_init_fields("zero")
    for k in ("Ex", "Ey", "Ez", "Bx", "By", "Bz", "Bmx", "Bmy", "Bmz"):
        assert not np.any(g.pic_get_field(k)), k
    # particles are untouched
    assert g.pic_diag()["np"] == 5000


def test_poisson_start_needs_periodic_fields():
    run, _ = W.lwfa_2d(n=(64, 32), d=(0.125, 0.5), patch=(16, 16), ppc=(1, 1), ramp=4.0)
    run["moving_window"] = None
    g = pic.Pic(pic.config_from_run(run, "fp64"))
    with pytest.raises(pic.PicError) as e:
        g.pic_init_fields("poisson")
    assert e.value.status == pic.PIC_EINVAL
    rc = pic.lib().pic_init_fields(g.h, 7)
    assert rc == pic.PIC_EINVAL


@pytest.mark.parametrize("prec,tol", [("fp64", TOL64), ("fp32", 1e-5)])
def test_poisson_start_3d(prec, tol):
    run = W.periodic_run3((16, 8, 12), (0.1, 0.12, 0.1), (4, 4, 4))
    parts = W.small_random_particles3(run, 8000, seed=41, uth=0.2)
    o = Oracle3(run, track_continuity=True)
    o.load(parts)
    g = pic.Pic(pic.config_from_run(run, prec))
    g.pic_load_particles(parts)
    # a uniform background (a node-wise neutralising one would leave no field)
    bg = -float(o.field("rho").mean())
    o.set_background("uniform", bg)
    g.pic_set_background("uniform", bg)
    g.pic_init_fields("poisson")
    rho = o.field("rho") + bg
    assert float(np.max(np.abs(rho))) > 0.1
    E = poisson_periodic3(rho, run["d"])
    for k, v in zip(("Ex", "Ey", "Ez"), E):
        assert rel_err(g.pic_get_field(k), v) <= tol, k
    if prec == "fp64":
        scale = float(np.max(np.abs(rho)))
        assert g.pic_diag()["gauss"] < 1e-12 * scale
        for k, v in zip(("Ex", "Ey", "Ez"), E):
            o.set_field(k, v)
        o.step(3)
        g.pic_step(3)
        for k in ("Ex", "Ey", "Ez", "Bx", "By", "Bz", "Jx", "Jy", "Jz"):
            assert rel_err(g.pic_get_field(k), o.field(k)) <= 1e-10, k
