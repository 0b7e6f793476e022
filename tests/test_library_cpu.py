"""Host-side checks of libpic that need no GPU: the library builds, loads and
exports every entry point declared in include/pic.h; the ctypes mirrors of
the C structs have the C layout; configurations are validated before any
CUDA call; the HBM footprint used for admission is consistent."""
import ctypes as C
import os
import re
import subprocess

import pytest

from paper_1912_04064_gb300 import build as pic_build
from paper_1912_04064_gb300 import pic
from paper_1912_04064_gb300 import workloads as W

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "pic.h")


@pytest.fixture(scope="module")
def libpic():
    pic_build.build()
    return pic.lib()


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(pic_[a-z_]+)\s*\(", text)))


def test_exports_every_declared_symbol(libpic):
    names = declared_functions()
    assert len(names) >= 14
    out = subprocess.run(["nm", "-D", "--defined-only", pic.LIB_PATH], capture_output=True,
                         text=True, check=True).stdout
    exported = set(re.findall(r" T (pic_\w+)", out))
    missing = [n for n in names if n not in exported]
    assert not missing, missing
    for n in names:
        assert hasattr(libpic, n)
    assert set(pic.EXPORTS) <= exported


def test_struct_layout_matches_header(tmp_path):
    src = tmp_path / "layout.c"
    src.write_text(
        '#include <stdio.h>\n#include <stddef.h>\n#include "pic.h"\n'
        "int main(void){printf(\"%zu %zu %zu %zu %zu %zu %zu\\n\", sizeof(pic_config),"
        " sizeof(pic_diag_t), offsetof(pic_config, stream), offsetof(pic_config, block),"
        " offsetof(pic_config, inj_ppc), offsetof(pic_diag_t, ms_particles),"
        " offsetof(pic_diag_t, particle_step_launches));"
        "printf(\"%zu %zu %zu %zu\\n\", sizeof(pic_batch_config), offsetof(pic_batch_config, task_chunk),"
        " sizeof(pic_batch_diag_t), offsetof(pic_batch_diag_t, grid));"
        "printf(\"%zu %zu %zu %zu %zu %zu %zu %zu\\n\", sizeof(pic_tune_t), offsetof(pic_tune_t, candidates),"
        " sizeof(pic_server_config), offsetof(pic_server_config, use_graph),"
        " sizeof(pic_request_info), offsetof(pic_request_info, t_done),"
        " sizeof(pic_server_stats), offsetof(pic_server_stats, busy_s));"
        "printf(\"%zu %zu\\n\", offsetof(pic_config, current_float),"
        " offsetof(pic_config, staging_wait_polls));return 0;}\n")
    exe = tmp_path / "layout"
    subprocess.run(["gcc", "-I", os.path.dirname(HEADER), str(src), "-o", str(exe)], check=True)
    got = [int(v) for v in subprocess.run([str(exe)], capture_output=True, text=True,
                                          check=True).stdout.split()]
    want = [C.sizeof(pic.pic_config), C.sizeof(pic.pic_diag_t), pic.pic_config.stream.offset,
            pic.pic_config.block.offset, pic.pic_config.inj_ppc.offset,
            pic.pic_diag_t.ms_particles.offset, pic.pic_diag_t.particle_step_launches.offset,
            C.sizeof(pic.pic_batch_config), pic.pic_batch_config.task_chunk.offset,
            C.sizeof(pic.pic_batch_diag_t), pic.pic_batch_diag_t.grid.offset,
            C.sizeof(pic.pic_tune_t), pic.pic_tune_t.candidates.offset,
            C.sizeof(pic.pic_server_config), pic.pic_server_config.use_graph.offset,
            C.sizeof(pic.pic_request_info), pic.pic_request_info.t_done.offset,
            C.sizeof(pic.pic_server_stats), pic.pic_server_stats.busy_s.offset,
            pic.pic_config.current_float.offset, pic.pic_config.staging_wait_polls.offset]
    assert got == want


def test_version(libpic):
    assert "sm_103a" in pic.pic_version()


@pytest.mark.parametrize("mutate", [
    lambda c: setattr(c, "dims", 3),
    lambda c: c.patch.__setitem__(0, 30),
    lambda c: c.patch.__setitem__(1, 0),
    lambda c: c.n.__setitem__(0, 100),
    lambda c: setattr(c, "dt", 0.2),
    lambda c: setattr(c, "prec", 7),
    lambda c: c.bc_part[0].__setitem__(0, 0),     # periodic particles, open fields
    lambda c: setattr(c, "block", 100),
    lambda c: setattr(c, "m", 0.0),
    lambda c: setattr(c, "dev_alloc", 4096),       # allocator without its free
    lambda c: setattr(c, "dev_free", 4096),        # free without its allocator
    lambda c: setattr(c, "task_chunk", 8192),      # above the fixed-point tile's item bound
])
def test_invalid_configs_rejected_before_cuda(libpic, mutate):
    run, _ = W.lwfa_2d(n=(256, 128), patch=(32, 32))
    cfg = pic.config_from_run(run, "fp32")
    mutate(cfg)
    h = C.c_void_p()
    assert libpic.pic_create(C.byref(cfg), C.byref(h)) == pic.PIC_EINVAL
    assert not h.value
    assert pic.pic_footprint(cfg, 1000) == 0


@pytest.mark.parametrize("mutate", [
    lambda c: c.patch.__setitem__(2, 64),            # 3D patches up to 32
    lambda c: setattr(c, "filter_passes", 1),        # the filter is 2D only
    lambda c: setattr(c, "dt", 0.3),                 # 3D Courant condition
    lambda c: c.n.__setitem__(2, 4),                 # periodic axis below 8 cells
    lambda c: setattr(c, "dims", 4),
])
def test_invalid_3d_configs_rejected_before_cuda(libpic, mutate):
    run = W.periodic_run3((32, 16, 16), (0.1, 0.1, 0.1), (8, 8, 8))
    cfg = pic.config_from_run(run, "fp64")
    assert pic.pic_footprint(cfg, 1000) > 0
    if mutate is not None:
        mutate(cfg)
        if cfg.n[2] == 4:
            cfg.patch[2] = 4
    h = C.c_void_p()
    assert libpic.pic_create(C.byref(cfg), C.byref(h)) == pic.PIC_EINVAL
    assert not h.value


def test_footprint_3d_counts_26_buckets(libpic):
    """The config-3 grid: footprint grows with the particle count and the
    precision, and fits the device (the FP32 run with capacity factor 2)."""
    run = W.lwfa_3d()
    f32 = pic.pic_footprint(pic.config_from_run(run, "fp32", capacity_factor=2.0), 1 << 26)
    f64 = pic.pic_footprint(pic.config_from_run(run, "fp64", capacity_factor=2.0), 1 << 26)
    assert 0 < f32 < f64 < 2 * f32 + 1
    assert f32 < 100e9


def test_laser_and_window_need_open_x(libpic):
    run = W.periodic_run((64, 64), (0.1, 0.1), (16, 16))
    cfg = pic.config_from_run(run, "fp64")
    cfg.laser_on = 1
    cfg.laser_waist, cfg.laser_tau = 5.0, 5.0
    h = C.c_void_p()
    assert libpic.pic_create(C.byref(cfg), C.byref(h)) == pic.PIC_EINVAL
    cfg.laser_on = 0
    cfg.moving_window = 1
    assert libpic.pic_create(C.byref(cfg), C.byref(h)) == pic.PIC_EINVAL


def test_footprint_scales_with_precision_and_particles(libpic):
    run, parts = W.lwfa_2d()
    n = parts["x"].size
    f32 = pic.pic_footprint(pic.config_from_run(run, "fp32"), n)
    f64 = pic.pic_footprint(pic.config_from_run(run, "fp64"), n)
    assert 1.8 < f64 / f32 < 2.2
    # the fullest patch is at least one injected column's worth with the
    # moving window; without it the footprint follows the particle count
    still = dict(run, moving_window=None)
    assert pic.pic_footprint(pic.config_from_run(still, "fp32"), n // 8) < f32
    assert pic.pic_footprint(pic.config_from_run(run, "fp32"), n // 8) == f32
    # particle storage dominates: ping-pong segments + buckets, 6 arrays
    assert f32 > 2 * 6 * 4 * n


def test_null_arguments(libpic):
    assert libpic.pic_create(None, None) == pic.PIC_EINVAL
    assert libpic.pic_step(None, 1) == pic.PIC_EINVAL
    assert libpic.pic_sync(None) == pic.PIC_EINVAL
    assert b"no context" in libpic.pic_last_error(None)
    libpic.pic_destroy(None)
    assert libpic.pic_batch_create(None, None) == pic.PIC_EINVAL
    assert libpic.pic_batch_set(None, None, 0) == pic.PIC_EINVAL
    assert libpic.pic_batch_step(None, 1) == pic.PIC_EINVAL
    assert libpic.pic_batch_size(None) == 0
    assert libpic.pic_batch_get_diag(None, None) == pic.PIC_EINVAL
    assert b"no batch" in libpic.pic_batch_last_error(None)
    libpic.pic_batch_destroy(None)
    assert libpic.pic_load_plasma(None) == pic.PIC_EINVAL
    assert libpic.pic_init_fields(None, 1) == pic.PIC_EINVAL
    assert libpic.pic_autotune_plasma(None, 2, None, None) == pic.PIC_EINVAL
    assert libpic.pic_autotune(None, None, None, None, None, None, None, 0, 0, 1, None,
                               None) == pic.PIC_EINVAL
    libpic.pic_autotune_clear_cache()
    assert libpic.pic_server_create(None, None) == pic.PIC_EINVAL
    assert libpic.pic_server_submit(None, None, 1, 0, None) == pic.PIC_EINVAL
    assert libpic.pic_server_tick(None, None) == pic.PIC_EINVAL
    assert libpic.pic_server_info(None, 1, None) == pic.PIC_EINVAL
    assert libpic.pic_server_take(None, 1, None) == pic.PIC_EINVAL
    assert libpic.pic_server_get_stats(None, None) == pic.PIC_EINVAL
    assert libpic.pic_server_clock(None) == 0.0
    libpic.pic_server_destroy(None)


def test_create_without_gpu_fails_loudly(libpic):
    """On a machine without a CUDA device the library reports an error; it
    never falls back to a CPU path."""
    try:
        import torch
        has_gpu = torch.cuda.is_available()
    except Exception:
        has_gpu = False
    if has_gpu:
        pytest.skip("a GPU is present")
    run = W.periodic_run((64, 64), (0.1, 0.1), (16, 16))
    with pytest.raises(pic.PicError) as e:
        pic.Pic(pic.config_from_run(run, "fp64"))
    assert e.value.status == pic.PIC_ECUDA
    for make in (pic.Batch, pic.Server):
        with pytest.raises(pic.PicError) as e:
            make()
        assert e.value.status == pic.PIC_ECUDA
