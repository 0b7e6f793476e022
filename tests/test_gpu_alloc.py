"""Contexts whose device memory comes from the caller's allocator
(pic_config.dev_alloc / dev_free), here PyTorch's caching allocator: the
results equal those of a context on cudaMalloc and of the oracle, every
allocation is given back by pic_destroy, and an allocator that fails makes
the call fail with PIC_ENOMEM."""
import ctypes as C

import numpy as np
import pytest

from oracle.oracle import Oracle
from paper_1912_04064_gb300 import pic
from paper_1912_04064_gb300 import workloads as W

from parity_utils import field_errors, pair, rel_err

pytestmark = pytest.mark.gpu


class Counting:
    """torch_allocator() wrapped to count live allocations and bytes."""

    def __init__(self, fail_after=None):
        import torch
        self.torch = torch
        self.live = {}
        self.calls = 0
        self.fail_after = fail_after

        def alloc(nbytes, _user):
            self.calls += 1
            if self.fail_after is not None and self.calls > self.fail_after:
                return None
            p = torch.cuda.caching_allocator_alloc(int(nbytes), 0)
            self.live[p] = int(nbytes)
            return p

        def free(ptr, _user):
            assert ptr in self.live, "freed a pointer that was not allocated here"
            del self.live[ptr]
            torch.cuda.caching_allocator_delete(ptr)

        self.pair = (pic.DEV_ALLOC(alloc), pic.DEV_FREE(free))


def test_2d_context_on_caller_allocator_matches_oracle_and_frees_all():
    import torch
    base = torch.cuda.memory_allocated(0)
    run = W.periodic_run((64, 64), (0.1, 0.1), (16, 16))
    parts = W.small_random_particles(run, 20000, seed=11, uth=0.5)
    fields = W.random_fields((64, 64), seed=12, amp=0.1)
    o, ref = pair(run, parts, fields)
    cnt = Counting()
    g = pic.Pic(pic.config_from_run(run, "fp64", auto_grow=True), allocator=cnt.pair)
    g.pic_load_particles(parts)
    for k, v in fields.items():
        g.pic_set_field(k, v)
    assert cnt.live and torch.cuda.memory_allocated(0) > base
    o.step(3)
    ref.pic_step(3)
    g.pic_step(3)
    errs = field_errors(o, g)
    assert max(errs.values()) <= 1e-12, errs
    for k in ("Ex", "Bz", "Jx"):
        assert rel_err(g.pic_get_field(k), ref.pic_get_field(k)) <= 1e-13
    g.pic_snapshot()
    g.close()
    ref.close()
    assert not cnt.live, f"{len(cnt.live)} allocations not given back"
    assert torch.cuda.memory_allocated(0) == base


def test_3d_context_and_poisson_start_on_caller_allocator():
    import torch
    base = torch.cuda.memory_allocated(0)
    run = W.periodic_run3((16, 8, 16), (0.1, 0.1, 0.1), (4, 4, 4))
    parts = W.small_random_particles3(run, 5000, seed=3, uth=0.2)
    cnt = Counting()
    g = pic.Pic(pic.config_from_run(run, "fp64"), allocator=cnt.pair)
    g.pic_load_particles(parts)
    rho0 = g.pic_get_field("rho")
    g.pic_set_background("uniform", -float(rho0.mean()))
    n_before = cnt.calls
    g.pic_init_fields("poisson")
    assert cnt.calls > n_before  # scratch and FFT work area
    g.pic_step(2)
    assert g.pic_diag()["gauss"] < 1e-11 * float(np.max(np.abs(rho0)))
    g.close()
    assert not cnt.live
    assert torch.cuda.memory_allocated(0) == base


def test_failing_allocator_gives_enomem():
    run = W.periodic_run((64, 64), (0.1, 0.1), (16, 16))
    cnt = Counting(fail_after=2)
    cfg = pic.config_from_run(run, "fp64")
    cfg.dev_alloc = C.cast(cnt.pair[0], C.c_void_p)
    cfg.dev_free = C.cast(cnt.pair[1], C.c_void_p)
    h = C.c_void_p()
    assert pic.lib().pic_create(C.byref(cfg), C.byref(h)) == pic.PIC_ENOMEM
    assert not h.value
    assert not cnt.live  # what was taken before the failure is given back
