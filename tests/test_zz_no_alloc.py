"""Allocation-free field energy (pic_field_energy_noalloc), through the C-ABI.

Callers that cannot let the library allocate device memory -- an application
that owns the device memory budget through its own allocator, or a serving
loop in which a device allocation would synchronise the device under live
requests -- use this entry point.  It must give the same field energies as the
context's own reduction (pic_diag), call after call: the second call uses a
smaller grid than the first, so rows left in the shared scratch array by the
first call must not leak into the second result.  The largest accepted grid
is checked against a host sum, and a call after the set-up is checked to
leave the device's free memory unchanged.

This file is collected last on purpose.
"""
import numpy as np
import pytest

from paper_1912_04064_gb300 import pic
from paper_1912_04064_gb300 import workloads as W

pytestmark = pytest.mark.gpu

NAMES = ("Ex", "Ey", "Ez", "Bmx", "Bmy", "Bmz")
MAX_ROWS = 65536  # PIC_NOALLOC_MAX_ROWS in include/pic.h


def _context_energy(n, d, seed):
    run = W.periodic_run(n, d, (16, 16))
    g = pic.Pic(pic.config_from_run(run, "fp64"))
    g.pic_load_particles(W.small_random_particles(run, 500, seed=seed))
    fields = W.random_fields((n[1], n[0]), seed=seed + 1, amp=0.3, names=NAMES)
    for k, v in fields.items():
        g.pic_set_field(k, v)
    diag = g.pic_diag()
    g.close()
    return fields, diag


def test_noalloc_energy_matches_context_reduction():
    import torch

    L = pic.lib()
    out = torch.zeros(2, dtype=torch.float64, device="cuda")
    cases = [((256, 192), (0.1, 0.07), 3), ((128, 64), (0.2, 0.1), 7)]
    for n, d, seed in cases:
        fields, diag = _context_energy(n, d, seed)
        dev = {k: torch.from_numpy(np.ascontiguousarray(v)).cuda() for k, v in fields.items()}
        out.fill_(-1.0)
        torch.cuda.synchronize()
        rc = L.pic_field_energy_noalloc(*[dev[k].data_ptr() for k in NAMES], n[0], n[1],
                                        d[0] * d[1], out.data_ptr(), None)
        assert rc == pic.PIC_OK
        torch.cuda.synchronize()
        ue, ub = out.tolist()
        assert abs(ue - diag["U_E"]) <= 1e-12 * diag["U_E"], (ue, diag["U_E"])
        assert abs(ub - diag["U_B"]) <= 1e-12 * diag["U_B"], (ub, diag["U_B"])
    # the largest accepted grid (ny = PIC_NOALLOC_MAX_ROWS rows) against a
    # float64 sum on the host
    rng = np.random.default_rng(11)
    big = {k: rng.standard_normal((MAX_ROWS, 4)) for k in NAMES}
    dbig = {k: torch.from_numpy(v).cuda() for k, v in big.items()}
    rc = L.pic_field_energy_noalloc(*[dbig[k].data_ptr() for k in NAMES], 4, MAX_ROWS, 0.5,
                                    out.data_ptr(), None)
    assert rc == pic.PIC_OK
    torch.cuda.synchronize()
    ue, ub = out.tolist()
    ref_e = 0.25 * sum(float(np.sum(big[k] ** 2)) for k in NAMES[:3])
    ref_b = 0.25 * sum(float(np.sum(big[k] ** 2)) for k in NAMES[3:])
    assert abs(ue - ref_e) <= 1e-12 * ref_e and abs(ub - ref_b) <= 1e-12 * ref_b
    # once set up on the device, a call allocates nothing: the device's free
    # memory and PyTorch's allocation counters are the same after it
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    alloc0 = torch.cuda.memory_allocated()
    rc = L.pic_field_energy_noalloc(*[dbig[k].data_ptr() for k in NAMES], 4, MAX_ROWS, 0.5,
                                    out.data_ptr(), None)
    assert rc == pic.PIC_OK
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    assert free1 == free0 and torch.cuda.memory_allocated() == alloc0
    assert out.tolist() == [ue, ub]  # and gives the same bits again
    # sizes beyond the scratch array are refused before any launch
    rc = L.pic_field_energy_noalloc(*[dev[k].data_ptr() for k in NAMES], 8, MAX_ROWS + 1, 1.0,
                                    out.data_ptr(), None)
    assert rc == pic.PIC_EINVAL
    rc = L.pic_field_energy_noalloc(None, None, None, None, None, None, 8, 8, 1.0,
                                    out.data_ptr(), None)
    assert rc == pic.PIC_EINVAL
