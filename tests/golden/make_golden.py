"""Writes the oracle regression fixtures of tests/golden/ (run from the repo
root: python tests/golden/make_golden.py).  It calls only oracle/ and the
seeded input generators: the stored numbers are the oracle's own outputs
on small seeded cases, so they pin nothing about correctness (the pins in
test_oracle_pins.py and test_oracle3d_pins.py do that); they catch an
unintended change of the oracle's arithmetic.  A deliberate change
regenerates them, in a commit that names the passage of the paper (or the
reading of it) that justifies the change.
"""
import json
import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

from oracle.oracle import Oracle, Oracle3, poisson_periodic  # noqa: E402
from paper_1912_04064_gb300 import workloads as W  # noqa: E402

KEYS = ("U_E", "U_B", "U_K", "charge", "gauss", "np")
FIELDS2 = ("Ex", "Ey", "Ez", "Bx", "By", "Bz", "Jx", "Jy", "Jz")


def summary(o, names):
    d = o.diag()
    out = {k: float(d[k]) for k in KEYS}
    for k in names:
        a = o.field(k)
        out[k + ".sum"] = float(np.sum(a))
        out[k + ".sumsq"] = float(np.sum(a * a))
    return out


def thermal_2d():
    """32x32 periodic thermal plasma, 8x8 patches, 4 ppc, Poisson start on a
    uniform ion background, 20 steps."""
    run, parts = W.thermal_2d(n=(32, 32), patch=(8, 8), seed=3)
    o = Oracle(run, track_continuity=True)
    o.load(parts)
    o.set_background("uniform", 1.0)
    Ex, Ey = poisson_periodic(o.field("rho") + 1.0, *run["d"])
    o.set_field("Ex", Ex)
    o.set_field("Ey", Ey)
    rec = {}
    for n in (0, 10, 20):
        if n:
            o.step(10)
        rec[str(n)] = summary(o, FIELDS2)
    return rec


def lwfa_2d_window():
    """64x32 LWFA-shaped run (laser, open faces, removal and reflection, two
    window shifts, injection), 8x8 patches, 90 steps."""
    run, parts = W.lwfa_2d(n=(64, 32), d=(0.125, 0.5), patch=(8, 8), ppc=(2, 2), ramp=4.0,
                           a0=1.0, waist=4.0, tau=3.0, t_mw=2.0)
    o = Oracle(run)
    o.load(parts)
    o.set_background("neutralising")
    rec = {}
    for n in (30, 60, 90):
        o.step(30)
        rec[str(n)] = summary(o, FIELDS2)
        rec[str(n)]["shifts"] = int(o.diag()["shifts"])
    return rec


def periodic_3d():
    """16x8x8 periodic 3D3V run, 4x4x4 patches, 3000 random particles and
    random fields, 5 steps."""
    run = W.periodic_run3((16, 8, 8), (0.1, 0.1, 0.1), (4, 4, 4))
    parts = W.small_random_particles3(run, 3000, seed=5, uth=0.3)
    fields = W.random_fields(W.field_shape3(run), seed=6, amp=0.05)
    o = Oracle3(run, track_continuity=True)
    o.load(parts)
    for k, v in fields.items():
        o.set_field(k, v)
    o.step(5)
    return {"5": summary(o, FIELDS2)}


CASES = {"thermal_2d": thermal_2d, "lwfa_2d_window": lwfa_2d_window, "periodic_3d": periodic_3d}

if __name__ == "__main__":
    out = {name: f() for name, f in CASES.items()}
    with open(os.path.join(HERE, "oracle_regression.json"), "w") as fh:
        json.dump(out, fh, indent=1, sort_keys=True)
        fh.write("\n")
