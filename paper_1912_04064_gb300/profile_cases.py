"""Small, fixed workloads for kernel profiling (ncu) of the 3D path.

Used by the commands recorded in the ncu summaries: `python -m
paper_1912_04064_gb300.profile_cases lwfa3d_small` runs the 3D3V
LWFA-shaped case at a quarter of config 3's transverse size (256 x 128 x
128 cells, 4.19 M electrons, 8 x 8 x 8 GPU patches, FP32) for 160 steps,
so that a capture holds a few GB of device memory.
"""
import sys

from . import pic
from . import workloads as W


def lwfa3d_small(steps=160):
    run = W.lwfa_3d(n=(256, 128, 128), waist=10.0, tau=10.0)
    g = pic.Pic(pic.config_from_run(run, "fp32", capacity_factor=2.0, patch=(8, 8, 8)))
    g.pic_load_plasma()
    g.pic_step(steps)
    d = g.pic_diag()
    print("np", d["np"], "U_E", d["U_E"], "step", d["step"])


if __name__ == "__main__":
    {"lwfa3d_small": lwfa3d_small}[sys.argv[1]](*[int(a) for a in sys.argv[2:]])
