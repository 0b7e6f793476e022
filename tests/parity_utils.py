"""Helpers of the GPU-vs-oracle parity tests (identical states on both sides).

Tolerance metric: ||a - b||_inf / ||b||_inf per field component; particles
are compared as sets (sorted by position), element by element.
"""
import numpy as np

from oracle.oracle import Oracle
from paper_1912_04064_gb300 import pic

FIELD_NAMES = ("Ex", "Ey", "Ez", "Bx", "By", "Bz", "Bmx", "Bmy", "Bmz", "Jx", "Jy", "Jz")


def pair(run, parts, fields=None, prec="fp64", background=None, **kw):
    """An oracle and a GPU context loaded with the same state."""
    o = Oracle(run, track_continuity=True)
    o.load(parts)
    g = pic.Pic(pic.config_from_run(run, prec, **kw))
    g.pic_load_particles(parts)
    if fields:
        for k, v in fields.items():
            o.set_field(k, v)
            g.pic_set_field(k, v)
    if background is not None:
        mode, val = background
        o.set_background(mode, val)
        g.pic_set_background(mode, val)
    return o, g


def rel_err(a, b):
    scale = np.max(np.abs(b))
    if scale == 0:
        return float(np.max(np.abs(a)))
    return float(np.max(np.abs(a - b)) / scale)


def field_errors(o, g, names=FIELD_NAMES):
    return {k: rel_err(g.pic_get_field(k), o.field(k)) for k in names}


def match_particles(a, b):
    """Pair every particle of `a` with its nearest particle of `b` in
    (x, y, ux, uy, uz, w) space; particles are unordered sets and regularly
    injected ones share exact positions, so sorting alone is ambiguous.
    Returns b re-ordered to match a; asserts the pairing is one-to-one."""
    from scipy.spatial import cKDTree

    keys = ("x", "y", "ux", "uy", "uz", "w")
    A = np.stack([a[k] for k in keys], 1)
    B = np.stack([b[k] for k in keys], 1)
    scale = np.maximum(np.max(np.abs(B), 0), 1e-30)
    _, idx = cKDTree(B / scale).query(A / scale, k=1)
    assert np.unique(idx).size == idx.size, "particle pairing is not one-to-one"
    return {k: b[k][idx] for k in keys}


def particle_errors(o, g):
    a, b = g.pic_get_particles(), o.particles()
    assert a["x"].size == b["x"].size, (a["x"].size, b["x"].size)
    if a["x"].size == 0:
        return {k: 0.0 for k in a}
    b = match_particles(a, b)
    out = {}
    for k in a:
        scale = max(np.max(np.abs(b[k])), 1e-300)
        out[k] = float(np.max(np.abs(a[k] - b[k])) / scale)
    return out
