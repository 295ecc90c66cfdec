"""Helpers for the GPU parity tests: build contexts from oracle or library
hierarchies and run the oracle on the same seeded inputs."""
import numpy as np

import paper_2606_19251_gb300 as P
import workloads as W
from oracle import setup as OS
from oracle import solve as O


def ctx_from_oracle(levels, precision=P.AMG_FP64, **kw):
    """Context whose hierarchy is the oracle's (isolates the solve path)."""
    ctx = P.amg_create(precision=precision, **kw)
    P.amg_load_hierarchy(ctx, [l.A for l in levels], [l.P for l in levels[:-1]], [l.R for l in levels[:-1]])
    return ctx


def ctx_setup(A, precision=P.AMG_FP64, **kw):
    ctx = P.amg_create(precision=precision, **kw)
    P.amg_setup(ctx, A)
    return ctx


def oracle_hier(levels, smoother="jacobi", coeffs=None):
    h = O.OHierarchy.of(levels)
    if smoother == "jacobi":
        h.set_jacobi()
    else:
        h.set_pseudo_inverse(coeffs)
    return h


def rel_err(a, b):
    a, b = np.asarray(a), np.asarray(b)
    return float(np.abs(a - b).max() / max(np.abs(b).max(), 1e-300))


def library_levels(ctx):
    """The library's host hierarchy as workloads.CSR objects."""
    out = []
    nl = P.amg_num_levels(ctx)
    for l in range(nl):
        A, Pm = P.amg_get_level(ctx, l)
        a = W.CSR(A["n"], A["n"], A["row_ptr"], A["col"], A["val"])
        p = None if Pm is None else W.CSR(Pm["n"], Pm["nc"], Pm["row_ptr"], Pm["col"], Pm["val"])
        out.append((a, p))
    return out


CASES = {
    "c1_64": lambda: W.poisson5(64),
    "grid_33": lambda: W.poisson5(33),
    "uniform_3k": lambda: W.fv_mesh("uniform", 3000, 1)[0],
    "graded_5k": lambda: W.fv_mesh("graded", 5000, 2)[0],
    "band_4k": lambda: W.fv_mesh("band", 4000, 3, max_aspect=100.0)[0],
}
