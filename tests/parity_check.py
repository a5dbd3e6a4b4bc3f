"""Element-wise comparison of a CUDA result with the oracle's, with the
achieved errors recorded.

Each comparison asserts two bounds:
  relative L2      |out - ref|_2 / |ref|_2            <= l2
  element-wise     max_i |out_i - ref_i| / max|ref|   <= inf
so that a few wrong elements (a bad tile edge, a mis-indexed band) cannot hide
in the norm of a long vector.  When the environment variable BSE_PARITY_LOG
names a file, every comparison appends one JSON line with its name, the two
achieved errors and the bounds.

Bounds per arithmetic (H psi of one vector):
  fp64        1e-11 / 1e-11   rounding order only
  fp32        1e-5  / 3e-5    FP32 band<->grid sums over Nb and Nx terms
  split_bf16  1e-5  / 3e-5    three bf16 products (~2^-17 relative each) with
                              FP32 accumulation; bf16 hi/lo operands
"""
import json
import os

import numpy as np

TOL = {"fp64": (1e-11, 1e-11), "fp32": (1e-5, 3e-5), "split_bf16": (1e-5, 3e-5)}


def errors(out, ref):
    out = np.asarray(out)
    ref = np.asarray(ref)
    d = out - ref
    l2 = float(np.linalg.norm(d) / max(np.linalg.norm(ref), 1e-300))
    inf = float(np.abs(d).max() / max(np.abs(ref).max(), 1e-300)) if d.size else 0.0
    return l2, inf


def record(name, l2, inf, bounds):
    path = os.environ.get("BSE_PARITY_LOG")
    if not path:
        return
    with open(path, "a") as f:
        f.write(json.dumps({"name": name, "rel_l2": l2, "rel_inf": inf, "bound_l2": bounds[0],
                            "bound_inf": bounds[1]}) + "\n")


def close(name, out, ref, tol):
    """Assert both bounds; tol is a precision name or an (l2, inf) pair."""
    bounds = TOL[tol] if isinstance(tol, str) else tuple(tol)
    l2, inf = errors(out, ref)
    record(name, l2, inf, bounds)
    assert np.all(np.isfinite(np.asarray(out))), name
    assert l2 <= bounds[0] and inf <= bounds[1], "%s: rel L2 %.3e (bound %.1e), rel inf %.3e (bound %.1e)" % (
        name, l2, bounds[0], inf, bounds[1])
    return l2, inf
