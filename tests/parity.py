"""Field comparisons of the GPU parity tests (no method arithmetic).

Two measures per field group (phi, Pi, theta, E) between a float32 engine state
and the FP64 oracle's state after the same steps from the same float32 start:

* ``field_errors``: relative L2 error of the whole group;
* ``site_errors``: the largest error at any single site and component, divided by
  the group's RMS over the lattice, so one wrong site shows at full size however
  many sites there are.

theta enters through the link variable exp(-i theta) (theta is defined modulo
2 pi and carries the float32 rounding of its own magnitude); its scale is the RMS
of theta, floored at 1e-3 rad for the nearly zero link angles of a random-phase
start.
"""
import math

import numpy as np

GROUPS = {"phi": slice(0, 2), "Pi": slice(2, 4), "theta": slice(4, 7), "E": slice(7, 10)}
THETA_FLOOR = 1e-3


def rel(a, b):
    return np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-30)


def rms(a):
    return math.sqrt(float(np.mean(np.square(a)))) if a.size else 0.0


def field_errors(got, ref):
    th = GROUPS["theta"]
    return {
        "phi": rel(got[GROUPS["phi"]], ref[GROUPS["phi"]]),
        "Pi": rel(got[GROUPS["Pi"]], ref[GROUPS["Pi"]]),
        "theta": np.linalg.norm(np.exp(-1j * got[th]) - np.exp(-1j * ref[th]))
        / max(np.linalg.norm(ref[th]), THETA_FLOOR * math.sqrt(ref[th].size)),
        "E": rel(got[GROUPS["E"]], ref[GROUPS["E"]]),
    }


def site_errors(got, ref):
    out = {}
    for name, sl in GROUPS.items():
        g, r = got[sl], ref[sl]
        if name == "theta":
            diff = np.abs(np.exp(-1j * g) - np.exp(-1j * r))
            scale = max(rms(r), THETA_FLOOR)
        else:
            diff = np.abs(g - r)
            scale = max(rms(r), 1e-30)
        out[name] = float(diff.max()) / scale if diff.size else 0.0
    return out


def worst_site(got, ref, name):
    """(plane, z, y, x) of the largest error of one group, for failure messages."""
    sl = GROUPS[name]
    g, r = got[sl], ref[sl]
    diff = np.abs(np.exp(-1j * g) - np.exp(-1j * r)) if name == "theta" else np.abs(g - r)
    idx = np.unravel_index(int(np.argmax(diff)), diff.shape)
    return (idx[0] + sl.start,) + tuple(int(v) for v in idx[1:])
