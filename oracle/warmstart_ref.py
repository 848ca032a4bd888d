"""FP64 numpy definition of the warm start's phase-field projection (test
infrastructure; only tests, the smoke check and the benchmark's CPU baseline use
this package).

The paper has no warm start.  Its equilibrium interface profile is
phi(d) = tanh(d / (sqrt(2) W)) (Sec. 2, with d the signed distance, heavy fluid
phi = +1); the projection rebuilds that profile from a predicted field and shifts it
so that sum phi equals a target (the Allen-Cahn LBE conserves sum phi, Eq. 7):

  contour: d(x, y) = y_c(x) + s - y, y_c(x) the lowest height at which the predicted
           field changes sign from positive to non-positive going up column x (linear
           interpolation between nodes y = j and j + 1; a column without a sign
           change uses its node of least |phi|);
  atanh:   d / (sqrt(2) W) = atanh(clip(phi, -(1 - 1e-7), 1 - 1e-7)) + s.

s is found by bisection (sum tanh(.) is increasing in s) to 1e-12 per node.
"""
from __future__ import annotations

import numpy as np

CLIP = 1.0 - 1e-7


def contour_heights(phi):
    """y_c(x) of a (ny, nx) field, as defined above."""
    ny, nx = phi.shape
    yc = np.empty(nx)
    for x in range(nx):
        col = phi[:, x]
        found = False
        for j in range(ny - 1):
            if col[j] > 0 and col[j + 1] <= 0:
                yc[x] = j + col[j] / (col[j] - col[j + 1])
                found = True
                break
        if not found:
            yc[x] = float(np.argmin(np.abs(col[:ny - 1])))
    return yc


def scaled_distance(phi, W, mode):
    """a = d / (sqrt(2) W) of every node before the offset."""
    phi = np.asarray(phi, dtype=np.float64)
    if mode == "atanh":
        return np.arctanh(np.clip(phi, -CLIP, CLIP))
    ny, nx = phi.shape
    y = np.arange(ny, dtype=np.float64)[:, None]
    return (contour_heights(phi)[None, :] - y) / (np.sqrt(2.0) * W)


def project_phi(phi, W, target_sum, mode="contour"):
    """(projected phi, offset s, achieved sum) with sum tanh(a + s) = target_sum."""
    a = scaled_distance(phi, W, mode)
    n = a.size
    if not abs(target_sum) < n:
        raise ValueError("target sum must lie strictly inside (-N, N)")
    lo, hi = -1.0, 1.0
    while np.tanh(a + lo).sum() > target_sum:
        lo *= 2.0
    while np.tanh(a + hi).sum() < target_sum:
        hi *= 2.0
    for _ in range(200):
        mid = 0.5 * (lo + hi)
        s_mid = np.tanh(a + mid).sum()
        if abs(s_mid - target_sum) <= 1e-12 * n:
            lo = hi = mid
            break
        if s_mid > target_sum:
            hi = mid
        else:
            lo = mid
    s = 0.5 * (lo + hi)
    out = np.tanh(a + s)
    return out, s, float(out.sum())


def forced_init_state(nx, ny, params, fields):
    """Populations of the half-source initialisation, from the FP64 oracle's own parts:
    its equilibrium populations of the given fields, minus half of its Allen-Cahn
    interface source R_i (d_t(phi u) = 0) and half of its NS forcing G_i, both with the
    interface normal, density gradient and interfacial force of its macroscopic pass on
    those fields (Eq. 11, Eq. 14, Sec. 3.1).  Returns the state dict of OracleSim."""
    from .oracle import OracleSim, node_ops

    o = OracleSim(nx, ny, params)
    o.init(**{k: np.asarray(v, dtype=np.float64) for k, v in fields.items()})
    st = o.get_state()
    a = o.aux()
    phi = np.asarray(fields["phi"], dtype=np.float64)
    ux = np.asarray(fields["ux"], dtype=np.float64)
    uy = np.asarray(fields["uy"], dtype=np.float64)
    for y in range(ny):
        for x in range(nx):
            R = node_ops.Ri(phi[y, x], 0.0, 0.0, a["nx"][y, x], a["ny"][y, x], params["W"])
            G = node_ops.Gi(ux[y, x], uy[y, x], a["grx"][y, x], a["gry"][y, x], a["Fx"][y, x], a["Fy"][y, x])
            st["f"][:, y, x] -= 0.5 * R
            st["g"][:, y, x] -= 0.5 * G
    return st
