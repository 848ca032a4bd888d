"""Pins of the local interface-normal variant (Sec. 3: the normal of the Allen-Cahn
source recovered from the populations' first non-equilibrium moment instead of the
stencil gradient of phi), in the FP64 oracle (CPU)."""
import numpy as np

from oracle.oracle import OracleSim
from paper_2306_11320_gb300 import workloads as WL


def _drop():
    n, R, W = 80, 16.0, 4.0
    p, f, _ = WL.static_drop(n=n, R=R, sigma=1e-3, mu=0.3, W=W)
    return n, R, W, p, f


def test_local_normal_equals_stencil_normal_on_a_relaxed_drop():
    """On the same relaxed state both laws give the same unit normal in the interface
    band |phi| < 0.95 (Chapman-Enskog: J = -cs2 tau grad phi + M Theta n is parallel to
    grad phi), to a fraction of a degree."""
    n, R, W, p, f = _drop()
    a = OracleSim(n, n, p)
    a.init(**f)
    a.step(2000)
    b = OracleSim(n, n, dict(p, normal_law=1))
    b.init(**f)
    b.set_state(a.get_state())
    A, B = a.aux(), b.aux()
    band = np.abs(a.fields()["phi"]) < 0.95
    cos = A["nx"] * B["nx"] + A["ny"] * B["ny"]
    assert band.sum() > 1000
    assert cos[band].min() > 1 - 1e-6


def test_laplace_law_with_local_normal():
    """Static drop: p_in - p_out = sigma / R within the same 4% as the stencil law."""
    n, R, W, p, f = _drop()
    s = OracleSim(n, n, dict(p, normal_law=1))
    s.init(**f)
    s.step(4000)
    fl = s.fields()
    y, x = np.mgrid[0:n, 0:n]
    c = 0.5 * (n - 1)
    r = np.hypot(x - c, y - c)
    row = fl["phi"][n // 2 - 1:n // 2 + 1].mean(axis=0)
    xs = np.arange(n) - c
    R0 = float(np.interp(0.0, row[xs > 0], xs[xs > 0]))
    dp = fl["p"][r < R0 - 2 * W].mean() - fl["p"][r > R0 + 2 * W].mean()
    assert abs(dp * R0 / 1e-3 - 1.0) < 0.04
