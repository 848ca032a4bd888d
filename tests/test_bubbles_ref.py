"""Pins of the per-bubble reference (oracle/bubbles_ref.py, Sec. 4.3 u_b and x_b)."""
import math

import numpy as np
import pytest

from oracle.bubbles_ref import bubbles, label
from paper_2306_11320_gb300 import workloads as WL


def _blobs(nx, ny, seed):
    rng = np.random.default_rng(seed)
    a = rng.normal(size=(ny, nx))
    k = np.ones(5) / 5.0
    for axis in (0, 1):
        a = np.apply_along_axis(lambda v: np.convolve(v, k, mode="same"), axis, a)
    return 0.15 - a  # phi < 0 on about a quarter of the nodes, in many separate blobs


@pytest.mark.parametrize("seed", range(4))
def test_labels_match_scipy(seed):
    """Non-periodic lattices: the components equal scipy.ndimage.label's with the
    4-neighbour structure (same count, same node sets)."""
    ndimage = pytest.importorskip("scipy.ndimage")
    phi = _blobs(53, 37, seed)
    lab, firsts = label(phi)
    ref, n = ndimage.label(phi < 0)
    assert len(firsts) == n and n > 3
    for k in range(n):
        ks = np.unique(ref[lab == k])
        assert len(ks) == 1 and ks[0] > 0
        assert np.array_equal(lab == k, ref == ks[0])


def test_periodic_wrap_joins_regions():
    """A drop across the periodic x seam (and one across the y seam) is one bubble, whose
    centroid sits on the seam; without the wrap it splits in two."""
    n, R, W = 64, 10.0, 4.0
    y, x = np.mgrid[0:n, 0:n].astype(float)
    dx = np.minimum(np.abs(x - 0.0), n - np.abs(x - 0.0))  # centre at x = 0 (the seam)
    phi = np.tanh((np.hypot(dx, y - 31.0) - R) / (math.sqrt(2) * W))
    z = np.zeros_like(phi)
    b = bubbles(phi, z, z, periodic_x=True)
    assert len(b) == 1
    assert min(b[0]["x_b"], n - b[0]["x_b"]) < 1e-9 and abs(b[0]["y_b"] - 31.0) < 1e-9
    assert len(bubbles(phi, z, z, periodic_x=False)) == 2
    bt = bubbles(phi.T.copy(), z, z, periodic_y=True)
    assert len(bt) == 1 and min(bt[0]["y_b"], n - bt[0]["y_b"]) < 1e-9 and abs(bt[0]["x_b"] - 31.0) < 1e-9


def test_two_drops_closed_form():
    """Two separate tanh drops, each moving with its own uniform velocity: two bubbles,
    u_b and v_b equal those velocities (Sec. 4.3 formula with uniform u), x_b and y_b the
    drop centres (each drop is symmetric about its centre), node counts pi R^2 to within
    the boundary layer, ordered by x_b."""
    nx, ny, W = 200, 96, 4.0
    y, x = np.mgrid[0:ny, 0:nx].astype(float)
    c1, c2 = (140.0, 47.0), (55.0, 47.0)
    d1 = np.hypot(x - c1[0], y - c1[1]) - 20.0
    d2 = np.hypot(x - c2[0], y - c2[1]) - 14.0
    phi = np.tanh(np.minimum(d1, d2) / (math.sqrt(2) * W))
    ux = np.where(d1 < d2, 3e-4, -2e-4)
    uy = np.where(d1 < d2, 1e-4, 5e-5)
    b = bubbles(phi, ux, uy)
    assert len(b) == 2
    (lo, hi) = b
    assert abs(lo["x_b"] - c2[0]) < 1e-9 and abs(lo["y_b"] - c2[1]) < 1e-9
    assert abs(hi["x_b"] - c1[0]) < 1e-9 and abs(hi["y_b"] - c1[1]) < 1e-9
    assert lo["u_b"] == pytest.approx(-2e-4, rel=1e-12) and lo["v_b"] == pytest.approx(5e-5, rel=1e-12)
    assert hi["u_b"] == pytest.approx(3e-4, rel=1e-12) and hi["v_b"] == pytest.approx(1e-4, rel=1e-12)
    assert abs(hi["nodes"] - math.pi * 400) < 2 * math.pi * 20 and abs(lo["nodes"] - math.pi * 196) < 2 * math.pi * 14


def test_bubble_workload_has_two_bubbles():
    """The 2048 x 512 channel of Sec. 4.3 starts with its two bubbles at the placed centres."""
    p, f, m = WL.bubbles()
    z = np.zeros_like(f["phi"])
    b = bubbles(f["phi"], z, z)
    assert len(b) == 2
    assert abs(b[0]["x_b"] - m["x2"]) < 1e-6 and abs(b[1]["x_b"] - m["x1"]) < 1e-6
    assert abs(b[0]["y_b"] - m["yc"]) < 1e-6
