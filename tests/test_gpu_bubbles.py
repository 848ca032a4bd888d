"""Per-bubble velocity and position (Sec. 4.3) from the library's device labelling
(tpflbm_bubbles) against the plain flood-fill reference (oracle/bubbles_ref.py) on the
oracle's fields of the same state (needs a GB300)."""
import math

import numpy as np
import pytest

from oracle.bubbles_ref import bubbles as ref_bubbles
from oracle.oracle import OracleSim
from paper_2306_11320_gb300 import workloads as WL

pytestmark = pytest.mark.gpu


def _regions(nx, ny, seed, n_max=24):
    """A phase field with several separate phi < 0 regions (a smoothed random field,
    kept at least 1e-3 away from zero so both sides take the same sign decisions),
    with the regions of the random-state workload's parameters."""
    rng = np.random.default_rng(seed)
    for _ in range(50):
        a = rng.normal(size=(ny, nx))
        k = np.ones(7) / 7.0
        for axis in (0, 1):
            a = np.apply_along_axis(lambda v: np.convolve(v, k, mode="same"), axis, a)
        phi = np.tanh(4.0 * (0.35 - a))  # phi < 0 above about 2.5 standard deviations
        phi = np.where(np.abs(phi) < 1e-3, np.sign(phi + 1e-12) * 1e-3, phi)
        z = np.zeros_like(phi)
        if 2 <= len(ref_bubbles(phi, z, z)) <= n_max:
            return phi
    raise AssertionError("no field with a few regions")


def _compare(gpu_b, ref_b, rel=1e-5, count_tol=0):
    assert len(gpu_b) == len(ref_b), (len(gpu_b), len(ref_b))
    scale_u = max(1e-12, max(abs(b[k]) for b in ref_b for k in ("u_b", "v_b")))
    for g, r in zip(gpu_b, ref_b):
        assert abs(g["nodes"] - r["nodes"]) <= count_tol, (g, r)
        assert g["sum_phi"] == pytest.approx(r["sum_phi"], rel=max(rel, 2.0 * count_tol / max(r["nodes"], 1.0)))
        for k in ("x_b", "y_b"):
            assert abs(g[k] - r[k]) < 1e-3, (k, g, r)
        for k in ("u_b", "v_b"):
            assert abs(g[k] - r[k]) <= 1e-3 * scale_u + rel * abs(r[k]), (k, g, r)


@pytest.mark.parametrize("bc_x,bc_y,seed", [(0, 1, 1), (0, 0, 2), (1, 0, 3)])
def test_labelling_matches_reference(bc_x, bc_y, seed):
    """Random multi-region states on fully periodic, walled and inlet/outflow lattices
    (regions wrap across periodic seams): node counts equal, moments within float32
    rounding, right after initialisation and after 50 steps."""
    from paper_2306_11320_gb300.tpflbm import Lattice

    nx, ny = 96, 64
    p, f, _ = WL.random_state(nx, ny, seed=seed, bc_x=bc_x, bc_y=bc_y)
    f["phi"] = _regions(nx, ny, seed)
    f32 = {k: np.asarray(v, dtype=np.float32) for k, v in f.items()}
    lat = Lattice(nx, ny, p)
    lat.init(**f32)
    o = OracleSim(nx, ny, p)
    o.init(**{k: v.astype(np.float64) for k, v in f32.items()})
    for steps in (0, 50):
        lat.step(steps)
        o.step(steps)
        fl = o.fields()
        ref = ref_bubbles(fl["phi"], fl["ux"], fl["uy"], periodic_x=bc_x == 0, periodic_y=bc_y == 1)
        # after steps, nodes whose phi is within float32 rounding of zero may flip
        _compare(lat.bubbles(), ref, rel=1e-5 if steps == 0 else 1e-3, count_tol=0 if steps == 0 else 2)


def test_seam_bubble_is_one():
    """A drop across the periodic x seam is one bubble with its centroid on the seam."""
    from paper_2306_11320_gb300.tpflbm import Lattice

    n, W = 64, 4.0
    y, x = np.mgrid[0:n, 0:n].astype(float)
    dx = np.minimum(x, n - x)
    phi = np.tanh((np.hypot(dx, y - 31.0) - 10.0) / (math.sqrt(2) * W))
    p = WL.base_params(bc_x=0, bc_y=1)
    z = np.zeros_like(phi, dtype=np.float32)
    lat = Lattice(n, n, p)
    lat.init(phi=phi.astype(np.float32), ux=z, uy=z, p=z, T=z)
    b = lat.bubbles()
    assert len(b) == 1
    assert min(b[0]["x_b"], n - b[0]["x_b"]) < 1e-4 and abs(b[0]["y_b"] - 31.0) < 1e-4


def test_too_many_regions_is_an_error():
    from paper_2306_11320_gb300.tpflbm import Lattice, TpfError

    n = 64
    y, x = np.mgrid[0:n, 0:n]
    phi = np.where((x % 4 == 1) & (y % 4 == 1), -1.0, 1.0).astype(np.float32)  # 256 single nodes
    z = np.zeros_like(phi)
    lat = Lattice(n, n, WL.base_params(bc_y=1))
    lat.init(phi=phi, ux=z, uy=z, p=z, T=z)
    with pytest.raises(TpfError):
        lat.bubbles()


@pytest.mark.parametrize("storage", [0, 1])
def test_recalcitrant_bubbles(storage):
    """The two-bubble channel of Sec. 4.3 (2048 x 512, parabolic sigma(T) with its minimum
    at mid-channel, Poiseuille inflow) over 400,000 steps.  The bubbles start as two
    separate regions at their placed centres.  The inflow first carries them downstream;
    once the walls' heat reaches them, the thermocapillary force towards T_ref (upstream)
    overcomes the drag and both move against the flow: u_b < 0 and x_b falling, the
    recalcitrant motion the paper reports (Figs. 10-11)."""
    from paper_2306_11320_gb300.tpflbm import Lattice

    p, f, m = WL.bubbles()
    if storage:
        p = dict(p, **WL.fp16_scales(p))
    lat = Lattice(2048, 512, p, storage=storage)
    lat.init(**{k: v.astype(np.float32) for k, v in f.items()})
    b0 = lat.bubbles()
    assert len(b0) == 2
    assert abs(b0[0]["x_b"] - m["x2"]) < 1e-3 and abs(b0[1]["x_b"] - m["x1"]) < 1e-3
    assert abs(b0[0]["y_b"] - m["yc"]) < 1e-3 and abs(b0[1]["y_b"] - m["yc"]) < 1e-3
    track = {}
    for t in range(50000, 400001, 50000):
        lat.step(t - lat.t)
        bs = lat.bubbles()
        assert len(bs) == 2 and lat.diagnostics()["nonfinite"] == 0
        track[t] = bs
    print("x_b", {t: [round(b["x_b"], 2) for b in bs] for t, bs in track.items()})
    print("u_b", {t: ["%.2e" % b["u_b"] for b in bs] for t, bs in track.items()})
    for k in range(2):
        # first carried downstream by the inflow ...
        assert track[50000][k]["x_b"] > b0[k]["x_b"] + 1.0 and track[50000][k]["u_b"] > 0
        # ... then moving upstream, against the flow
        assert all(track[t][k]["u_b"] < 0 for t in (300000, 350000, 400000)), k
        assert track[400000][k]["x_b"] < track[250000][k]["x_b"] - 2.0, k
