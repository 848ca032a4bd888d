"""Physics of the GPU path on the workloads' own sizes (needs a GB300).

* Drop migration (Sec. 4.2): at Ma = Re = 0.1 the drop's migration velocity U_r
  (FP64 device reduction, Sec. 4.2 definition) approaches the Young-Goldstein-Block
  speed of Eq. 60.  The lattice is periodic in x (an array of drops 8 R apart) and
  walled 16 R above and below, so the confined drop moves somewhat slower than the
  unbounded theory; the paper's own errors at finite density ratio are 2-4%.
* Mass: sum phi drifts by less than 2e-5 relative over 40k float32 steps.
"""
import numpy as np
import pytest

from paper_2306_11320_gb300 import workloads as WL

pytestmark = pytest.mark.gpu


def _lat(nx, ny, params, fields, **kw):
    from paper_2306_11320_gb300.tpflbm import Lattice

    lat = Lattice(nx, ny, params, **kw)
    lat.init(**{k: v.astype(np.float32) for k, v in fields.items()})
    return lat


@pytest.mark.parametrize("storage", [0, 1])
def test_drop_migration_speed(storage):
    p, f, m = WL.drop_migration(Ma=0.1)
    if storage == 1:
        p.update(WL.fp16_scales(p))
    lat = _lat(256, 1024, p, f, storage=storage)
    d0 = lat.diagnostics()
    speeds = []
    for _ in range(8):
        lat.step(5000)
        d = lat.diagnostics()
        assert d["nonfinite"] == 0
        speeds.append(d["Ur_num"] / d["Ur_den"])
    ratio = speeds[-1] / m["U_ygb"]
    print("storage", storage, "U_r/U_YGB over time:", ["%.3f" % (s / m["U_ygb"]) for s in speeds])
    # terminal: the last two samples agree within 2%, and the speed is within 15% of Eq. 60
    assert abs(speeds[-1] - speeds[-2]) < 0.02 * abs(speeds[-1])
    assert 0.85 < ratio < 1.15, ratio
    # the drop moves towards the hot wall (up the temperature gradient)
    assert speeds[-1] > 0
    if storage == 0:
        # float32 rounding of the collision sums drifts sum phi by about 1e-10 per
        # node and step (4.4e-6 relative after these 40k steps)
        assert abs(d["sum_phi"] - d0["sum_phi"]) < 2e-5 * np.abs(f["phi"]).sum()


def test_marangoni_number_trend():
    """Sec. 4.2, finite Ma: at Ma = 10 the terminal migration speed is lower than at
    Ma = 0.1 (convection of heat weakens the surface temperature gradient)."""
    out = {}
    for Ma in (0.1, 10.0):
        p, f, m = WL.drop_migration(Ma=Ma)
        lat = _lat(256, 1024, p, f)
        lat.step(40000)
        d = lat.diagnostics()
        out[Ma] = d["Ur_num"] / d["Ur_den"] / m["U_ygb"]
    print("U_r / U_YGB:", out)
    assert out[10.0] < out[0.1]


def test_finite_marangoni_sweep_at_re_1():
    """Sec. 4.2 at finite Marangoni number: Re = 1, Ma = 1, 10, 100 set through c_p with
    the conductivity fixed, equal property ratios.  The paper reports that (i) early on
    the drop speeds up alike for every Ma, (ii) Ma = 1 settles without overshoot while
    Ma >= 10 first overshoots and then slows to its terminal speed, and (iii) the
    terminal speed decreases with Ma.  Terminal: the mean over t U/R in [30, 46], where
    every case has settled (the Ma = 100 temperature field needs about 30 R/U); later
    the drop feels the hot wall of this 1024-high channel (beyond about 60 R/U)."""
    hist = {}
    for Ma in (1.0, 10.0, 100.0):
        p, f, m = WL.drop_migration(Ma=Ma, Re=1.0, ratio=1.0)
        lat = _lat(256, 1024, p, f)
        us = []
        for _ in range(92):
            lat.step(2560)
            d = lat.diagnostics()
            assert d["nonfinite"] == 0
            us.append(d["Ur_num"] / d["Ur_den"] / m["U_ygb"])
        hist[Ma] = np.array(us)
    t = 2560 * np.arange(1, 93) / (m["R"] / m["U"])      # R / U = 5120 steps at Re = 1
    win = (t >= 30) & (t <= 46)
    term = {Ma: u[win].mean() for Ma, u in hist.items()}
    for Ma, u in hist.items():
        print("Ma %g: U_r/U_YGB at t U/R = 0.5, 1, 2, 4, 8, 16, 32:" % Ma,
              ["%.3f" % u[np.argmin(np.abs(t - s))] for s in (0.5, 1, 2, 4, 8, 16, 32)],
              "peak %.3f at %.1f, terminal %.3f" % (u.max(), t[u.argmax()], term[Ma]))
        assert np.ptp(u[win]) < 0.04 * term[Ma], (Ma, np.ptp(u[win]) / term[Ma])  # settled
    for s in (0.5, 1.0):
        early = [u[np.argmin(np.abs(t - s))] for u in hist.values()]
        assert np.ptp(early) < 0.02 * max(early)                              # (i)
    assert hist[1.0].max() < 1.01 * term[1.0]                                # (ii) Ma = 1 settles from below
    for Ma in (10.0, 100.0):
        assert hist[Ma].max() > 1.03 * term[Ma], (Ma, hist[Ma].max(), term[Ma])  # (ii) overshoot
    assert term[1.0] > term[10.0] > term[100.0] > 0                          # (iii)


def test_density_ratio_drops_table2():
    """Table 2 (Sec. 4.2): the drop at density ratios 10, 100, 500, 1000 (workload
    drop_density_ratio, on the paper's 160 x 320 lattice) runs stably with this
    pressure-based NS LBE and reaches a steady terminal speed.  Measured 0.896, 0.865,
    0.856, 0.854 U_YGB, below the paper's 0.958-0.977: the printed inputs are not
    consistent with each other (the reading that reproduces the U_YGB column is used),
    and the speed depends on the confinement (0.925 at rho_r = 10 with the periodic
    spacing widened to 16 R), so the bound here is loose."""
    import json
    import os

    g = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "paper_values.json")))["table2_U_r"]
    got = {}
    for rho_r, U_paper in zip(g["rho_r"], g["U_r"]):
        p, f, m = WL.drop_density_ratio(rho_r)
        lat = _lat(160, 320, p, f)
        us = []
        for _ in range(16):
            lat.step(10000)
            d = lat.diagnostics()
            assert d["nonfinite"] == 0, rho_r
            us.append(d["Ur_num"] / d["Ur_den"])
        got[rho_r] = (us[-1], m["U_ygb"], U_paper)
        print("rho_r %g: U_r/U_YGB every 10k steps:" % rho_r, ["%.4f" % (u / m["U_ygb"]) for u in us],
              "paper %.4f" % (U_paper / m["U_ygb"]))
        assert abs(us[-1] - us[-2]) < 0.01 * abs(us[-1])
    for rho_r, (u, ygb, up) in got.items():
        assert 0.8 < u / ygb < 1.05, (rho_r, u / ygb)
