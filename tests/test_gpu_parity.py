"""GPU path vs the FP64 oracle, through the C-ABI (needs a GB300 and the built library).

FP32 tolerance: relative L2 error <= 1e-5 per field (phi, u_x, u_y, p, T), the
bound the design targets for FP32 populations.  Single-step population parity is
checked element by element against the population scale: the FP32 step rounds
each of the ~500 operations per node to 2^-24 relative, so 2e-6 of the largest
population magnitude bounds a one-step difference.
"""
import numpy as np
import pytest

from oracle.oracle import OracleSim
from paper_2306_11320_gb300 import workloads as WL

pytestmark = pytest.mark.gpu

FIELDS = ("phi", "ux", "uy", "p", "T")


def _lattice(nx, ny, params, **kw):
    from paper_2306_11320_gb300.tpflbm import Lattice

    return Lattice(nx, ny, params, **kw)


def rel_l2(a, b):
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    den = np.sqrt((b ** 2).sum())
    return float(np.sqrt(((a - b) ** 2).sum()) / den) if den > 0 else float(np.abs(a - b).max())


def _check_fields(a, b, tol):
    errs = {k: rel_l2(a[k], b[k]) for k in FIELDS}
    assert max(errs.values()) <= tol, errs


def _pair(nx, ny, params, fields, **kw):
    f32 = {k: np.asarray(v, dtype=np.float32) for k, v in fields.items()}
    gpu = _lattice(nx, ny, params, **kw)
    gpu.init(**f32)
    orc = OracleSim(nx, ny, params)
    orc.init(**{k: v.astype(np.float64) for k, v in f32.items()})
    return gpu, orc


CASES = [
    # nx, ny, bc_x, bc_y, sigma_law : ragged tiles, a lattice thinner than one tile,
    # periodic / walled / inlet-outflow, linear and parabolic sigma(T)
    (37, 23, 0, 0, 0),
    (37, 23, 0, 1, 1),
    (41, 19, 1, 0, 1),
    (8, 8, 0, 1, 0),
    (70, 4, 0, 0, 0),
    (33, 9, 1, 0, 0),
]


@pytest.mark.parametrize("nx,ny,bc_x,bc_y,law", CASES)
def test_one_step_populations(nx, ny, bc_x, bc_y, law):
    """One fused step: every population of f, g, h and (phi u) element by element."""
    p, f, _ = WL.random_state(nx, ny, seed=nx * 7 + ny, bc_x=bc_x, bc_y=bc_y, sigma_law=law)
    gpu, orc = _pair(nx, ny, p, f)
    a0, b0 = gpu.get_state(), orc.get_state()
    for k in ("f", "g", "h"):
        assert np.abs(a0[k] - b0[k]).max() <= 1e-6 * max(1.0, np.abs(b0[k]).max()), k
    gpu.step(1)
    orc.step(1)
    a, b = gpu.get_state(), orc.get_state()
    for k in ("f", "g", "h", "phiu"):
        scale = max(np.abs(b[k]).max(), 1e-30)
        err = np.abs(a[k] - b[k]).max() / scale
        assert err <= 2e-6, (k, err)


@pytest.mark.parametrize("nx,ny,bc_x,bc_y,law", CASES)
def test_fields_after_steps(nx, ny, bc_x, bc_y, law):
    """60 steps from a random two-phase state; fields within rel-L2 1e-5."""
    p, f, _ = WL.random_state(nx, ny, seed=3 * nx + ny, bc_x=bc_x, bc_y=bc_y, sigma_law=law)
    gpu, orc = _pair(nx, ny, p, f)
    gpu.step(60)
    orc.step(60)
    a, b = gpu.fields(), orc.fields()
    _check_fields(a, b, 1e-5)


def test_set_state_round_trip():
    nx, ny = 29, 17
    p, f, _ = WL.random_state(nx, ny, seed=2)
    gpu, orc = _pair(nx, ny, p, f)
    orc.step(3)
    st = orc.get_state()
    gpu.set_state(st)
    back = gpu.get_state()
    for k in ("f", "g", "h", "phiu"):
        assert np.abs(back[k] - st[k].astype(np.float32)).max() == 0.0
    gpu.step(4)
    orc.step(4)
    a, b = gpu.fields(), orc.fields()
    _check_fields(a, b, 1e-5)


def test_microchannel_full_horizon():
    """Heated microchannel, 128 x 32, 20k steps (the FP64 closed-form workload): FP32 GPU
    fields against the FP64 oracle."""
    p, f, _ = WL.microchannel()
    gpu, orc = _pair(128, 32, p, f)
    gpu.step(20000)
    orc.step(20000)
    a, b = gpu.fields(), orc.fields()
    _check_fields(a, b, 1e-5)


def test_drop_migration_short():
    """256 x 1024 drop at Ma = 10 (heat-capacity contrast active), 300 steps."""
    p, f, _ = WL.drop_migration(Ma=10.0)
    gpu, orc = _pair(256, 1024, p, f)
    gpu.step(300)
    orc.step(300)
    a, b = gpu.fields(), orc.fields()
    _check_fields(a, b, 1e-5)


def test_bubbles_full_size():
    """2048 x 512 bubble channel (inlet, outflow, parabolic sigma), 20 steps at full size,
    compared on every node."""
    p, f, _ = WL.bubbles()
    gpu, orc = _pair(2048, 512, p, f)
    gpu.step(20)
    orc.step(20)
    a, b = gpu.fields(), orc.fields()
    _check_fields(a, b, 1e-5)


def test_mass_and_diagnostics():
    """FP64 device reductions against the oracle's fields; phi mass conserved in FP32."""
    nx, ny = 96, 64
    p, f, _ = WL.random_state(nx, ny, seed=5, bc_x=0, bc_y=0)
    gpu, orc = _pair(nx, ny, p, f)
    d0 = gpu.diagnostics()
    gpu.step(200)
    orc.step(200)
    d1 = gpu.diagnostics()
    fo = orc.fields()
    assert d1["nonfinite"] == 0 and d1["rc"] == 0
    assert abs(d1["sum_phi"] - d0["sum_phi"]) <= 1e-5 * np.abs(fo["phi"]).sum()
    assert d1["sum_phi"] == pytest.approx(fo["phi"].sum(), abs=1e-4 * np.abs(fo["phi"]).sum())
    assert d1["sum_T"] == pytest.approx(fo["T"].sum(), rel=1e-5)
    rcp = orc.aux()["rcp"]
    assert d1["sum_rcpT"] == pytest.approx((rcp * fo["T"]).sum(), rel=1e-5)
    neg = fo["phi"] < 0
    assert d1["Ur_den"] == pytest.approx(fo["phi"][neg].sum(), rel=1e-4)
    assert d1["Ur_num"] / d1["Ur_den"] == pytest.approx(
        (fo["phi"][neg] * fo["uy"][neg]).sum() / fo["phi"][neg].sum(), rel=1e-3, abs=1e-9)


def test_library_is_in_tree():
    import os

    from paper_2306_11320_gb300 import tpflbm
    from paper_2306_11320_gb300.build import LIB

    lat = _lattice(16, 16, WL.base_params())
    assert os.path.abspath(lat.lib._name) == os.path.abspath(LIB)
