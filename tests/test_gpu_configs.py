"""Every workload configuration against the FP64 oracle, at the horizons where a
pointwise comparison is meaningful (GPU through the C ABI; needs a GB300).

  microchannel 128 x 32 (Sec. 4.1)   FP16 storage at its full 20,000 steps (FP32: test_gpu_parity)
  drop 256 x 1024 (Sec. 4.2)         Ma = 0.1, 3,000 steps, FP32 and FP16
  drop 160 x 320, density ratio 10 and 1000 (Table 2)   4,000 steps, FP32
  bubbles 2048 x 512 (Sec. 4.3)      1,000 and 10,000 steps, FP32 and FP16, every node compared
  microchannel 512 x 128, the warm-start geometry   5,000 steps, FP32 and FP16

Bounds (tests/fieldcheck.py): FP32 max(1e-5, 3 x the float32 floor), FP16
max(5e-3, 3 x the float32 floor), the floor being the float32 oracle's own deviation
from the FP64 oracle on the same inputs and horizon.  Past 10,000 steps the two
bubbles of Sec. 4.3 approach coalescence, where pointwise parity stops being well
posed; the run is compared through its bubble diagnostics instead (test_gpu_bubbles).
"""
import numpy as np
import pytest

from fieldcheck import check_fields, oracle_horizons
from paper_2306_11320_gb300 import workloads as WL
from paper_2306_11320_gb300 import warmstart as WS

pytestmark = pytest.mark.gpu


def _gpu(nx, ny, params, fields, storage):
    from paper_2306_11320_gb300.tpflbm import Lattice

    p = dict(params, **WL.fp16_scales(params)) if storage else params
    lat = Lattice(nx, ny, p, storage=storage)
    lat.init(**{k: np.asarray(v, dtype=np.float32) for k, v in fields.items()})
    return lat


def _tol(storage):
    return 5e-3 if storage else 1e-5


def _horizons(lat, ref, storage, tag, bubbles=False):
    for steps, (fp64, fl) in sorted(ref.items()):
        lat.step(steps - lat.t)
        errs = check_fields(lat.fields(), fp64, _tol(storage), fl)
        print(tag, "storage", storage, "steps", steps, {k: "%.2e (bound %.2e)" % v for k, v in errs.items()})
        if bubbles:
            _bubbles_vs_oracle(lat, fp64, fl, storage)
    d = lat.diagnostics()
    assert d["nonfinite"] == 0


def _bubbles_vs_oracle(lat, fp64, fl, storage):
    """Sec. 4.3 per-bubble position and velocity from the device labelling against the
    flood-fill reference on the FP64 oracle's fields: the same two bubbles, node counts
    within a few interface nodes, centroid and velocity within max(a floor, 3 x the
    float32 oracle's own deviation) like the fields (floors: 1e-4 nodes and 1e-5 of the
    bubble speed for FP32, 1e-2 nodes and 5e-3 for FP16)."""
    from oracle.bubbles_ref import bubbles as ref_bubbles

    g = lat.bubbles()
    r = ref_bubbles(fp64["phi"], fp64["ux"], fp64["uy"])
    r32 = ref_bubbles(fl["phi"], fl["ux"], fl["uy"])
    assert len(g) == len(r) == len(r32) == 2, (g, r)
    x_floor, u_floor = (1e-2, 5e-3) if storage else (1e-4, 1e-5)
    for a, b, c in zip(g, r, r32):
        assert abs(a["nodes"] - b["nodes"]) <= 4, (a, b)
        for k in ("x_b", "y_b"):
            bound = max(x_floor, 3.0 * abs(c[k] - b[k]))
            assert abs(a[k] - b[k]) <= bound, (k, a[k], b[k], bound)
        speed = max(abs(b["u_b"]), abs(b["v_b"]))
        for k in ("u_b", "v_b"):
            bound = max(u_floor * speed, 3.0 * abs(c[k] - b[k]))
            assert abs(a[k] - b[k]) <= bound, (k, a[k], b[k], bound)
    print("bubbles", [(round(b["x_b"], 3), "%.3e" % b["u_b"]) for b in g])


# ------------------------------------------------------------ bubbles, Sec. 4.3

@pytest.fixture(scope="module")
def bubbles_ref():
    """FP64 and float32 oracles of the 2048 x 512 two-bubble channel at 1,000 and
    10,000 steps (several minutes on the host cores)."""
    p, f, _ = WL.bubbles()
    return p, f, oracle_horizons(2048, 512, p, f, (1000, 10000))


@pytest.mark.parametrize("storage", [0, 1])
def test_bubbles_1000_and_10000_steps(bubbles_ref, storage):
    """The bench workload at its full size through the TMA kernel the bench times:
    every field on every node after 1,000 and after 10,000 steps."""
    p, f, ref = bubbles_ref
    _horizons(_gpu(2048, 512, p, f, storage), ref, storage, "bubbles", bubbles=True)


# ------------------------------------------------------- microchannel, Sec. 4.1

def test_microchannel_fp16_full_horizon():
    """Heated microchannel 128 x 32 with FP16 population storage, all 20,000 steps."""
    p, f, _ = WL.microchannel()
    ref = oracle_horizons(128, 32, p, f, (5000, 20000))
    _horizons(_gpu(128, 32, p, f, 1), ref, 1, "microchannel")


@pytest.mark.parametrize("storage", [0, 1])
@pytest.mark.parametrize("inst", [dict(lam_r=0.2, hr=1.0, k=1), dict(lam_r=5.0, hr=0.7, k=3)])
def test_warmstart_channel(inst, storage):
    """The 512 x 128 channel of the warm-start study (two draws of conductivity ratio,
    layer-height ratio and wall wavenumber), 5,000 steps from the cold start."""
    p, f, _ = WS.channel(inst)
    ref = oracle_horizons(WS.NX, WS.NY, p, f, (1000, 5000))
    _horizons(_gpu(WS.NX, WS.NY, p, f, storage), ref, storage, "channel %s" % inst)


# --------------------------------------------------------------- drops, Sec. 4.2

@pytest.fixture(scope="module")
def drop_ref():
    p, f, _ = WL.drop_migration(Ma=0.1)
    return p, f, oracle_horizons(256, 1024, p, f, (3000,))


@pytest.mark.parametrize("storage", [0, 1])
def test_drop_ma01_3000_steps(drop_ref, storage):
    """The 256 x 1024 drop at Ma = Re = 0.1 (heat-capacity ratio 0.5), 3,000 steps."""
    p, f, ref = drop_ref
    _horizons(_gpu(256, 1024, p, f, storage), ref, storage, "drop")


@pytest.mark.parametrize("rho_r", [10.0, 1000.0])
def test_density_ratio_drop(rho_r):
    """Table 2's drop at density ratio 10 and 1000 (rho and tau_g contrast of up to
    1000:1 inside the float32 arithmetic), 4,000 steps."""
    p, f, _ = WL.drop_density_ratio(rho_r)
    ref = oracle_horizons(160, 320, p, f, (1000, 4000))
    _horizons(_gpu(160, 320, p, f, 0), ref, 0, "rho_r %g" % rho_r)
