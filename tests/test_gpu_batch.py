"""Batched ensemble through the C-ABI (needs a GB300): uneven lattices with their own
parameters and boundary kinds, advanced by one persistent launch per step and
replayed from CUDA graphs, against the FP64 oracle lattice by lattice."""
import numpy as np
import pytest

from oracle.oracle import OracleSim
from paper_2306_11320_gb300 import workloads as WL

pytestmark = pytest.mark.gpu

FIELDS = ("phi", "ux", "uy", "p", "T")


def rel_l2(a, b):
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    den = np.sqrt((b ** 2).sum())
    return float(np.sqrt(((a - b) ** 2).sum()) / den) if den > 0 else float(np.abs(a - b).max())


def _members():
    """A small ensemble: sweep instances (microchannel / drop, Ma, viscosity and
    conductivity ratios) plus random two-phase states with every boundary kind."""
    out = [(m["nx"], m["ny"], p, f) for p, f, m in WL.ensemble(n=6, seed=3, nx_range=(32, 96),
                                                               ny_range=(24, 64))]
    # the last two run through TMA in the TMA-staged variant: every tile of the inlet /
    # outflow channel, the walled rows of the periodic lattice
    for (nx, ny, bx, by, law, seed) in ((41, 19, 1, 0, 1, 1), (64, 32, 0, 1, 0, 2), (37, 23, 0, 0, 1, 3),
                                        (128, 40, 1, 0, 1, 4), (96, 48, 0, 0, 0, 5)):
        p, f, _ = WL.random_state(nx, ny, seed=seed, bc_x=bx, bc_y=by, sigma_law=law)
        out.append((nx, ny, p, f))
    return out


def _batch(members, storage=0, variant=None):
    from paper_2306_11320_gb300.tpflbm import Batch

    b = Batch([(nx, ny, p) for nx, ny, p, _ in members], storage=storage)
    for k, (_, _, _, f) in enumerate(members):
        b.init(k, **{n: v.astype(np.float32) for n, v in f.items()})
    if variant == "tma":
        b.set_variant(Batch.tma_variant(b.lib))
    return b


@pytest.mark.parametrize("variant", [None, "tma"])
def test_batch_matches_single_lattices(variant):
    """Each member of the batch evolves as the same lattice stepped alone through the
    single-lattice API (the per-tile code is shared), with the general tile path and
    with the TMA-staged variant.  The two launches are different kernels, and the
    compiler may fuse a multiply-add differently in each; the small random states
    amplify such a 1-ulp difference (2e-6 of u_x, 1.2e-5 of phi on the 41 x 19 channel
    after 40 steps), as much as float32 evaluations that differ only by rounding
    spread among themselves.  Bound per member and field: max(1e-6, 3 x that spread
    (tests/fieldcheck.py)); a tile run with another lattice's parameters, buffers or
    tile coordinates is off by O(1)."""
    from fieldcheck import float32_spread
    from paper_2306_11320_gb300.tpflbm import Lattice

    members = _members()
    b = _batch(members, variant=variant)
    steps = 40
    b.step(steps)
    for k, (nx, ny, p, f) in enumerate(members):
        lat = Lattice(nx, ny, p)
        lat.init(**{n: v.astype(np.float32) for n, v in f.items()})
        lat.step(steps)
        a, c = b.fields(k), lat.fields()
        o = OracleSim(nx, ny, p)
        o.init(**{n: v.astype(np.float32).astype(np.float64) for n, v in f.items()})
        o.step(steps)
        spread = float32_spread(nx, ny, p, f, steps, o.fields())
        for n in FIELDS:
            bound = max(1e-6, 3.0 * spread[n])
            assert rel_l2(a[n], c[n]) <= bound, (k, n, rel_l2(a[n], c[n]), bound)


def test_batch_matches_oracle():
    """Against the FP64 oracle once the flows have developed (a few steps from rest
    the velocities are ~1e-9 and their relative error is pure rounding noise): each
    field within max(1e-5, 3 x the float32 floor), the floor being the largest
    deviation among float32 oracle runs that differ only by rounding (the plain one
    and three from +-1 ulp perturbed initial fields, tests/fieldcheck.py)."""
    from fieldcheck import float32_spread

    members = _members()
    b = _batch(members)
    steps = 300
    b.step(steps)
    for k, (nx, ny, p, f) in enumerate(members):
        f32 = {n: v.astype(np.float32).astype(np.float64) for n, v in f.items()}
        o = OracleSim(nx, ny, p)
        o.init(**f32)
        o.step(steps)
        a, ref = b.fields(k), o.fields()
        fl = float32_spread(nx, ny, p, f, steps, ref)
        for n in FIELDS:
            bound = max(1e-5, 3.0 * fl[n])
            assert rel_l2(a[n], ref[n]) <= bound, (k, n, rel_l2(a[n], ref[n]), bound)
    d, rc = b.diagnostics()
    assert rc == 0 and d.shape == (len(members), 8) and np.all(d[:, 7] == 0)


def test_graph_replay_equals_direct_launches():
    members = _members()
    b1, b2 = _batch(members), _batch(members)
    b1.step(30)          # 15 graph replays of two steps
    for _ in range(30):  # 30 direct launches
        b2.step(1)
    assert b1.t == b2.t == 30
    for k in range(len(members)):
        a, c = b1.fields(k), b2.fields(k)
        for n in FIELDS:
            assert np.array_equal(a[n], c[n]), (k, n)


def test_tile_shapes_agree_and_tuner_picks_one():
    from paper_2306_11320_gb300.tpflbm import Batch

    members = _members()
    shapes = Batch.variants()
    assert len(shapes) >= 2
    results = []
    for v in range(len(shapes)):
        b = _batch(members)
        b.set_variant(v)
        b.step(20)
        results.append([b.fields(k) for k in range(len(members))])
    for v in range(1, len(shapes)):
        for k in range(len(members)):
            for n in FIELDS:
                assert rel_l2(results[v][k][n], results[0][k][n]) <= 1e-6, (v, k, n)
    b = _batch(members)
    best, ms = b.tune(steps=10)
    assert 0 <= best < len(shapes) and all(t > 0 for t in ms)
    assert ms[best] == min(ms)
    assert b.t == len(shapes) * 12


@pytest.mark.parametrize("variant", [None, "tma"])
def test_fp16_batch(variant):
    """FP16 storage in the batch (general tile path, and the TMA-staged variant): within
    5e-3 relative L2 of the FP64 oracle, plus three times the float32 oracle's own
    deviation for members whose flow is so weak (|u| ~ 1e-7) that float32 arithmetic
    alone is off by more than that."""
    members = [m for m in _members()]
    members = [(nx, ny, dict(p, **WL.fp16_scales(p)), f) for nx, ny, p, f in members]
    b = _batch(members, storage=1, variant=variant)
    steps = 1500
    b.step(steps)
    for k, (nx, ny, p, f) in enumerate(members):
        f32 = {n: v.astype(np.float32).astype(np.float64) for n, v in f.items()}
        o = OracleSim(nx, ny, p)
        o.init(**f32)
        o.step(steps)
        o32 = OracleSim(nx, ny, p, real="float")
        o32.init(**f32)
        o32.step(steps)
        a, ref, fl = b.fields(k), o.fields(), o32.fields()
        for n in FIELDS:
            bound = 5e-3 + 3.0 * rel_l2(fl[n], ref[n])
            assert rel_l2(a[n], ref[n]) <= bound, (k, n, rel_l2(a[n], ref[n]), bound)
