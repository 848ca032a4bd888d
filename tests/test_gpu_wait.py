"""The step kernels' failure path without a GPU fault (needs a GB300): a bounded wait on
an mbarrier that nothing completes gives up and raises its flag, and the context keeps
working afterwards."""
import numpy as np
import pytest

from oracle.oracle import OracleSim
from paper_2306_11320_gb300 import workloads as WL

pytestmark = pytest.mark.gpu


def test_bounded_wait_gives_up_and_context_survives():
    from paper_2306_11320_gb300.tpflbm import Lattice, TpfError, check_bounded_wait

    assert check_bounded_wait(polls=4096)
    with pytest.raises(TpfError):
        check_bounded_wait(polls=0)
    # the same context then steps a lattice through the TMA kernel as usual
    nx, ny, steps = 64, 24, 10
    p, f, _ = WL.random_state(nx, ny, seed=11, bc_x=1, bc_y=0, sigma_law=1)
    f32 = {k: v.astype(np.float32) for k, v in f.items()}
    lat = Lattice(nx, ny, p)
    lat.init(**f32)
    lat.step(steps)
    gpu = lat.fields()
    orc = OracleSim(nx, ny, p)
    orc.init(**{k: v.astype(np.float64) for k, v in f32.items()})
    orc.step(steps)
    ref = orc.fields()
    for k in ("phi", "ux", "uy", "p", "T"):
        err = np.sqrt(((gpu[k] - ref[k]) ** 2).sum() / (ref[k] ** 2).sum())
        assert err <= 1e-5, (k, err)
    assert lat.diagnostics()["nonfinite"] == 0


def test_status_async_reads_each_step():
    """tpflbm_status_async copies the step kernels' error flag to pinned host memory
    without waiting, on the lattice's stream or on a copy stream behind its steps; after
    an event behind the copy the flag reads 0 for steps that completed, as
    tpflbm_status reports."""
    import ctypes as C

    import torch

    from paper_2306_11320_gb300.tpflbm import Lattice

    nx, ny = 96, 40
    p, f, _ = WL.random_state(nx, ny, seed=12, bc_x=1, bc_y=0)
    stream = torch.cuda.Stream()
    lat = Lattice(nx, ny, p, stream=stream)
    lat.init(**{k: v.astype(np.float32) for k, v in f.items()})
    copy = torch.cuda.Stream()
    flags = torch.full((8,), -7, dtype=torch.int32).pin_memory()
    events = [torch.cuda.Event() for _ in range(8)]
    for k in range(8):
        assert lat.lib.tpflbm_step(lat.h, 3) == 0
        # even k: on the lattice's stream; odd k: on a copy stream behind the steps
        cs = None if k % 2 == 0 else C.c_void_p(copy.cuda_stream)
        assert lat.lib.tpflbm_status_async(lat.h, C.c_void_p(flags[k].data_ptr()), cs) == 0
        events[k].record(stream if k % 2 == 0 else copy)
    for k in range(8):
        events[k].synchronize()
        assert int(flags[k]) == 0
    assert lat.lib.tpflbm_status(lat.h) == 0
    assert lat.lib.tpflbm_status_async(lat.h, None, None) != 0  # no destination
    assert lat.t == 24
