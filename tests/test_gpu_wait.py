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
