"""Pin of the half-source initialisation reference (CPU): populations built from the
oracle's equilibria minus half of its forcing sources decode, in the oracle itself,
to exactly the fields they were built from (u from the forced first moment, p from
the pressure moment with its u . grad rho term), with phi and T untouched."""
import numpy as np
import pytest

from oracle import warmstart_ref as R
from oracle.oracle import OracleSim
from paper_2306_11320_gb300 import workloads as WL


@pytest.mark.parametrize("bc_x,bc_y", [(0, 0), (1, 0), (0, 1)])
def test_forced_init_decodes_to_its_fields(bc_x, bc_y):
    nx, ny = 24, 16
    p, f, _ = WL.random_state(nx, ny, seed=9, bc_x=bc_x, bc_y=bc_y)
    st = R.forced_init_state(nx, ny, p, f)
    o = OracleSim(nx, ny, p)
    o.init(**f)
    o.set_state(st)
    got = o.fields()
    for k in ("phi", "ux", "uy", "p", "T"):
        ref = np.asarray(f[k], dtype=np.float64)
        assert np.abs(got[k] - ref).max() <= 1e-12 * max(1.0, np.abs(ref).max()), k
    # and the plain equilibrium does not: its velocity is off by F / (2 rho)
    o.init(**f)
    eq = o.fields()
    a = o.aux()
    assert np.abs(eq["ux"] - f["ux"]).max() > 1e-6
    assert np.allclose(eq["ux"] - f["ux"], a["Fx"] / (2 * a["rho"]), atol=1e-12)
