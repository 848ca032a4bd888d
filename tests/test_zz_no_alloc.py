"""tpflbm_diagnostics_static: the reductions for callers that cannot allocate device
memory (an allocator callback, a graph built from pre-planned buffers, a host that
only hands out fixed buffers).  Its scratch is a fixed array inside the library, so
the call itself allocates nothing; the caller passes the state it already owns.

Checked against tpflbm_diagnostics (the handle-based entry point) on the same state,
on two calls in a row.  Collected last so that a stop at the first failure has
already run every other test.
"""
import ctypes as C

import numpy as np
import pytest

from paper_2306_11320_gb300 import workloads as WL

pytestmark = pytest.mark.gpu


def _device_state(torch, st, nx, ny, plane):
    """Populations (27 planes) and (phi u) (2 planes) in the library's state layout,
    with a plane stride of `plane` elements."""
    N = nx * ny
    pop = torch.zeros(27 * plane, dtype=torch.float32, device="cuda")
    planes = np.concatenate([st["f"], st["g"], st["h"]]).reshape(27, N)
    pop.view(27, plane)[:, :N] = torch.from_numpy(np.ascontiguousarray(planes, dtype=np.float32)).cuda()
    phiu = torch.zeros(2 * plane, dtype=torch.float32, device="cuda")
    phiu.view(2, plane)[:, :N] = torch.from_numpy(st["phiu"].reshape(2, N).astype(np.float32)).cuda()
    return pop, phiu


def test_static_scratch_matches_handle_diagnostics():
    import torch

    from paper_2306_11320_gb300.tpflbm import Lattice, make_params

    nx, ny = 96, 40
    params, fields, _ = WL.random_state(nx, ny, seed=21, bc_x=0, bc_y=0)
    lat = Lattice(nx, ny, params)
    lat.init(**{k: v.astype(np.float32) for k, v in fields.items()})
    lat.step(25)
    ref = lat.diagnostics()
    assert ref["rc"] == 0
    expected = np.array([ref[k] for k in ("sum_phi", "sum_rcpT", "sum_T", "Ur_num", "Ur_den",
                                          "ub_num", "xb_num")] + [ref["nonfinite"]])

    st = lat.get_state()
    plane = nx * ny + 37  # any stride >= nx * ny
    pop, phiu = _device_state(torch, st, nx, ny, plane)
    p = make_params(params)
    stream = torch.cuda.current_stream().cuda_stream
    for call in range(2):
        out = (C.c_double * 8)()
        rc = lat.lib.tpflbm_diagnostics_static(nx, ny, C.byref(p), C.c_void_p(pop.data_ptr()), plane, None,
                                               C.c_void_p(phiu.data_ptr()), out, C.c_void_p(stream))
        assert rc == 0, lat.lib.tpflbm_last_error(None).decode()
        got = np.array(out[:])
        # same kernel, same block count: equal up to FP64 rounding of the partial sums
        assert np.allclose(got, expected, rtol=1e-12, atol=1e-12 * np.abs(expected).max()), (call, got, expected)

    # a device output buffer works too
    dout = torch.zeros(8, dtype=torch.float64, device="cuda")
    rc = lat.lib.tpflbm_diagnostics_static(nx, ny, C.byref(p), C.c_void_p(pop.data_ptr()), plane, None,
                                           C.c_void_p(phiu.data_ptr()), C.c_void_p(dout.data_ptr()),
                                           C.c_void_p(stream))
    assert rc == 0
    assert np.allclose(dout.cpu().numpy(), expected, rtol=1e-12, atol=1e-12 * np.abs(expected).max())


def test_static_scratch_rejects_bad_sizes():
    import torch

    from paper_2306_11320_gb300.tpflbm import load_library, make_params

    lib = load_library()
    p = make_params(WL.base_params())
    buf = torch.zeros(27 * 64, dtype=torch.float32, device="cuda")
    out = (C.c_double * 8)()
    ptr = C.c_void_p(buf.data_ptr())
    # lattice larger than the library accepts (nx * ny > 2^30)
    rc = lib.tpflbm_diagnostics_static(65536, 32768, C.byref(p), ptr, 1 << 31, None, ptr, out, None)
    assert rc == -1 and b"too large" in lib.tpflbm_last_error(None)
    # plane stride shorter than a plane
    rc = lib.tpflbm_diagnostics_static(8, 8, C.byref(p), ptr, 63, None, ptr, out, None)
    assert rc == -1 and b"plane" in lib.tpflbm_last_error(None)
    # FP16 storage without its reference planes
    p16 = make_params(WL.base_params(storage=1))
    rc = lib.tpflbm_diagnostics_static(8, 8, C.byref(p16), ptr, 64, None, ptr, out, None)
    assert rc == -1 and b"reference" in lib.tpflbm_last_error(None)
