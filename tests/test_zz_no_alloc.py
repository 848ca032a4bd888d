"""tpflbm_diagnostics_static: the reductions for callers that must not allocate device
memory (code running inside an allocator's or a memory pool's own callback, where a
cudaMalloc would re-enter the allocator, or a host that hands out only fixed buffers it
owns).  Its scratch is a fixed array inside the library, so the call itself allocates
nothing; the caller passes the state it already owns.

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


class _DeviceBytes:
    """A raw device address seen by torch as a uint8 array (__cuda_array_interface__)."""

    def __init__(self, addr, nbytes):
        self.__cuda_array_interface__ = {"shape": (nbytes,), "typestr": "|u1", "data": (addr, False),
                                         "version": 3, "strides": None}


def _copy_planes(torch, src_addr, nplanes, plane_src, plane_dst, n, elem_bytes):
    """Copy `nplanes` planes of n elements (elem_bytes each) from the handle's state at
    src_addr (stride plane_src) into a fresh caller buffer with stride plane_dst."""
    src = torch.as_tensor(_DeviceBytes(src_addr, nplanes * plane_src * elem_bytes), device="cuda")
    dst = torch.zeros(nplanes * plane_dst * elem_bytes, dtype=torch.uint8, device="cuda")
    for k in range(nplanes):
        dst[k * plane_dst * elem_bytes:(k * plane_dst + n) * elem_bytes] = \
            src[k * plane_src * elem_bytes:(k * plane_src + n) * elem_bytes]
    return dst


def test_static_scratch_fp16_records():
    """FP16 storage: the float16 populations and their reference records, copied from a
    stepped lattice into caller buffers with a plane stride of its own, give the handle's
    diagnostics on two calls in a row."""
    import torch

    from paper_2306_11320_gb300.tpflbm import STORAGE_FP16, Lattice, make_params

    nx, ny = 96, 40
    params, fields, _ = WL.random_state(nx, ny, seed=22, bc_x=1, bc_y=0, sigma_law=1)
    params = dict(params, **WL.fp16_scales(params))
    lat = Lattice(nx, ny, params, storage=STORAGE_FP16)
    lat.init(**{k: v.astype(np.float32) for k, v in fields.items()})
    lat.step(25)
    ref = lat.diagnostics()
    assert ref["rc"] == 0
    expected = np.array([ref[k] for k in ("sum_phi", "sum_rcpT", "sum_T", "Ur_num", "Ur_den",
                                          "ub_num", "xb_num")] + [ref["nonfinite"]])
    torch.cuda.synchronize()
    pop_a, ref_a, phiu_a, plane_a = lat.state_buffers()
    assert ref_a is not None and plane_a >= nx * ny
    N = nx * ny
    plane = N + 29  # a stride unlike the library's padded one
    pop = _copy_planes(torch, pop_a, 27, plane_a, plane, N, 2)
    rec = _copy_planes(torch, ref_a, 3, plane_a, plane, N, 8)
    phiu = _copy_planes(torch, phiu_a, 2, plane_a, plane, N, 4)
    p = make_params(params, STORAGE_FP16)
    stream = torch.cuda.current_stream().cuda_stream
    for call in range(2):
        out = (C.c_double * 8)()
        rc = lat.lib.tpflbm_diagnostics_static(nx, ny, C.byref(p), C.c_void_p(pop.data_ptr()), plane,
                                               C.c_void_p(rec.data_ptr()), C.c_void_p(phiu.data_ptr()), out,
                                               C.c_void_p(stream))
        assert rc == 0, lat.lib.tpflbm_last_error(None).decode()
        got = np.array(out[:])
        assert np.allclose(got, expected, rtol=1e-12, atol=1e-12 * np.abs(expected).max()), (call, got, expected)
