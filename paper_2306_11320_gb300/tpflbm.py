"""Python binding of the tpflbm C-ABI library (ctypes; argument marshalling only).

Every step of the method runs in the CUDA kernels of libtpflbm.so.  PyTorch
supplies device memory (the lattice workspace is a torch uint8 tensor passed to
tpflbm_create_in) and the CUDA stream (torch's current stream).  There is no
CPU fallback: constructing a Lattice without the built library or without a CUDA
device raises.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

from .build import LIB, build_library

_PARAM_DOUBLES = [
    "rho_l", "rho_h", "mu_l", "mu_h", "lambda_l", "lambda_h", "cp_l", "cp_h",
    "W", "M_phi",
    "sigma_ref", "sigma_T", "sigma_TT", "T_ref",
    "Gx", "Gy",
    "u_ave", "phi_in", "T_in", "p_out",
    "T_bot", "T_bot_amp", "T_bot_k", "T_bot_slope", "T_top", "T_top_slope",
    "fp16_scale_f", "fp16_scale_g", "fp16_scale_h",
    "trt_lambda",
]
_PARAM_INTS = ["sigma_law", "bc_x", "bc_y", "storage", "normal_law", "collision"]

STORAGE_FP32 = 0
STORAGE_FP16 = 1

ERRORS = {0: "ok", -1: "invalid argument", -2: "out of memory", -3: "CUDA error",
          -4: "non-finite state", -5: "timeout", -6: "unsupported"}


class Params(C.Structure):
    _fields_ = [(n, C.c_double) for n in _PARAM_DOUBLES] + [(n, C.c_int) for n in _PARAM_INTS]


class TpfError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__("tpflbm error %d (%s): %s" % (code, ERRORS.get(code, "?"), msg))
        self.code = code


_lib = None

# the entry points include/tpflbm.h declares, with (argtypes, restype)
_vp, _fp, _dp, _ip = C.c_void_p, C.POINTER(C.c_float), C.POINTER(C.c_double), C.c_int
SIGNATURES = {
    "tpflbm_workspace_bytes": ([_ip, _ip, C.POINTER(Params)], C.c_size_t),
    "tpflbm_create": ([_ip, _ip, C.POINTER(Params), C.POINTER(_vp)], _ip),
    "tpflbm_create_in": ([_ip, _ip, C.POINTER(Params), _vp, C.c_size_t, C.POINTER(_vp)], _ip),
    "tpflbm_set_stream": ([_vp, _vp], _ip),
    "tpflbm_init": ([_vp, _vp, _vp, _vp, _vp, _vp], _ip),
    "tpflbm_init_forced": ([_vp, _vp, _vp, _vp, _vp, _vp, _ip], _ip),
    "tpflbm_step": ([_vp, C.c_longlong], _ip),
    "tpflbm_status": ([_vp], _ip),
    "tpflbm_status_async": ([_vp, _vp, _vp], _ip),
    "tpflbm_get_fields": ([_vp, _vp, _vp, _vp, _vp, _vp], _ip),
    "tpflbm_get_state": ([_vp, _vp, _vp, _vp, _vp], _ip),
    "tpflbm_set_state": ([_vp, _vp, _vp, _vp, _vp], _ip),
    "tpflbm_diagnostics": ([_vp, _dp], _ip),
    "tpflbm_diagnostics_static": ([_ip, _ip, C.POINTER(Params), _vp, C.c_longlong, _vp, _vp, _vp, _vp], _ip),
    "tpflbm_state_buffers": ([_vp, C.POINTER(_vp), C.POINTER(_vp), C.POINTER(_vp), C.POINTER(C.c_longlong)], _ip),
    "tpflbm_bubbles": ([_vp, _ip, _dp, C.POINTER(C.c_int)], _ip),
    "tpflbm_residual": ([_vp, C.c_double, _dp], _ip),
    "tpflbm_project_phi": ([_vp, _vp, C.c_double, _ip, _vp, _dp], _ip),
    "tpflbm_time": ([_vp], C.c_longlong),
    "tpflbm_destroy": ([_vp], None),
    "tpflbm_last_error": ([_vp], C.c_char_p),
    "tpflbm_batch_create": ([_ip, C.POINTER(C.c_int), C.POINTER(C.c_int), C.POINTER(Params), C.POINTER(_vp)], _ip),
    "tpflbm_batch_set_stream": ([_vp, _vp], _ip),
    "tpflbm_batch_size": ([_vp], _ip),
    "tpflbm_batch_lattice": ([_vp, _ip, C.POINTER(_vp)], _ip),
    "tpflbm_batch_init": ([_vp, _ip, _vp, _vp, _vp, _vp, _vp], _ip),
    "tpflbm_batch_step": ([_vp, C.c_longlong], _ip),
    "tpflbm_batch_get_fields": ([_vp, _ip, _vp, _vp, _vp, _vp, _vp], _ip),
    "tpflbm_batch_diagnostics": ([_vp, _dp], _ip),
    "tpflbm_batch_residual": ([_vp, _dp, _dp], _ip),
    "tpflbm_batch_variants": ([C.POINTER(C.c_int), C.POINTER(C.c_int), C.POINTER(C.c_int)], _ip),
    "tpflbm_batch_set_variant": ([_vp, _ip], _ip),
    "tpflbm_check_bounded_wait": ([C.c_int, C.POINTER(C.c_int)], _ip),
    "tpflbm_batch_tune": ([_vp, _ip, _dp, C.POINTER(C.c_int)], _ip),
    "tpflbm_batch_time": ([_vp], C.c_longlong),
    "tpflbm_batch_destroy": ([_vp], None),
    "tpflbm_batch_last_error": ([_vp], C.c_char_p),
}


def load_library(path: str | None = None, build: bool = True):
    """Load libtpflbm.so (building it in-tree first when `build`)."""
    global _lib
    if _lib is not None and path is None:
        return _lib
    if path is None:
        path = build_library() if build else LIB
    if not os.path.exists(path):
        raise RuntimeError("libtpflbm.so is missing at %s: build it with "
                           "`python -c 'import __graft_entry__ as g; g.build()'`" % path)
    lib = C.CDLL(path)
    for name, (args, res) in SIGNATURES.items():
        fn = getattr(lib, name)
        fn.argtypes = args
        fn.restype = res
    if os.path.abspath(path) == os.path.abspath(LIB):
        _lib = lib
    return lib


def check_bounded_wait(polls: int = 4096, lib=None) -> bool:
    """tpflbm_check_bounded_wait: True when a bounded wait on an mbarrier that nothing
    completes gave up after `polls` polls and raised its flag."""
    lib = lib if lib is not None else load_library()
    out = C.c_int(0)
    rc = lib.tpflbm_check_bounded_wait(int(polls), C.byref(out))
    if rc != 0:
        raise TpfError(rc, lib.tpflbm_last_error(None).decode())
    return bool(out.value)


def make_params(p: dict, storage: int = STORAGE_FP32) -> Params:
    s = Params()
    for n in _PARAM_DOUBLES:
        setattr(s, n, float(p.get(n, 0.0)))
    for n in _PARAM_INTS:
        setattr(s, n, int(p.get(n, 0)))
    s.storage = int(p.get("storage", storage))
    return s


def _ptr(a):
    """Data pointer of a numpy array or torch tensor (host or device)."""
    if a is None:
        return None
    if hasattr(a, "data_ptr"):
        return C.c_void_p(a.data_ptr())
    return C.c_void_p(a.ctypes.data)


class Lattice:
    """One nx x ny lattice advanced on the GPU by the tpflbm library.

    Fields are float32, shape (ny, nx); populations (9, ny, nx) per LBE.
    `workspace="torch"` lets PyTorch own the device memory; `"library"` lets the
    library cudaMalloc it.
    """

    def __init__(self, nx: int, ny: int, params: dict, storage: int = STORAGE_FP32,
                 workspace: str = "torch", stream=None, lib=None):
        import torch

        if not torch.cuda.is_available():
            raise RuntimeError("tpflbm needs a CUDA device; there is no CPU fallback")
        self.torch = torch
        self.lib = lib if lib is not None else load_library()
        self.nx, self.ny = int(nx), int(ny)
        self.params = dict(params)
        self._p = make_params(params, storage)
        self.storage = self._p.storage
        h = C.c_void_p()
        self._ws = None
        if workspace == "torch":
            nbytes = self.lib.tpflbm_workspace_bytes(self.nx, self.ny, C.byref(self._p))
            if nbytes == 0:
                raise TpfError(-1, "invalid lattice size or parameters")
            self._ws = torch.empty(nbytes + 256, dtype=torch.uint8, device="cuda")
            base = self._ws.data_ptr()
            aligned = (base + 255) & ~255
            rc = self.lib.tpflbm_create_in(self.nx, self.ny, C.byref(self._p), C.c_void_p(aligned),
                                           nbytes, C.byref(h))
        else:
            rc = self.lib.tpflbm_create(self.nx, self.ny, C.byref(self._p), C.byref(h))
        if rc != 0:
            raise TpfError(rc, self.lib.tpflbm_last_error(None).decode())
        self.h = h
        s = stream if stream is not None else torch.cuda.current_stream()
        self.stream = s
        self._check(self.lib.tpflbm_set_stream(self.h, C.c_void_p(s.cuda_stream)))

    # ----------------------------------------------------------------- helpers
    def _check(self, rc):
        if rc != 0:
            raise TpfError(rc, self.lib.tpflbm_last_error(self.h).decode())

    def _field(self, a):
        if a is None:
            return None
        if hasattr(a, "data_ptr"):
            t = a.to(dtype=self.torch.float32).contiguous()
            assert tuple(t.shape) == (self.ny, self.nx)
            return t
        a = np.ascontiguousarray(np.broadcast_to(np.asarray(a, dtype=np.float32), (self.ny, self.nx)))
        return a

    def close(self):
        if getattr(self, "h", None):
            self.lib.tpflbm_destroy(self.h)
            self.h = None
        self._ws = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # -------------------------------------------------------------------- API
    def init(self, phi=None, ux=None, uy=None, p=None, T=None, forced=0):
        """Populations from fields: equilibria, or (forced = 1, 2, 3: bits for f, g)
        equilibria less half of the forcing sources (tpflbm_init_forced; with 3 they
        decode to exactly these u and p)."""
        arrs = [self._field(a) for a in (phi, ux, uy, p, T)]
        if forced:
            self._check(self.lib.tpflbm_init_forced(self.h, *[_ptr(a) for a in arrs], int(forced)))
        else:
            self._check(self.lib.tpflbm_init(self.h, *[_ptr(a) for a in arrs]))

    def step(self, n: int = 1):
        self._check(self.lib.tpflbm_step(self.h, int(n)))

    @property
    def t(self) -> int:
        return int(self.lib.tpflbm_time(self.h))

    def fields(self, device: bool = False):
        """dict of phi, ux, uy, p, T as numpy float32 (or torch CUDA tensors)."""
        if device:
            out = [self.torch.empty((self.ny, self.nx), dtype=self.torch.float32, device="cuda")
                   for _ in range(5)]
        else:
            out = [np.empty((self.ny, self.nx), dtype=np.float32) for _ in range(5)]
        self._check(self.lib.tpflbm_get_fields(self.h, *[_ptr(a) for a in out]))
        return dict(zip(("phi", "ux", "uy", "p", "T"), out))

    def get_state(self):
        f = np.empty((9, self.ny, self.nx), dtype=np.float32)
        g = np.empty_like(f)
        h = np.empty_like(f)
        pu = np.empty((2, self.ny, self.nx), dtype=np.float32)
        self._check(self.lib.tpflbm_get_state(self.h, _ptr(f), _ptr(g), _ptr(h), _ptr(pu)))
        return {"f": f, "g": g, "h": h, "phiu": pu}

    def set_state(self, st):
        arrs = [np.ascontiguousarray(st[k], dtype=np.float32) for k in ("f", "g", "h", "phiu")]
        self._check(self.lib.tpflbm_set_state(self.h, *[_ptr(a) for a in arrs]))

    def residual(self, dT: float):
        """(r_u, r_T, K) of the steady-state residual (inf before the first snapshot)."""
        out = (C.c_double * 3)()
        self._check(self.lib.tpflbm_residual(self.h, float(dT), out))
        return out[0], out[1], int(out[2])

    def project_phi(self, phi_pred, target_sum: float, mode: int = 1, out=None):
        """Mass-preserving projection of a predicted phase field (a float32 CUDA tensor
        of shape (ny, nx)) onto the tanh profile (mode 1: about each column's zero
        crossing; 0: through atanh); returns (phi, achieved FP64 sum)."""
        t = self.torch
        assert phi_pred.is_cuda and phi_pred.dtype == t.float32 and tuple(phi_pred.shape) == (self.ny, self.nx)
        phi_pred = phi_pred.contiguous()
        out = t.empty_like(phi_pred) if out is None else out
        got = C.c_double()
        self._check(self.lib.tpflbm_project_phi(self.h, C.c_void_p(phi_pred.data_ptr()), float(target_sum), int(mode),
                                                C.c_void_p(out.data_ptr()), C.byref(got)))
        return out, got.value

    def state_buffers(self):
        """tpflbm_state_buffers: (pop, ref, phiu, plane), device addresses of the current
        state (ref is None with FP32 storage) and the elements per plane."""
        pop, ref, phiu, plane = C.c_void_p(), C.c_void_p(), C.c_void_p(), C.c_longlong()
        self._check(self.lib.tpflbm_state_buffers(self.h, C.byref(pop), C.byref(ref), C.byref(phiu),
                                                  C.byref(plane)))
        return pop.value, ref.value, phiu.value, plane.value

    BUBBLE_KEYS = ("nodes", "sum_phi", "u_b", "v_b", "x_b", "y_b")

    def bubbles(self, max_bubbles: int = 32):
        """tpflbm_bubbles: the connected phi < 0 regions of the current state (Sec. 4.3),
        ordered by x_b, as a list of dicts with BUBBLE_KEYS."""
        out = (C.c_double * (6 * max_bubbles))()
        n = C.c_int()
        self._check(self.lib.tpflbm_bubbles(self.h, int(max_bubbles), out, C.byref(n)))
        vals = np.array(out[:]).reshape(max_bubbles, 6)
        return [dict(zip(self.BUBBLE_KEYS, row)) for row in vals[:min(n.value, max_bubbles)]]

    def diagnostics(self):
        out = (C.c_double * 8)()
        rc = self.lib.tpflbm_diagnostics(self.h, out)
        vals = np.array(out[:])
        if rc not in (0, -4):
            self._check(rc)
        return dict(sum_phi=vals[0], sum_rcpT=vals[1], sum_T=vals[2], Ur_num=vals[3], Ur_den=vals[4],
                    ub_num=vals[5], xb_num=vals[6], nonfinite=int(vals[7]), rc=rc)


class Batch:
    """An ensemble of independent lattices advanced together on the GPU.

    `lattices` is a list of (nx, ny, params) with a common storage.  Fields of
    lattice k are float32 arrays of shape (ny_k, nx_k).
    """

    def __init__(self, lattices, storage: int = STORAGE_FP32, stream=None, lib=None):
        import torch

        if not torch.cuda.is_available():
            raise RuntimeError("tpflbm needs a CUDA device; there is no CPU fallback")
        self.torch = torch
        self.lib = lib if lib is not None else load_library()
        self.n = len(lattices)
        self.sizes = [(int(nx), int(ny)) for nx, ny, _ in lattices]
        nxa = (C.c_int * self.n)(*[s[0] for s in self.sizes])
        nya = (C.c_int * self.n)(*[s[1] for s in self.sizes])
        pars = (Params * self.n)(*[make_params(p, storage) for _, _, p in lattices])
        h = C.c_void_p()
        rc = self.lib.tpflbm_batch_create(self.n, nxa, nya, pars, C.byref(h))
        if rc != 0:
            raise TpfError(rc, self.lib.tpflbm_batch_last_error(None).decode())
        self.h = h
        self.stream = stream
        if stream is not None:
            self._check(self.lib.tpflbm_batch_set_stream(self.h, C.c_void_p(stream.cuda_stream)))

    def _check(self, rc):
        if rc != 0:
            raise TpfError(rc, self.lib.tpflbm_batch_last_error(self.h).decode())

    def close(self):
        if getattr(self, "h", None):
            self.lib.tpflbm_batch_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def init(self, k, phi=None, ux=None, uy=None, p=None, T=None):
        nx, ny = self.sizes[k]
        arrs = [None if a is None else np.ascontiguousarray(np.broadcast_to(np.asarray(a, dtype=np.float32), (ny, nx)))
                for a in (phi, ux, uy, p, T)]
        self._check(self.lib.tpflbm_batch_init(self.h, int(k), *[_ptr(a) for a in arrs]))

    def step(self, n: int = 1):
        self._check(self.lib.tpflbm_batch_step(self.h, int(n)))

    @property
    def t(self) -> int:
        return int(self.lib.tpflbm_batch_time(self.h))

    def fields(self, k):
        nx, ny = self.sizes[k]
        out = [np.empty((ny, nx), dtype=np.float32) for _ in range(5)]
        self._check(self.lib.tpflbm_batch_get_fields(self.h, int(k), *[_ptr(a) for a in out]))
        return dict(zip(("phi", "ux", "uy", "p", "T"), out))

    def residual(self, dT):
        """(n, 3) array of (r_u, r_T, K) per lattice; dT a scalar or one per lattice."""
        d = np.broadcast_to(np.asarray(dT, dtype=np.float64), (self.n,)).copy()
        out = (C.c_double * (3 * self.n))()
        self._check(self.lib.tpflbm_batch_residual(self.h, d.ctypes.data_as(C.POINTER(C.c_double)), out))
        return np.array(out[:]).reshape(self.n, 3)

    def diagnostics(self):
        out = (C.c_double * (8 * self.n))()
        rc = self.lib.tpflbm_batch_diagnostics(self.h, out)
        if rc not in (0, -4):
            self._check(rc)
        return np.array(out[:]).reshape(self.n, 8), rc

    @staticmethod
    def variants(lib=None):
        lib = lib if lib is not None else load_library()
        cnt = C.c_int()
        lib.tpflbm_batch_variants(C.byref(cnt), None, None)
        bx = (C.c_int * cnt.value)()
        by = (C.c_int * cnt.value)()
        lib.tpflbm_batch_variants(C.byref(cnt), bx, by)
        return list(zip(bx[:], by[:]))

    @staticmethod
    def tma_variant(lib=None):
        """Index of the TMA-staged variant (the last one)."""
        return len(Batch.variants(lib)) - 1

    def set_variant(self, v: int):
        self._check(self.lib.tpflbm_batch_set_variant(self.h, int(v)))

    def tune(self, steps: int = 20):
        nv = len(self.variants(self.lib))
        ms = (C.c_double * nv)()
        best = C.c_int()
        self._check(self.lib.tpflbm_batch_tune(self.h, int(steps), ms, C.byref(best)))
        return best.value, list(ms[:])
