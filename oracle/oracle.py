"""ctypes front end of the FP64 CPU oracle (``tpflbm_oracle.c``).

TEST INFRASTRUCTURE: the slow, plain definition of one time step of the three
coupled D2Q9 lattice Boltzmann equations of arXiv 2306.11320 (Sec. 3 and 4),
used to check the CUDA path.  Only tests, the smoke check and the benchmark's
CPU-baseline leg may use it.  It does not import the CUDA package.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import sys

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "tpflbm_oracle.c")
_LIBS = {"double": os.path.join(_HERE, "_build", "libtpflbm_oracle.so"),
         "float": os.path.join(_HERE, "_build", "libtpflbm_oracle_f32.so")}
_LIB = _LIBS["double"]

_PARAM_DOUBLES = [
    "rho_l", "rho_h", "mu_l", "mu_h", "lambda_l", "lambda_h", "cp_l", "cp_h",
    "W", "M_phi",
    "sigma_ref", "sigma_T", "sigma_TT", "T_ref",
    "Gx", "Gy",
    "u_ave", "phi_in", "T_in", "p_out",
    "T_bot", "T_bot_amp", "T_bot_k", "T_bot_slope", "T_top", "T_top_slope",
    "trt_lambda",
]
_PARAM_INTS = ["sigma_law", "bc_x", "bc_y", "normal_law", "collision"]


class OrcParams(C.Structure):
    _fields_ = [(n, C.c_double) for n in _PARAM_DOUBLES] + [(n, C.c_int) for n in _PARAM_INTS]


def build_oracle(force: bool = False, real: str = "double") -> str:
    """Compile the oracle with gcc (OpenMP over rows) into oracle/_build.

    real="double" is the reference.  real="float" builds the same source in float32
    arithmetic; it only serves to measure the float32 rounding floor of the method."""
    lib = _LIBS[real]
    os.makedirs(os.path.dirname(lib), exist_ok=True)
    if not force and os.path.exists(lib) and os.path.getmtime(lib) >= os.path.getmtime(_SRC):
        return lib
    tmp = lib + ".%d.tmp" % os.getpid()
    cmd = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-fopenmp", "-o", tmp, _SRC, "-lm"]
    if real == "float":
        cmd[1:1] = ["-DORACLE_REAL=float", "-fsingle-precision-constant"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, lib)
    return lib


_lib = None
_lib32 = None


def _sim_signatures(lib):
    dp = C.POINTER(C.c_double)
    vp = C.c_void_p
    lib.orc_create.argtypes = [C.c_int, C.c_int, C.POINTER(OrcParams), C.POINTER(vp)]
    lib.orc_create.restype = C.c_int
    lib.orc_destroy.argtypes = [vp]
    lib.orc_init.argtypes = [vp, dp, dp, dp, dp, dp]
    lib.orc_init.restype = C.c_int
    lib.orc_step.argtypes = [vp, C.c_longlong]
    lib.orc_step.restype = C.c_int
    lib.orc_get_fields.argtypes = [vp, dp, dp, dp, dp, dp]
    lib.orc_get_state.argtypes = [vp, dp, dp, dp, dp]
    lib.orc_set_state.argtypes = [vp, dp, dp, dp, dp]
    lib.orc_get_aux.argtypes = [vp, dp]
    lib.orc_time.argtypes = [vp]
    lib.orc_time.restype = C.c_longlong
    lib.orc_num_threads.restype = C.c_int
    lib.orc_set_num_threads.argtypes = [C.c_int]


def _load32():
    global _lib32
    if _lib32 is None:
        lib = C.CDLL(build_oracle(real="float"))
        _sim_signatures(lib)
        _lib32 = lib
    return _lib32


def _load():
    global _lib
    if _lib is None:
        lib = C.CDLL(build_oracle())
        dp = C.POINTER(C.c_double)
        _sim_signatures(lib)
        lib.orc_feq.argtypes = [C.c_double] * 3 + [dp]
        lib.orc_Ri.argtypes = [C.c_double] * 6 + [dp]
        lib.orc_geq.argtypes = [C.c_double] * 4 + [dp]
        lib.orc_Gi.argtypes = [C.c_double] * 6 + [dp]
        lib.orc_heq.argtypes = [C.c_double, dp]
        lib.orc_Fhat_i.argtypes = [C.c_double, dp]
        lib.orc_interp.argtypes = [C.c_double] * 3
        lib.orc_interp.restype = C.c_double
        lib.orc_mu_phi.argtypes = [C.c_double] * 3
        lib.orc_mu_phi.restype = C.c_double
        lib.orc_Fs.argtypes = [C.c_double] * 7 + [dp, dp]
        lib.orc_lattice.argtypes = [C.POINTER(C.c_int), C.POINTER(C.c_int), dp, C.POINTER(C.c_int)]
        _lib = lib
    return _lib


def _dp(a: np.ndarray):
    return a.ctypes.data_as(C.POINTER(C.c_double))


def _params(p: dict) -> OrcParams:
    s = OrcParams()
    for n in _PARAM_DOUBLES:
        setattr(s, n, float(p.get(n, 0.0)))
    for n in _PARAM_INTS:
        setattr(s, n, int(p.get(n, 0)))
    return s


def set_threads(n: int) -> None:
    _load().orc_set_num_threads(int(n))


def num_threads() -> int:
    return int(_load().orc_num_threads())


def lattice():
    """(ex, ey, w, opp) of the oracle's D2Q9 set."""
    lib = _load()
    ex = (C.c_int * 9)()
    ey = (C.c_int * 9)()
    w = (C.c_double * 9)()
    opp = (C.c_int * 9)()
    lib.orc_lattice(ex, ey, w, opp)
    return np.array(ex), np.array(ey), np.array(w), np.array(opp)


class node_ops:
    """Per-node operators of the oracle, exposed for the moment-identity pins."""

    @staticmethod
    def _call9(fn, *args):
        out = np.zeros(9)
        fn(*[float(a) for a in args], _dp(out))
        return out

    @staticmethod
    def feq(phi, ux, uy):
        return node_ops._call9(_load().orc_feq, phi, ux, uy)

    @staticmethod
    def Ri(phi, dphiux, dphiuy, nx, ny, W):
        return node_ops._call9(_load().orc_Ri, phi, dphiux, dphiuy, nx, ny, W)

    @staticmethod
    def geq(p, rho, ux, uy):
        return node_ops._call9(_load().orc_geq, p, rho, ux, uy)

    @staticmethod
    def Gi(ux, uy, grx, gry, Fx, Fy):
        return node_ops._call9(_load().orc_Gi, ux, uy, grx, gry, Fx, Fy)

    @staticmethod
    def heq(T):
        return node_ops._call9(_load().orc_heq, T)

    @staticmethod
    def Fhat_i(F):
        return node_ops._call9(_load().orc_Fhat_i, F)

    @staticmethod
    def interp(phi, a_l, a_h):
        return float(_load().orc_interp(float(phi), float(a_l), float(a_h)))

    @staticmethod
    def mu_phi(phi, lap, W):
        return float(_load().orc_mu_phi(float(phi), float(lap), float(W)))

    @staticmethod
    def Fs(W, sigma, gsx, gsy, mu_phi, gpx, gpy):
        fx = C.c_double()
        fy = C.c_double()
        _load().orc_Fs(float(W), float(sigma), float(gsx), float(gsy), float(mu_phi),
                       float(gpx), float(gpy), C.byref(fx), C.byref(fy))
        return fx.value, fy.value


class OracleSim:
    """One lattice of nx x ny nodes advanced by the FP64 oracle (real="float": the
    same algorithm in float32, for the rounding-floor measurement only).

    Fields are numpy arrays of shape (ny, nx), row-major, y = 0 the bottom row.
    """

    def __init__(self, nx: int, ny: int, params: dict, real: str = "double"):
        self.lib = _load() if real == "double" else _load32()
        self.nx, self.ny = int(nx), int(ny)
        self._p = _params(params)
        h = C.c_void_p()
        rc = self.lib.orc_create(self.nx, self.ny, C.byref(self._p), C.byref(h))
        if rc != 0:
            raise ValueError("orc_create failed (%d) for %dx%d" % (rc, nx, ny))
        self.h = h

    def __del__(self):
        if getattr(self, "h", None):
            self.lib.orc_destroy(self.h)
            self.h = None

    def _field(self, a):
        a = np.ascontiguousarray(a, dtype=np.float64)
        if a.shape != (self.ny, self.nx):
            a = np.broadcast_to(a, (self.ny, self.nx)).copy()
        return a

    def init(self, phi, ux, uy, p, T):
        arrs = [self._field(a) for a in (phi, ux, uy, p, T)]
        self.lib.orc_init(self.h, *[_dp(a) for a in arrs])

    def step(self, n: int = 1):
        self.lib.orc_step(self.h, int(n))

    @property
    def t(self) -> int:
        return int(self.lib.orc_time(self.h))

    def fields(self):
        out = [np.zeros((self.ny, self.nx)) for _ in range(5)]
        self.lib.orc_get_fields(self.h, *[_dp(a) for a in out])
        return dict(zip(("phi", "ux", "uy", "p", "T"), out))

    def aux(self):
        """Per-node quantities of the macroscopic pass on the current state: density,
        heat capacitance, thermal source, interfacial force, relaxation times, interface
        normal and density gradient."""
        out = np.zeros((11, self.ny, self.nx))
        self.lib.orc_get_aux(self.h, _dp(out))
        return dict(zip(("rho", "rcp", "Fhat", "Fx", "Fy", "tau_g", "tau_h", "nx", "ny", "grx", "gry"), out))

    def get_state(self):
        f = np.zeros((9, self.ny, self.nx))
        g = np.zeros_like(f)
        h = np.zeros_like(f)
        pu = np.zeros((2, self.ny, self.nx))
        self.lib.orc_get_state(self.h, _dp(f), _dp(g), _dp(h), _dp(pu))
        return {"f": f, "g": g, "h": h, "phiu": pu}

    def set_state(self, st):
        arrs = [np.ascontiguousarray(st[k], dtype=np.float64) for k in ("f", "g", "h", "phiu")]
        self.lib.orc_set_state(self.h, *[_dp(a) for a in arrs])
