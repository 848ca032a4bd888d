"""CPU checks of the C-ABI boundary: the library builds for sm_103a, loads, and
exports every entry point that include/tpflbm.h and include/tpfnet.h declare, each
with a binding signature (no compute calls)."""
import ctypes as C
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


HEADERS = ("tpflbm.h", "tpfnet.h")


def _declared(header=None):
    out = set()
    for h in ([header] if header else HEADERS):
        src = open(os.path.join(ROOT, "include", h)).read()
        src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
        out |= set(re.findall(r"\b((?:tpflbm|tpfnet)_[a-z_0-9]+)\s*\(", src))
    return sorted(out)


def test_header_declares_the_boundary():
    names = _declared()
    for n in ("tpflbm_create", "tpflbm_init", "tpflbm_step", "tpflbm_get_fields", "tpflbm_destroy",
              "tpflbm_batch_step", "tpfnet_conv3x3", "tpfnet_conv3x3_wgrad", "tpfnet_adam"):
        assert n in names


def test_library_exports_every_declared_symbol():
    from paper_2306_11320_gb300.build import build_library
    from paper_2306_11320_gb300.tpflbm import SIGNATURES as S1
    from paper_2306_11320_gb300.unet import SIGNATURES as S2

    SIGNATURES = dict(S1, **S2)

    path = build_library()
    try:
        lib = C.CDLL(path)
    except OSError as e:  # pragma: no cover - a CUDA runtime must be loadable
        pytest.fail("libtpflbm.so does not load: %s" % e)
    for n in _declared():
        assert hasattr(lib, n), n
        assert n in SIGNATURES, "binding lacks %s" % n


def test_params_struct_matches_header():
    """The ctypes mirror has the header's fields in the header's order."""
    from paper_2306_11320_gb300.tpflbm import Params

    src = open(os.path.join(ROOT, "include", "tpflbm.h")).read()
    body = src[src.index("typedef struct tpflbm_params {"):src.index("} tpflbm_params;")]
    names = re.findall(r"\b([A-Za-z_][A-Za-z_0-9]*)\s*[,;]", body)
    assert [f[0] for f in Params._fields_] == names


def test_workspace_size_rejects_bad_sizes():
    from paper_2306_11320_gb300.tpflbm import load_library, make_params
    from paper_2306_11320_gb300 import workloads as WL

    lib = load_library()
    p = make_params(WL.base_params())
    assert lib.tpflbm_workspace_bytes(2, 64, C.byref(p)) == 0
    n = lib.tpflbm_workspace_bytes(64, 64, C.byref(p))
    # 2 x 27 float planes at least
    assert n >= 2 * 27 * 64 * 64 * 4
    p16 = make_params(WL.base_params(storage=1))
    assert lib.tpflbm_workspace_bytes(64, 64, C.byref(p16)) < n
    bad = make_params(WL.base_params(mu_l=-1.0))
    assert lib.tpflbm_workspace_bytes(64, 64, C.byref(bad)) == 0
    # rho c_p < 1 makes the weight (1 - 1/(rho c_p)) of Eq. 28 negative: rejected
    low = make_params(WL.base_params(rho_l=0.5, cp_l=1.0))
    assert lib.tpflbm_workspace_bytes(64, 64, C.byref(low)) == 0
    ok = make_params(WL.base_params(rho_l=0.5, cp_l=2.0))
    assert lib.tpflbm_workspace_bytes(64, 64, C.byref(ok)) > 0


def test_bounded_wait_check_rejects_bad_arguments():
    """tpflbm_check_bounded_wait validates its arguments before any CUDA call."""
    from paper_2306_11320_gb300.tpflbm import load_library

    lib = load_library()
    out = C.c_int(7)
    assert lib.tpflbm_check_bounded_wait(0, C.byref(out)) == -1  # TPF_ERR_INVALID_ARG
    assert b"polls" in lib.tpflbm_last_error(None)
    assert lib.tpflbm_check_bounded_wait(16, None) == -1
