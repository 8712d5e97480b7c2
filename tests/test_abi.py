"""The C-ABI library builds, loads and exports every declared symbol; host-side
argument validation (no GPU needed)."""
import ctypes

import numpy as np
import pytest

import paper_1207_5558_gb300 as pkg
from paper_1207_5558_gb300 import _abi


@pytest.fixture(scope="module")
def lib():
    from paper_1207_5558_gb300 import build
    build.build()
    return _abi.load()


def test_exports_every_declared_symbol(lib):
    names = _abi.header_functions()
    assert len(names) >= 15
    for n in names:
        assert hasattr(lib, n), n
    # and nothing in the library named slsht_* is undeclared in the header
    import subprocess
    out = subprocess.run(["nm", "-D", "--defined-only", _abi.LIB_PATH], capture_output=True, text=True).stdout
    exported = sorted({ln.split()[-1] for ln in out.splitlines() if " T slsht_" in ln})
    assert exported == names


def test_strerror_and_version(lib):
    assert pkg.slsht_strerror(0) == "ok"
    assert "h_0^0" in pkg.slsht_strerror(_abi.SLSHT_E_H00)
    assert pkg.slsht_strerror(12345) == "unknown status code"
    assert "sm_103a" in pkg.slsht_version()


def test_check_args(lib):
    d = pkg.make_desc(16, 4, (31, 16, 7))
    ok = np.array([[0, 0], [17, -17], [15, 3]], dtype=np.int32)
    assert pkg.slsht_check_args(d, ok, 3) == 0
    for bad in ([[19, 0]], [[3, 4]], [[-1, 0]], [[5, -6]]):
        assert pkg.slsht_check_args(d, np.array(bad, np.int32), 1) == _abi.SLSHT_E_ARG
    assert pkg.slsht_check_args(d, ok, -1) == _abi.SLSHT_E_ARG
    for desc in [pkg.make_desc(0, 4, (3, 3, 3)), pkg.make_desc(4, 0, (3, 3, 3)),
                 pkg.make_desc(4, 65, (3, 3, 3)), pkg.make_desc(4, 2, (0, 3, 3)),
                 pkg.make_desc(4, 2, (3, 3, 3), prec=7)]:
        assert pkg.slsht_check_args(desc, ok[:1], 1) == _abi.SLSHT_E_ARG
    assert pkg.slsht_check_args(pkg.make_desc(1, 1, (1, 1, 1)), np.zeros((1, 2), np.int32), 1) == 0


def test_null_context_is_rejected(lib):
    assert lib.slsht_forward(None, None, None, None, None, 0, None, None) == _abi.SLSHT_E_ARG
    assert lib.slsht_poll(None, ctypes.c_uint64(1)) == _abi.SLSHT_E_ARG
    lib.slsht_destroy(None)
