"""The C-ABI library builds, loads and exports every symbol declared in include/mgx.h (no GPU)."""
import os
import re
import ctypes

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "mgx.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(mgx_[a-z_0-9]+)\s*\(", src)))


@pytest.fixture(scope="module")
def libpath():
    from paper_2503_21935_gb300 import build
    return build.build()


def test_exports_every_declared_symbol(libpath):
    L = ctypes.CDLL(libpath)
    names = _declared()
    assert "mgx_compute" in names and "mgx_process_create" in names
    assert "mgx_compute_noalloc" in names and "mgx_noalloc_scratch_bytes" in names
    for n in names:
        assert hasattr(L, n), n


def test_binding_covers_every_declared_symbol(libpath):
    """The Python binding sets a signature for every entry point the header declares."""
    import paper_2503_21935_gb300 as pkg
    L = pkg.lib()
    for n in _declared():
        assert getattr(L, n).argtypes is not None or getattr(L, n).restype is not ctypes.c_int, n


def test_host_only_calls(libpath):
    import paper_2503_21935_gb300 as pkg
    assert pkg.lib().mgx_version() >= 100
    assert "g g > t t~ g g" in pkg.builtin_processes()
    p = pkg.default_params()
    assert abs(p.mt - 173.0) < 1e-12 and abs(p.alpha_em - 1 / 132.507) < 1e-15
    assert pkg.lib().mgx_status_string(-2) == b"unknown process"
    # argument validation happens before any device call
    h = ctypes.c_void_p()
    assert pkg.lib().mgx_process_create(None, None, 0, 0, ctypes.byref(h)) == -1
    assert pkg.lib().mgx_compute(None, 10, None, None, None, None, None, None, None, 0, None, 0, None) == -1


def test_binding_constants_match_header():
    """Constants the binding repeats from include/mgx.h (sizes and enum values) equal the header's."""
    import paper_2503_21935_gb300 as pkg
    src = open(os.path.join(ROOT, "include", "mgx.h")).read()
    assert int(re.search(r"#define MGX_MOMENTS_BLOCKS (\d+)", src).group(1)) == pkg.MGX_MOMENTS_BLOCKS
    assert pkg.MGX_MOMENTS_LEN == 3 * (1 + pkg.MGX_MOMENTS_BLOCKS)
    assert re.search(r"MGX_KERNEL_HELICITY = 4, MGX_KERNEL_SPLIT = 5", src)
