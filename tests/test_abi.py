"""Host-side checks of the boundary: the library builds, loads, and exports
every entry point include/soft.h declares (no GPU needed, no compute call)."""
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def header_functions():
    txt = open(os.path.join(ROOT, "include", "soft.h")).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    names = re.findall(r"^\s*(?:[A-Za-z_][\w\s\*]*?)\b((?:soft|sse)_\w+)\s*\(", txt, flags=re.M)
    return sorted(set(names))


@pytest.fixture(scope="module")
def lib():
    from paper_1505_06707_gb300 import _build
    _build.build()
    import paper_1505_06707_gb300 as S
    return S.load()


def test_header_declares_the_paper_calls():
    names = header_functions()
    for n in ("soft_create", "soft_step", "sse_pcg_solve", "soft_create_batch", "soft_step_batch",
              "soft_observe", "soft_destroy"):
        assert n in names


def test_library_exports_every_declared_symbol(lib):
    import paper_1505_06707_gb300 as S
    names = header_functions()
    missing = [n for n in names if not hasattr(lib, n)]
    assert not missing, missing
    assert sorted(S.exported_symbols) == names


def test_strerror_and_defaults(lib):
    import ctypes as C
    import paper_1505_06707_gb300 as S
    assert lib.soft_strerror(0) == b"ok"
    assert b"power of two" in lib.soft_strerror(-2)
    o = S.Options()
    lib.soft_default_options(C.byref(o))
    assert o.prec == S.SOFT_C128 and o.band_width == 10 and o.soft_a2 == 2.0


def test_invalid_arguments_rejected_on_host(lib):
    """Argument checks run before any CUDA call, so they work without a GPU."""
    import paper_1505_06707_gb300 as S
    with pytest.raises(S.SoftError) as e:
        S.soft_create(1000, (-10.0, 10.0), 5.0, 0.5, 0.01)          # not a power of two
    assert e.value.status == -2
    with pytest.raises(S.SoftError) as e:
        S.soft_create(1024, (-10.0, 12.0), 5.0, 0.5, 0.01)          # asymmetric box
    assert e.value.status == -1
    with pytest.raises(S.SoftError) as e:
        S.soft_create(1024, (-10.0, 10.0), 11.0, 0.5, 0.01)         # R0 outside the box
    assert e.value.status == -1
    with pytest.raises(S.SoftError):
        S.soft_create(1024, (-10.0, 10.0), 5.0, 0.5, 0.0)           # dt = 0
