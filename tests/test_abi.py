"""The C-ABI library loads and exports every entry point include/hm.h declares
(no GPU needed: nothing is called)."""
import ctypes
import os
import re

from conftest import ROOT


def declared_functions():
    src = open(os.path.join(ROOT, "include", "hm.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    names = re.findall(r"\b(hm_[a-z0-9_]+)\s*\(", src)
    return sorted(set(names))


def test_header_declares_core_entry_points():
    names = declared_functions()
    for n in ("hm_build", "hm_matvec", "hm_free", "hm_last_error", "hm_build_ex",
              "hm_matvec_ex", "hm_cg", "hm_build_batch", "hm_matvec_batch"):
        assert n in names


def test_library_exports_every_declared_symbol():
    from paper_1708_09707_gb300 import build, hm
    build.build()
    L = hm.lib()
    missing = [n for n in declared_functions() if not hasattr(L, n)]
    assert not missing, missing


def test_options_and_stats_layout():
    from paper_1708_09707_gb300 import hm
    o = hm.options()
    assert o.k_cap == 64 and o.precision == hm.PREC_FP64
    # struct sizes match the C layout (offsets are natural alignment)
    assert ctypes.sizeof(hm.Options) == 80
    assert ctypes.sizeof(hm.Stats) == (8 * 5 + 4 * 2 + 8 + 8 + 8 * 9 + 8 * 4 + 4 * 3 + 4
                                       + 8 + 8 + 8 + 8 * 4 + 8 * 2 + 8 * 12 + 8 * 3)


def test_library_is_not_a_cpu_fallback():
    # the product path has no CPU implementation: the binding refuses to run
    # without the compiled library
    from paper_1708_09707_gb300 import hm
    src = open(hm.__file__).read()
    assert "oracle" not in src
