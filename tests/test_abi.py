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


def _c_layout():
    import os
    import subprocess
    import tempfile
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    src = r"""
#include <stddef.h>
#include <stdio.h>
#include "hm.h"
int main(void) {
    printf("sizeof_options %zu\n", sizeof(hm_options));
    printf("off_stream %zu\n", offsetof(hm_options, stream));
    printf("off_on_the_fly %zu\n", offsetof(hm_options, on_the_fly));
    printf("off_row_lo %zu\n", offsetof(hm_options, row_lo));
    printf("off_row_hi %zu\n", offsetof(hm_options, row_hi));
    printf("sizeof_stats %zu\n", sizeof(hm_stats));
    printf("soff_t_aca_class_ms %zu\n", offsetof(hm_stats, t_aca_class_ms));
    printf("soff_t_np_near_ms %zu\n", offsetof(hm_stats, t_np_near_ms));
    printf("soff_traversal_reruns %zu\n", offsetof(hm_stats, traversal_reruns));
    printf("soff_t_mvp_tail_ms %zu\n", offsetof(hm_stats, t_mvp_tail_ms));
    printf("soff_mvp_tail_bytes %zu\n", offsetof(hm_stats, mvp_tail_bytes));
    return 0;
}
"""
    with tempfile.TemporaryDirectory() as d:
        c = os.path.join(d, "layout.c")
        exe = os.path.join(d, "layout")
        open(c, "w").write(src)
        subprocess.run(["gcc", "-I", os.path.join(root, "include"), c, "-o", exe], check=True)
        out = subprocess.run([exe], capture_output=True, text=True, check=True).stdout
    return {k: int(v) for k, v in (line.split() for line in out.splitlines())}


def test_options_and_stats_layout():
    from paper_1708_09707_gb300 import hm
    o = hm.options()
    assert o.k_cap == 64 and o.precision == hm.PREC_FP64
    # struct sizes and offsets match the C layout, as the C compiler lays it out
    c = _c_layout()
    assert ctypes.sizeof(hm.Options) == c["sizeof_options"] == 96
    for f in ("stream", "on_the_fly", "row_lo", "row_hi"):
        assert getattr(hm.Options, f).offset == c["off_" + f], f
    assert ctypes.sizeof(hm.Stats) == c["sizeof_stats"] == (
        8 * 5 + 4 * 2 + 8 + 8 + 8 * 9 + 8 * 4 + 4 * 3 + 4 + 8 + 8 + 8 + 8 * 4 + 8 * 2 + 8 * 12
        + 8 * 3 + 8 + 8 + 8)
    for f in ("t_aca_class_ms", "t_np_near_ms", "traversal_reruns", "t_mvp_tail_ms",
              "mvp_tail_bytes"):
        assert getattr(hm.Stats, f).offset == c["soff_" + f], f


def test_library_is_not_a_cpu_fallback():
    # the product path has no CPU implementation: the binding refuses to run
    # without the compiled library
    from paper_1708_09707_gb300 import hm
    src = open(hm.__file__).read()
    assert "oracle" not in src


def test_test_hook_ranges_without_a_gpu():
    # hm_set_test_hook only records process-wide settings: no device call
    from paper_1708_09707_gb300 import build, hm
    build.build()
    L = hm.lib()
    assert L.hm_set_test_hook(hm.HOOK_TRAVERSAL_KAPPA, -1) == hm.EINVAL
    assert L.hm_set_test_hook(hm.HOOK_TRAVERSAL_KAPPA, (1 << 20) + 1) == hm.EINVAL
    assert L.hm_set_test_hook(hm.HOOK_TRAVERSAL_TRIES, 65) == hm.EINVAL
    assert L.hm_set_test_hook(99, 1) == hm.EINVAL
    for hook in (hm.HOOK_TRAVERSAL_KAPPA, hm.HOOK_TRAVERSAL_TRIES):
        assert L.hm_set_test_hook(hook, 3) == hm.OK
        assert L.hm_set_test_hook(hook, 0) == hm.OK


def test_batch_limits_without_a_gpu():
    from paper_1708_09707_gb300 import build, hm
    build.build()
    L = hm.lib()
    assert L.hm_set_batch_limits(-1, 0) == hm.EINVAL
    assert L.hm_set_batch_limits(0, -5) == hm.EINVAL
    assert L.hm_set_batch_limits(1 << 20, 16) == hm.OK
    assert L.hm_set_batch_limits(0, 0) == hm.OK
