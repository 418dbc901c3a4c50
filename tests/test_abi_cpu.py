"""C-ABI checks that need no GPU: the library builds and loads, exports
every function declared in include/*.h, and its host-only logic (tuple
counts, option defaults, argument validation) behaves as documented."""

import ctypes
import glob
import math
import os
import re

import pytest

import paper_2502_20072_gb300 as l0

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared_functions():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        src = open(h).read()
        src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
        src = re.sub(r"//[^\n]*", "", src)
        for m in re.finditer(r"\b(sisso_l0_\w+)\s*\(", src):
            names.add(m.group(1))
    return names


def test_library_exports_every_declared_function():
    L = l0.lib()
    declared = _declared_functions()
    assert "sisso_l0_fit" in declared and "sisso_l0_create" in declared
    for name in sorted(declared):
        assert hasattr(L, name), name
    assert set(l0.EXPORTS) <= declared


def test_default_options_struct_size_matches_binding():
    o = l0.Options()
    assert l0.lib().sisso_l0_default_options(ctypes.byref(o)) == 0
    assert o.struct_size == ctypes.sizeof(l0.Options)
    assert o.precision == l0.FP64 and o.task_mode == l0.PER_TASK
    assert o.fp32_fallback_pivot_ratio == 1e-6
    assert o.rank_deficient_pivot_ratio == 1e-12


@pytest.mark.parametrize("m,n", [(5, 0), (5, 1), (10, 3), (200, 2), (1000, 3), (400, 4),
                                 (20000, 3), (60, 8)])
def test_count_tuples_is_binomial(m, n):
    assert l0.count_tuples(m, n) == math.comb(m, n)


def test_count_tuples_paper_counts():
    # Sec. 3.1.1 and 3.1.2 state these model counts
    assert l0.count_tuples(5000, 3) == 20820835000
    assert l0.count_tuples(50000, 2) == 1249975000


def test_count_tuples_overflow_is_zero():
    assert l0.count_tuples(10 ** 9, 8) == 0


def test_null_and_bad_arguments_rejected_without_device():
    L = l0.lib()
    assert L.sisso_l0_create(None, None) == l0.EINVAL
    assert L.sisso_l0_fit(None, None, None, None, 1, 10, 2, 1, None, None) == l0.EINVAL
    assert L.sisso_l0_get_stats(None, None) == l0.EINVAL
    assert L.sisso_l0_last_error(None) == b"null handle"
    L.sisso_l0_destroy(None)   # NULL-safe
    o = l0.Options()
    L.sisso_l0_default_options(ctypes.byref(o))
    o.struct_size = 12
    h = ctypes.c_void_p()
    assert L.sisso_l0_create(ctypes.byref(h), ctypes.byref(o)) == l0.EINVAL
