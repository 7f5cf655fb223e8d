"""The C-ABI library builds, loads and exports every entry point include/mlcc.h declares
(no GPU needed: nothing here launches a kernel)."""
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "mlcc.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(mlcc_[a-z0-9_]+)\s*\(", src)))


@pytest.fixture(scope="module")
def lib():
    from paper_2006_05226_gb300 import mlcc
    if not os.path.exists(mlcc.LIB_PATH):
        from paper_2006_05226_gb300 import build
        build.build()
    return mlcc.load()


def test_every_declared_symbol_is_exported(lib):
    from paper_2006_05226_gb300 import mlcc
    names = _declared()
    assert len(names) >= 19
    missing = [n for n in names if not hasattr(lib, n)]
    assert not missing, missing
    assert sorted(mlcc.EXPORTS) == names


def test_default_options(lib):
    from paper_2006_05226_gb300 import mlcc
    o = mlcc.default_options()
    assert o.n_roots == 3 and o.diis_dim == 8 and o.precision == mlcc.MLCC_FP64
    assert o.gs_tol == 1e-11 and o.es_res_tol == 1e-8 and o.lowp_res_tol == 1e-4
    assert o.refine_precision == mlcc.MLCC_FP64 and o.reserved == 0


def test_binding_struct_sizes_match_header(lib):
    import ctypes
    from paper_2006_05226_gb300 import mlcc
    # layouts fixed by include/mlcc.h (natural alignment, no packing)
    assert ctypes.sizeof(mlcc.mlcc_problem) == 24
    assert ctypes.sizeof(mlcc.mlcc_dims) == 56
    assert ctypes.sizeof(mlcc.mlcc_options) == 80
    assert ctypes.sizeof(mlcc.mlcc_gs_info) == 32
    assert ctypes.sizeof(mlcc.mlcc_es_info) == 32


def test_product_path_does_not_import_the_oracle():
    pkg = os.path.join(ROOT, "paper_2006_05226_gb300")
    for dirpath, _, files in os.walk(pkg):
        for f in files:
            if f.endswith((".py", ".cu", ".cuh", ".cpp", ".h")):
                text = open(os.path.join(dirpath, f)).read()
                assert "oracle" not in text.replace("oracle-", ""), f
