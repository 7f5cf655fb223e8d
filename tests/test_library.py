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
    assert o.refine_precision == mlcc.MLCC_FP64 and o.sigma_graph == 0


def test_binding_struct_sizes_match_header(lib):
    import ctypes
    from paper_2006_05226_gb300 import mlcc
    # layouts fixed by include/mlcc.h (natural alignment, no packing)
    assert ctypes.sizeof(mlcc.mlcc_problem) == 24
    assert ctypes.sizeof(mlcc.mlcc_dims) == 56
    assert ctypes.sizeof(mlcc.mlcc_options) == 80
    assert ctypes.sizeof(mlcc.mlcc_gs_info) == 32
    assert ctypes.sizeof(mlcc.mlcc_es_info) == 32
    assert ctypes.sizeof(mlcc.mlcc_request_result) == 112
    assert ctypes.sizeof(mlcc.mlcc_server_info) == 72
    assert ctypes.sizeof(mlcc.mlcc_result) == 64 + 7 * 8


def test_struct_layouts_match_the_header_compiled_with_gcc(lib, tmp_path):
    """Every field offset and struct size of the binding equals the C compiler's for
    include/mlcc.h."""
    import ctypes
    import json
    import shutil
    import subprocess
    from paper_2006_05226_gb300 import mlcc
    if shutil.which("gcc") is None:
        pytest.skip("gcc not available")
    structs = [mlcc.mlcc_problem, mlcc.mlcc_dims, mlcc.mlcc_options, mlcc.mlcc_gs_info, mlcc.mlcc_es_info,
               mlcc.mlcc_request_result, mlcc.mlcc_server_info, mlcc.mlcc_result, mlcc.mlcc_cnto_result]
    lines = ['#include <stdio.h>', '#include <stddef.h>', '#include "mlcc.h"', 'int main(void) {', 'printf("{");']
    for st in structs:
        n = st.__name__
        lines.append(f'printf("\\"{n}\\": [%zu", sizeof({n}));')
        for f, _ in st._fields_:
            lines.append(f'printf(", %zu", offsetof({n}, {f}));')
        lines.append('printf("],");')
    lines += ['printf("\\"end\\": 0}");', 'return 0; }']
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines))
    exe = tmp_path / "layout"
    subprocess.run(["gcc", "-std=c11", f"-I{os.path.join(ROOT, 'include')}", str(src), "-o", str(exe)], check=True)
    got = json.loads(subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout)
    for st in structs:
        want = [ctypes.sizeof(st)] + [getattr(st, f).offset for f, _ in st._fields_]
        assert got[st.__name__] == want, st.__name__


def test_problem_queries_without_a_device(lib):
    """mlcc_vector_len and mlcc_solve_footprint are host computations."""
    import numpy as np
    from paper_2006_05226_gb300 import mlcc
    from synth import CONFIGS
    from synth.generator import level_map
    for name, s in CONFIGS.items():
        lev = level_map(s.n_occ, s.n_vir, s.s_occ, s.s_vir, s.t_occ, s.t_vir)
        assert mlcc.vector_len(s.n_mo, s.n_occ, s.n_chol, lev) == s.n_vir * s.n_occ + (s.s_vir * s.s_occ) ** 2
        o64 = mlcc.default_options(n_roots=s.n_roots)
        omix = mlcc.default_options(n_roots=s.n_roots, precision=mlcc.MLCC_BF16X3, refine_fp64=1,
                                    refine_precision=mlcc.MLCC_FP64E)
        f64 = mlcc.solve_footprint(s.n_mo, s.n_occ, s.n_chol, lev, o64)
        fmix = mlcc.solve_footprint(s.n_mo, s.n_occ, s.n_chol, lev, omix)
        nn = s.n_mo ** 2
        # at least the Cholesky vectors and their dressed copy plus the Davidson basis and
        # sigma vectors (2 x 8 n_roots vectors), in whole 2 MiB pages
        dim = s.n_vir * s.n_occ + (s.s_vir * s.s_occ) ** 2
        assert f64 >= 8 * (2 * s.n_chol * nn + 16 * s.n_roots * dim)
        assert f64 % (2 << 20) == 0 and fmix >= f64
    lev = level_map(8, 40, 8, 40, 3, 12)
    a = mlcc.solve_footprint(48, 8, 200, lev)
    b = mlcc.solve_footprint(48, 8, 400, lev)
    assert b > a                                        # grows with the Cholesky count
    bad = np.array([0] * 47 + [3], dtype=np.int8)
    assert mlcc.vector_len(48, 8, 200, bad) == -1
    with pytest.raises(mlcc.MLCCError):
        mlcc.solve_footprint(48, 8, 200, bad)
    with pytest.raises(mlcc.MLCCError):
        mlcc.solve_footprint(48, 48, 200, lev)          # no virtual orbitals


def test_product_path_does_not_import_the_oracle():
    pkg = os.path.join(ROOT, "paper_2006_05226_gb300")
    for dirpath, _, files in os.walk(pkg):
        for f in files:
            if f.endswith((".py", ".cu", ".cuh", ".cpp", ".h")):
                text = open(os.path.join(dirpath, f)).read()
                assert "oracle" not in text.replace("oracle-", ""), f


def _header_enums():
    """name -> value of every enumerator in include/mlcc.h (the enums use explicit or
    implicit consecutive values)."""
    src = open(os.path.join(ROOT, "include", "mlcc.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    out = {}
    for body in re.findall(r"typedef\s+enum\s*\{(.*?)\}", src, flags=re.S):
        nxt = 0
        for item in body.split(","):
            item = item.strip()
            if not item:
                continue
            if "=" in item:
                name, val = (x.strip() for x in item.split("="))
                nxt = int(val, 0)
            else:
                name = item
            out[name] = nxt
            nxt += 1
    return out


def test_every_header_enum_has_a_binding_constant():
    from paper_2006_05226_gb300 import mlcc
    enums = _header_enums()
    assert "MLCC_E_STATE" in enums and "MLCC_PENDING" in enums and len(enums) >= 20
    for name, val in enums.items():
        assert hasattr(mlcc, name), f"binding lacks {name}"
        assert getattr(mlcc, name) == val, (name, getattr(mlcc, name), val)
    # the status table names every status code the header declares
    for name, val in enums.items():
        if name.startswith("MLCC_E_") or name in ("MLCC_OK", "MLCC_PENDING"):
            assert mlcc.STATUS[val] == name
