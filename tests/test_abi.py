"""The C ABI library loads and exports every function include/tmamg.h declares (no GPU needed)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "tmamg.h")


def declared():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(tmamg_[a-z0-9_]+)\s*\(", src)))


def test_header_declares_entry_points():
    names = declared()
    assert "tmamg_create" in names and "tmamg_dirac" in names


def test_library_exports_all_declared_symbols():
    from paper_2201_03872_gb300 import tmamg as T
    if not os.path.exists(T.LIB_PATH):
        import __graft_entry__
        __graft_entry__.build()
    lib = ctypes.CDLL(T.LIB_PATH)
    missing = [n for n in declared() if not hasattr(lib, n)]
    assert not missing, missing
    # the Python binding wraps every declared entry point under the same name
    assert set(declared()) <= set(T.SIGNATURES), set(declared()) - set(T.SIGNATURES)


def test_binding_refuses_without_library(tmp_path, monkeypatch):
    from paper_2201_03872_gb300 import tmamg as T
    monkeypatch.setattr(T, "LIB_PATH", str(tmp_path / "missing.so"))
    monkeypatch.setattr(T, "_lib", None)
    with pytest.raises(ImportError):
        T.lib()


def _c_layout(tmp_path):
    """Offsets and sizes of the parameter structs as the C compiler lays them out from the header."""
    import shutil
    import subprocess
    cc = shutil.which("gcc") or shutil.which("cc")
    if not cc:
        pytest.skip("no C compiler")
    fields = {
        "tmamg_setup_params": ["levels", "agg", "nv", "sap_block", "sap_cycles", "sap_mr_steps", "setup_iters",
                               "mu_setup", "seed", "setup_gmres_steps"],
        "tmamg_solve_params": ["tol", "restart", "max_outer", "coarse_tol", "coarse_restart", "coarse_maxiter",
                               "coarse_solver", "delta_mu", "precision", "use_nn", "poll", "coarse_precision",
                               "mid_tol", "mid_restart", "mid_maxiter", "mid_smooth", "inner_cycles", "sap_cycles",
                               "sap_mr_steps"],
        "tmamg_system_stats": ["status", "outer_iters", "inner_iters", "coarse_iters", "true_rel_res"],
        "tmamg_nn_params": ["pairs", "batch", "epochs", "lr", "pair_tol", "mu", "seed", "gate_systems",
                            "window"],
        "tmamg_nn_report": ["loss_first", "loss_last", "iters_plain", "iters_nn", "enabled"],
    }
    lines = ['#include <stdio.h>', '#include <stddef.h>', f'#include "{HEADER}"', "int main(void) {"]
    for st, fs in fields.items():
        lines.append(f'  printf("{st} sizeof %zu\\n", sizeof({st}));')
        for f in fs:
            lines.append(f'  printf("{st} {f} %zu\\n", offsetof({st}, {f}));')
    lines.append("  return 0;\n}")
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines))
    exe = tmp_path / "layout"
    subprocess.run([cc, "-std=c99", "-o", str(exe), str(src)], check=True, capture_output=True)
    out = subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout
    table = {}
    for line in out.splitlines():
        st, f, v = line.split()
        table[(st, f)] = int(v)
    return fields, table


def test_binding_structs_match_the_header(tmp_path):
    # the ctypes mirrors of the parameter structs must have the C layout field by field
    from paper_2201_03872_gb300 import tmamg as T
    fields, table = _c_layout(tmp_path)
    mirrors = {"tmamg_setup_params": T.SetupParams, "tmamg_solve_params": T.SolveParams,
               "tmamg_system_stats": T.SystemStats, "tmamg_nn_params": T.NNParams, "tmamg_nn_report": T.NNReport}
    for st, cls in mirrors.items():
        assert ctypes.sizeof(cls) == table[(st, "sizeof")], st
        assert [f[0] for f in cls._fields_] == fields[st], st
        for f in fields[st]:
            assert getattr(cls, f).offset == table[(st, f)], (st, f)


def test_default_parameters():
    # host-only entry points: the defaults of the paper's configuration (Sec. 4: FGMRES at the top to 1e-10,
    # r_b = 0.1 at the bottom, r_m = 7e-2 on the middle level)
    from paper_2201_03872_gb300 import tmamg as T
    if not os.path.exists(T.LIB_PATH):
        import __graft_entry__
        __graft_entry__.build()
    sp = T.tmamg_default_solve_params()
    assert sp.tol == 1e-10 and sp.coarse_tol == 0.1 and sp.mid_tol == 7e-2
    assert (sp.restart, sp.mid_restart, sp.mid_maxiter, sp.mid_smooth) == (10, 10, 50, 3)
    assert sp.precision == 32 and sp.coarse_precision == 16 and sp.delta_mu == 1.0
    p = T.tmamg_default_setup_params()
    assert p.levels == 2 and list(p.agg[0]) == [4, 4, 4, 4] and list(p.agg[1]) == [2, 2, 2, 2]
    assert (p.nv[0], p.nv[1], p.setup_gmres_steps) == (24, 32, 20)
    q = T.setup_params(levels=3, agg=(2, 2, 2, 2), nv=8, agg2=(1, 2, 2, 2), nv2=12, setup_gmres_steps=7)
    assert q.levels == 3 and list(q.agg[1]) == [1, 2, 2, 2] and q.nv[1] == 12 and q.setup_gmres_steps == 7
