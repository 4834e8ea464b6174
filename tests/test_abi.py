"""CPU-only checks of the C ABI boundary: the library builds, loads and
exports every entry point that include/blest.h declares."""
import os
import re
import subprocess

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "blest.h")


def _declared():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(blest_[a-z_0-9]+)\s*\(", text)))


def test_header_declares_the_boundary():
    names = _declared()
    for must in ["blest_build", "blest_bfs", "blest_msbfs", "blest_closeness", "blest_build_many",
                 "blest_bfs_many", "blest_load_model", "blest_last_timings", "blest_status_string",
                 "blest_destroy"]:
        assert must in names


def test_library_builds_and_exports_every_symbol():
    import __graft_entry__ as ge
    lib = ge._load_build_module().build()
    out = subprocess.run(["nm", "-D", "--defined-only", lib], capture_output=True, text=True, check=True).stdout
    exported = set(re.findall(r"\bT (blest_[a-z_0-9]+)", out))
    missing = [n for n in _declared() if n not in exported]
    assert not missing, f"declared but not exported: {missing}"


def test_binding_loads_and_matches_header():
    import paper_2606_05081_gb300 as blest
    assert set(blest.EXPORTED) >= set(_declared())
    assert blest._lib.blest_status_string(blest.OK) == b"ok"
    assert blest._lib.blest_status_string(blest.ERR_TIMEOUT) == b"device wait timed out"
    o = blest.default_opts()
    assert o.sigma == 8 and abs(o.eta - 10.0) < 1e-6 and o.udiv_threshold == 25000.0
    assert o.jaccard_window == 65536 and o.probe_switch == 1


def test_binding_rejects_bad_dtypes():
    import numpy as np

    import paper_2606_05081_gb300 as blest
    with pytest.raises(TypeError):
        blest.build(3, np.array([0, 1, 2, 2], np.int32), np.array([1, 0], np.int32))


def test_no_product_module_imports_oracle():
    """The library path never routes through the CPU oracle."""
    pkg = os.path.join(ROOT, "paper_2606_05081_gb300")
    for dirpath, _, files in os.walk(pkg):
        for f in files:
            if f.endswith((".py", ".cu", ".cuh", ".h", ".cpp")):
                src = open(os.path.join(dirpath, f)).read()
                assert "import oracle" not in src and "from oracle" not in src, f
                assert "bfs_oracle" not in src, f


def test_mlp_buffer_shapes_checked_before_the_c_call():
    """The C entry points cannot see buffer sizes, so the binding checks them
    (a wrong width would let the library write past a host array)."""
    b = pytest.importorskip("paper_2606_05081_gb300")
    assert b.MLP_NW == 1589 and b.NUM_CHOICES == 9
    X = np.zeros((3, 6), np.float32)
    with pytest.raises(ValueError):
        b.mlp_predict(np.zeros(1457, np.float32), X)
    with pytest.raises(ValueError):
        b.mlp_train(X, np.zeros((3, 5), np.float32), np.ones((3, 5), np.float32), np.zeros(b.MLP_NW, np.float32))
    with pytest.raises(ValueError):
        b.mlp_loss_grad(np.zeros((3, 5), np.float32), np.zeros((3, 9)), np.ones((3, 9)), np.zeros(b.MLP_NW))
    for c in range(b.NUM_CHOICES):
        m, k = b.choice_mode_batch(c)
        assert b.choice_of(m, k) == c


def test_ctypes_structs_match_the_header_layout(tmp_path):
    """Every struct of the boundary has the same size and field offsets in
    the C header (compiled by gcc) as in the ctypes binding."""
    import ctypes

    import paper_2606_05081_gb300 as blest
    pairs = {"blest_build_opts": blest.BuildOpts, "blest_info": blest.Info,
             "blest_level_log": blest.LevelLog, "blest_bvss_view": blest.BvssView,
             "blest_degree_report": blest.DegreeReport, "blest_scale_free_report": blest.ScaleFreeReport,
             "blest_msbfs_counters": blest.MsbfsStats}
    lines = ['#include <stdio.h>', '#include <stddef.h>', '#include "blest.h"', 'int main(void) {']
    for cname, cls in pairs.items():
        lines.append(f'printf("{cname} sizeof %zu\\n", sizeof({cname}));')
        for f, _ in cls._fields_:
            lines.append(f'printf("{cname} {f} %zu\\n", offsetof({cname}, {f}));')
    lines.append('return 0; }')
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines))
    exe = tmp_path / "layout"
    subprocess.run(["gcc", "-std=c11", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    got = {}
    for ln in subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout.splitlines():
        s, f, v = ln.split()
        got[(s, f)] = int(v)
    for cname, cls in pairs.items():
        assert got[(cname, "sizeof")] == ctypes.sizeof(cls), cname
        for f, _ in cls._fields_:
            assert got[(cname, f)] == getattr(cls, f).offset, (cname, f)
