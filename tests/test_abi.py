"""The C-ABI library builds for sm_103a, loads without a GPU, and exports every entry
point include/*.h declares; the Python binding's struct layouts match the C ones."""
import ctypes
import os
import re
import subprocess

import pytest

import paper_2009_07463_gb300 as gt
from paper_2009_07463_gb300 import native

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
INCLUDE = os.path.join(ROOT, "include")


def declared_symbols():
    names = []
    for f in sorted(os.listdir(INCLUDE)):
        if f.endswith(".h"):
            src = open(os.path.join(INCLUDE, f)).read()
            names += re.findall(r"GT_API\s+[\w\s\*]+?\b(gt_\w+)\s*\(", src)
    return names


def test_library_exports_declared_symbols():
    path = native.build()
    lib = ctypes.CDLL(path)
    names = declared_symbols()
    assert len(names) >= 15
    missing = [n for n in names if not hasattr(lib, n)]
    assert not missing, f"declared but not exported: {missing}"
    out = subprocess.run(["nm", "-D", "--defined-only", path], capture_output=True, text=True).stdout
    exported = set(re.findall(r" T (gt_\w+)", out))
    assert exported == set(names), f"exported but not declared: {exported - set(names)}"


def test_struct_layouts_match_header(tmp_path):
    prog = tmp_path / "sizes.c"
    prog.write_text('#include <stdio.h>\n#include <stddef.h>\n#include "gt.h"\n'
                    'int main(void){printf("%zu %zu %zu %zu %zu %zu\\n", sizeof(gt_config), sizeof(gt_tuning),'
                    ' sizeof(gt_stats), sizeof(gt_level_info), offsetof(gt_stats, mh), offsetof(gt_level_info, frontier));'
                    ' printf("%zu %zu %zu\\n", sizeof(gt_serve_config), offsetof(gt_serve_config, policy),'
                    ' sizeof(gt_serve_stats));'
                    ' return 0;}\n')
    exe = tmp_path / "sizes"
    subprocess.check_call(["gcc", "-std=c11", "-I", INCLUDE, str(prog), "-o", str(exe)])
    got = list(map(int, subprocess.check_output([str(exe)]).split()))
    want = [ctypes.sizeof(gt.gt_config), ctypes.sizeof(gt.gt_tuning), ctypes.sizeof(gt.gt_stats),
            ctypes.sizeof(gt.gt_level_info), gt.gt_stats.mh.offset, gt.gt_level_info.frontier.offset,
            ctypes.sizeof(gt.gt_serve_config), gt.gt_serve_config.policy.offset, ctypes.sizeof(gt.gt_serve_stats)]
    assert got == want


def test_defaults_and_errors_without_gpu():
    L = gt.lib()
    t = gt.tuning_default()
    assert (t.alpha, t.beta, t.td_warp_min, t.launch_mode, t.batch_alpha) == (32, 256, 32, 0, 14)
    assert (t.bu_thread_scan, t.bu_hub_first) == (24, 0)  # ascending bottom-up order by default
    assert L.gt_strerror(-1) == b"invalid argument"
    # argument checks fail before any device work
    h = ctypes.c_void_p()
    assert L.gt_graph_build(None, 5, 10, None, None, ctypes.byref(h)) == gt.GT_EINVAL
    assert L.gt_graph_build(None, 0, 0, None, None, ctypes.byref(h)) == gt.GT_EINVAL
    assert L.gt_bfs(None, 0, None, None, None) == gt.GT_EINVAL
    assert L.gt_bfs_roots(None, None, 0, None, None, None) == gt.GT_EINVAL
    assert b"n <= 2^31" in L.gt_last_error() or L.gt_last_error()
    # server configuration is checked before the server touches a device
    c = gt.gt_serve_config()
    L.gt_serve_config_default(ctypes.byref(c))
    assert (c.streams, c.max_batch_roots, c.policy, c.join_levels) == (4, 256, gt.GT_SERVE_ADAPTIVE, 0)
    c.policy = 3
    assert L.gt_serve_create(ctypes.byref(c), ctypes.byref(h)) == gt.GT_EINVAL
    c.policy = gt.GT_SERVE_ADAPTIVE
    c.join_levels = -1
    assert L.gt_serve_create(ctypes.byref(c), ctypes.byref(h)) == gt.GT_EINVAL


def test_no_cpu_fallback_in_binding():
    src = open(os.path.join(ROOT, "paper_2009_07463_gb300", "__init__.py")).read()
    assert "import oracle" not in src and "from oracle" not in src


def test_binding_checks_output_buffers():
    import numpy as np
    ok = np.zeros(10, dtype=np.int32)
    assert gt._out(ok, 10, "x") == ok.ctypes.data
    for bad in (np.zeros(9, dtype=np.int32), np.zeros(10, dtype=np.int64), np.zeros(20, dtype=np.int32)[::2]):
        with pytest.raises(ValueError):
            gt._out(bad, 10, "x")
    assert gt._out(None, 10, "x") == 0 and gt._out(1234, 10, "x") == 1234
