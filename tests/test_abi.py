"""CPU-only checks of the C ABI: the library loads, exports every entry point
include/cm.h declares, the ctypes structs match the C layout, and argument
errors are reported without touching a GPU."""
import ctypes
import os
import re
import subprocess

import pytest

import paper_2411_10372_gb300 as cm
from paper_2411_10372_gb300 import _binding as B

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "cm.h")


def declared_functions():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(cm_[a-z_0-9]+)\s*\(", src)))


def test_library_exports_every_declared_symbol():
    L = cm.lib()
    names = declared_functions()
    assert len(names) >= 20
    missing = [n for n in names if not hasattr(L, n)]
    assert missing == []
    # and the binding wraps every one of them under the same name
    assert [n for n in names if not hasattr(cm, n)] == []


def test_struct_layout_matches_c(tmp_path):
    probe = tmp_path / "probe.c"
    probe.write_text('''
#include <stdio.h>
#include <stddef.h>
#include "cm.h"
#define O(T, f) printf(#T "." #f " %zu\\n", offsetof(T, f))
int main(void) {
  printf("cm_grid %zu\\ncm_params %zu\\ncm_diag %zu\\n", sizeof(cm_grid), sizeof(cm_params), sizeof(cm_diag));
  O(cm_params, seed); O(cm_params, precision); O(cm_params, stream); O(cm_params, state_buf);
  O(cm_diag, status); O(cm_diag, mach_max); O(cm_grid, aspect); O(cm_grid, zstretch); O(cm_grid, znodes); O(cm_ext, r_max);
  return 0; }
''')
    exe = tmp_path / "probe"
    subprocess.run(["gcc", "-I", os.path.join(ROOT, "include"), str(probe), "-o", str(exe)], check=True)
    out = dict(line.rsplit(" ", 1) for line in subprocess.run([str(exe)], capture_output=True, text=True,
                                                             check=True).stdout.split("\n") if line)
    assert int(out["cm_grid"]) == ctypes.sizeof(B.cm_grid)
    assert int(out["cm_params"]) == ctypes.sizeof(B.cm_params)
    assert int(out["cm_diag"]) == ctypes.sizeof(B.cm_diag)
    for key, val in out.items():
        if "." in key:
            st, f = key.split(".")
            assert getattr(B, st).__dict__[f].offset == int(val), key


def test_default_params_and_state_bytes():
    p = cm.cm_default_params()
    assert p.eps == 0.1 and p.D == 0.5 and p.cfl == 0.5
    assert abs(p.t_top - 0.4) < 1e-15 and p.t_bot == 1.0
    assert abs(p.stokes + 2.0 / 3.0) < 1e-15 and p.tvd_form == cm.CM_TVD_DAVIS
    g = cm.cm_grid(2, 4096, 1, 1024, 4.0)
    assert cm.cm_state_bytes(g, cm.CM_FP32) == 2 * 4 * 1024 * 4096 * 4
    assert cm.cm_state_bytes(g, cm.CM_FP64) == 2 * 4 * 1024 * 4096 * 8
    g = cm.cm_grid(2, 250, 1, 64, 4.0)  # rows padded to 256 bytes
    assert cm.cm_state_bytes(g, cm.CM_FP64) == 2 * 4 * 64 * 256 * 8


def test_argument_errors_need_no_gpu():
    with pytest.raises(cm.CMError) as e:
        cm.cm_init(cm.cm_grid(2, 2, 1, 3, 4.0), 1e6, 1.0, 5 / 3)
    assert e.value.code == cm.CM_EINVAL
    with pytest.raises(cm.CMError) as e:
        cm.cm_init(cm.cm_grid(2, 64, 1, 16, 4.0), -1.0, 1.0, 5 / 3)
    assert e.value.code == cm.CM_EINVAL
    p = cm.cm_default_params()
    p.precision = 7
    with pytest.raises(cm.CMError) as e:
        cm.cm_init(cm.cm_grid(2, 64, 1, 16, 4.0), 1e6, 1.0, 5 / 3, p)
    assert e.value.code == cm.CM_EINVAL
    with pytest.raises(cm.CMError) as e:
        cm.cm_step(1)
    assert e.value.code == cm.CM_ENOTINIT
    assert cm.cm_state_ptr(0) == 0
    assert "cm_init" in cm.cm_last_error() or "no context" in cm.cm_last_error()


def test_stretched_grid_argument_errors_need_no_gpu():
    """The z-grid is validated before any device work: planes must run from
    exactly 0 to exactly 1 and increase; beta must be in [0, 20]; the batch
    checks each box's grid the same way, and cm_diag_noalloc its grid."""
    import numpy as np
    bad = [np.linspace(0, 1, 16) * 0.99, np.r_[0.0, 0.5, 0.3, np.linspace(0.6, 1, 13)],
           np.r_[1e-9, np.linspace(0.1, 1, 15)], np.r_[0.0, np.nan, np.linspace(0.2, 1, 14)]]
    for z in bad:
        g = cm.cm_grid(2, 64, 1, 16, 4.0, 0.0, z.ctypes.data_as(ctypes.POINTER(ctypes.c_double)))
        with pytest.raises(cm.CMError) as e:
            cm.cm_init(g, 1e6, 1.0, 5 / 3)
        assert e.value.code == cm.CM_EINVAL, z
    for beta in (-1.0, 25.0, float("nan")):
        with pytest.raises(cm.CMError) as e:
            cm.cm_init(cm.cm_grid(2, 64, 1, 16, 4.0, beta), 1e6, 1.0, 5 / 3)
        assert e.value.code == cm.CM_EINVAL, beta
    p = cm.cm_default_params()
    p.precision = cm.CM_FP32
    for beta in (-1.0, 25.0):
        with pytest.raises(cm.CMError) as e:
            cm.cm_batch_init([cm.cm_grid(2, 64, 1, 16, 4.0), cm.cm_grid(2, 64, 1, 16, 4.0, beta)], [1e6, 1e6], 1.0,
                             5 / 3, p)
        assert e.value.code == cm.CM_EINVAL and "box 1" in cm.cm_last_error(), beta
        with pytest.raises(cm.CMError) as e:  # rejected before the scratch array is touched
            cm.cm_diag_noalloc(1 << 20, cm.CM_FP32, cm.cm_grid(2, 64, 1, 16, 4.0, beta), 64, 1e6, 1.0, 5 / 3, p)
        assert e.value.code == cm.CM_EINVAL and "zstretch" in cm.cm_last_error(), beta


def test_missing_library_fails_loudly(monkeypatch, tmp_path):
    """No CPU fallback: without libcm.so the binding raises instead of
    computing anything."""
    from paper_2411_10372_gb300 import _binding as B
    monkeypatch.setattr(B, "_lib", None)
    monkeypatch.setattr(B, "LIB_PATH", str(tmp_path / "absent" / "libcm.so"))
    with pytest.raises(RuntimeError, match="missing"):
        B.lib(build_if_missing=False)
