"""The C-ABI library builds, loads and exports every function include/teuk.h
declares; the ctypes structs match the C layout; host-side validation works
without a GPU (no compute is launched here)."""
import ctypes
import os
import subprocess
import sys

import pytest

import paper_1001_3631_gb300 as P
from paper_1001_3631_gb300 import _lib


@pytest.fixture(scope="module")
def lib():
    from paper_1001_3631_gb300 import build
    build.build()
    return _lib.load()


def test_exports_every_declared_function(lib):
    names = _lib.header_functions()
    assert len(names) >= 13
    for n in names:
        assert hasattr(lib, n), n
    # nm confirms they are real dynamic exports
    out = subprocess.run(["nm", "-D", "--defined-only", _lib.LIB_PATH], capture_output=True,
                         text=True).stdout
    for n in names:
        assert (" T " + n) in out, n
    # the checked build exports the same functions
    chk = os.path.join(os.path.dirname(_lib.LIB_PATH), "libteuk_check.so")
    out = subprocess.run(["nm", "-D", "--defined-only", chk], capture_output=True, text=True).stdout
    for n in names:
        assert (" T " + n) in out, n
    assert lib.teuk_checked_build() == 0 and ctypes.CDLL(chk).teuk_checked_build() == 1


def test_struct_layout_matches_header(tmp_path):
    src = tmp_path / "layout.c"
    src.write_text('''
#include <stddef.h>
#include <stdio.h>
#include "teuk.h"
int main(void) {
  printf("%zu %zu %zu %zu %zu %zu\\n", sizeof(teuk_params), offsetof(teuk_params, n_rstar),
         offsetof(teuk_params, courant), offsetof(teuk_params, rstar_ext),
         offsetof(teuk_params, wave_capacity), sizeof(teuk_orbit));
  return 0;
}''')
    exe = tmp_path / "layout"
    subprocess.check_call(["gcc", "-I", os.path.join(_lib.ROOT, "include"), str(src), "-o", str(exe)])
    got = [int(v) for v in subprocess.check_output([str(exe)]).split()]
    tp = _lib.teuk_params
    want = [ctypes.sizeof(tp), tp.n_rstar.offset, tp.courant.offset, tp.rstar_ext.offset,
            tp.wave_capacity.offset, ctypes.sizeof(_lib.teuk_orbit)]
    assert got == want


@pytest.mark.parametrize("bad", [dict(a=1.0), dict(a=1.2), dict(M=0.0), dict(n_rstar=7),
                                 dict(n_theta=3), dict(n_theta=2048), dict(rstar_max=-60.0),
                                 dict(rstar_ext=151.0), dict(rstar_ext=-51.0), dict(prec=5),
                                 dict(dt_rule=7), dict(courant=0.0), dict(wave_capacity=-1)])
def test_invalid_parameters_rejected_before_any_device_work(lib, bad):
    p = P.make_params(**{k: v for k, v in bad.items() if k != "prec"})
    if "prec" in bad:
        p.prec = bad["prec"]
    h = ctypes.c_void_p()
    st = lib.teuk_create(ctypes.byref(p), 1, None, ctypes.byref(h))
    assert st == _lib.TEUK_EINVAL
    assert h.value is None
    assert lib.teuk_last_error(None)


def test_null_and_mixed_precision_rejected(lib):
    h = ctypes.c_void_p()
    assert lib.teuk_create(None, 1, None, ctypes.byref(h)) == _lib.TEUK_EINVAL
    arr = (_lib.teuk_params * 2)(P.make_params(prec="fp64"), P.make_params(prec="fp32"))
    assert lib.teuk_create(arr, 2, None, ctypes.byref(h)) == _lib.TEUK_EINVAL
    assert b"precision" in lib.teuk_last_error(None)
    # calls on a NULL context are rejected, not crashed
    assert lib.teuk_step_n(None, 1) == _lib.TEUK_EINVAL
    assert lib.teuk_sync(None) == _lib.TEUK_EINVAL
    lib.teuk_destroy(None)


def test_no_cpu_fallback_without_a_gpu(lib):
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    p = P.make_params()
    h = ctypes.c_void_p()
    st = lib.teuk_create(ctypes.byref(p), 1, None, ctypes.byref(h))
    assert st == _lib.TEUK_ECUDA
    assert h.value is None
