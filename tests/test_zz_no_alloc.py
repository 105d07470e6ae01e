"""teuk_waveform_sum_noalloc: the allocation-free reduction of waveform records.

It exists for callers that must not allocate device memory (an application whose
device memory all belongs to its own pool, or a latency-critical loop that cannot
afford a driver allocation).  Its result must equal what teuk_extract returns for
the same records; it is checked on two calls in a row because every call reuses
the same fixed device array.  This file is collected last on purpose."""
import ctypes

import numpy as np
import pytest

from paper_1001_3631_gb300 import TeukSolver, _lib

pytestmark = pytest.mark.gpu


def test_noalloc_sum_matches_extract_twice():
    import torch
    lib = _lib.load()
    # a call with no records places the fixed array on this device (the warm-up a caller
    # makes before a region that must not allocate)
    assert lib.teuk_waveform_sum_noalloc(None, 0, 48, None, None) == _lib.TEUK_OK
    params = dict(s=-2, m=3, a=0.7, rstar_min=-20.0, rstar_max=40.0, n_rstar=301, n_theta=48,
                  rstar_ext=11.0, dt_rule=1, courant=0.5, prec="fp64")
    with TeukSolver(params) as s:
        s.set_source(8.0)
        s.step(700)
        rec, first, sc_ref = s.extract(scalar=True)   # the existing entry point
    assert rec.shape == (701, 48, 2) and np.abs(sc_ref).max() > 0
    # the records in caller-owned device memory (allocated by the caller, not the library)
    wave_dev = torch.from_numpy(np.ascontiguousarray(rec)).cuda()
    stream = torch.cuda.current_stream()
    for _ in range(2):
        out = np.full((701, 2), np.nan)
        st = lib.teuk_waveform_sum_noalloc(ctypes.c_void_p(wave_dev.data_ptr()), 701, 48,
                                           _lib.ptr(out), ctypes.c_void_p(stream.cuda_stream))
        assert st == _lib.TEUK_OK, lib.teuk_last_error(None)
        assert np.allclose(out, sc_ref, rtol=1e-13, atol=0.0)
    # a smaller call after the larger one still returns only its own results
    out = np.full((5, 2), np.nan)
    assert lib.teuk_waveform_sum_noalloc(ctypes.c_void_p(wave_dev.data_ptr()), 5, 48,
                                         _lib.ptr(out), None) == _lib.TEUK_OK
    assert np.allclose(out, sc_ref[:5], rtol=1e-13, atol=0.0)
    # sizes beyond the fixed array are refused with a message
    big = _lib.TEUK_NOALLOC_MAX_RECORDS + 1
    st = lib.teuk_waveform_sum_noalloc(ctypes.c_void_p(wave_dev.data_ptr()), big, 48,
                                       _lib.ptr(out), None)
    assert st == _lib.TEUK_EINVAL
    assert b"outside" in lib.teuk_last_error(None)


def test_noalloc_calls_allocate_no_device_memory():
    """After the warm-up call, calls at the largest accepted size leave the device's free
    memory unchanged: nothing is allocated, not even temporarily held past the call."""
    import torch
    lib = _lib.load()
    n, nth = _lib.TEUK_NOALLOC_MAX_RECORDS, 4
    rec = np.random.default_rng(3).standard_normal((n, nth, 2))
    wave_dev = torch.from_numpy(rec).cuda()
    out = np.empty((n, 2))
    stream = torch.cuda.current_stream()
    assert lib.teuk_waveform_sum_noalloc(None, 0, nth, None, None) == _lib.TEUK_OK
    assert lib.teuk_waveform_sum_noalloc(ctypes.c_void_p(wave_dev.data_ptr()), n, nth, _lib.ptr(out),
                                         ctypes.c_void_p(stream.cuda_stream)) == _lib.TEUK_OK
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    for _ in range(4):
        assert lib.teuk_waveform_sum_noalloc(ctypes.c_void_p(wave_dev.data_ptr()), n, nth,
                                             _lib.ptr(out), ctypes.c_void_p(stream.cuda_stream)) == _lib.TEUK_OK
        assert torch.cuda.mem_get_info()[0] == free0
    th = (np.arange(nth) + 0.5) * np.pi / nth
    ref = (rec * (np.sin(th) * np.pi / nth)[None, :, None]).sum(axis=1)
    assert np.allclose(out, ref, rtol=1e-12, atol=1e-14)
