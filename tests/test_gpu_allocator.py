"""teuk_set_allocator: device memory through the caller's allocator.  With torch's caching
allocator the library's buffers show up in torch's accounting and the results are those
of the default allocator bit for bit; a capped allocator that refuses makes teuk_create
fail with TEUK_ENOMEM and give back everything it had taken."""
import numpy as np
import pytest

from paper_1001_3631_gb300 import TeukError, TeukSolver, inputs, set_allocator, use_torch_allocator

pytestmark = pytest.mark.gpu

PARAMS = dict(s=-2, m=2, a=0.9, rstar_min=-20.0, rstar_max=60.0, n_rstar=400, n_theta=48,
              rstar_ext=30.0, dt_rule=1, courant=0.5)


def run(prec):
    with TeukSolver(dict(PARAMS, prec=prec)) as s:
        s.set_source(8.0, inputs.amplitudes(50, seed=2))
        s.set_state(inputs.smooth_state(48, 400, seed=3), 0)
        s.step(40)
        u = s.get_state()
        w, _ = s.extract()
        s.adjoint(10, step0=40, grad_wave=np.ones((10, 48, 2)))   # adjoint buffers too
        s.sync()
    return u, w


@pytest.mark.parametrize("prec", ["fp64", "fp32_kahan"])
def test_torch_caching_allocator(prec):
    import torch
    ref = run(prec)
    torch.cuda.synchronize()
    base = torch.cuda.memory_allocated()
    use_torch_allocator()
    try:
        with TeukSolver(dict(PARAMS, prec=prec)) as s:
            torch.cuda.synchronize()
            assert torch.cuda.memory_allocated() > base + 400 * 64 * 16   # the state planes at least
        torch.cuda.synchronize()
        assert torch.cuda.memory_allocated() == base   # all of it given back on destroy
        got = run(prec)
    finally:
        set_allocator()
    assert np.array_equal(got[0], ref[0]) and np.array_equal(got[1], ref[1])


def test_capped_allocator_reports_enomem_and_releases_everything():
    import torch
    live, calls = {}, {"alloc": 0, "free": 0}
    cap = 8 << 20

    def alloc(n, stream):
        calls["alloc"] += 1
        if sum(live.values()) + n > cap:
            return 0
        p = torch.cuda.caching_allocator_alloc(n, stream=stream)
        live[p] = n
        return p

    def free(p, stream):
        calls["free"] += 1
        live.pop(p)
        torch.cuda.caching_allocator_delete(p)

    set_allocator(alloc, free)
    try:
        big = dict(PARAMS, n_rstar=8192, n_theta=128)   # 33 MB of FP64 state per buffer
        with pytest.raises(TeukError) as e:
            TeukSolver(dict(big, prec="fp64"))
        assert e.value.status == 2   # TEUK_ENOMEM
        assert not live and calls["free"] == calls["alloc"] - 1   # the refused call took nothing
        with TeukSolver(dict(PARAMS, prec="fp32_kahan")) as s:   # a grid under the cap works
            s.set_source(8.0)
            s.step(5)
            s.sync()
        assert not live
    finally:
        set_allocator()
