"""GPU adjoint (teuk_adjoint_n, TeukWaveformFn) against the oracle's FP64 adjoint and
against central finite differences of the GPU forward sweep."""
import numpy as np
import pytest

from paper_1001_3631_gb300 import TeukSolver, inputs

pytestmark = pytest.mark.gpu


def rel(a, b):
    nb = np.linalg.norm(b)
    return np.linalg.norm(np.asarray(a) - np.asarray(b)) / (nb if nb > 0 else 1.0)


SMALL = dict(s=-2, a=0.7, rstar_min=-10.0, rstar_max=30.0, n_rstar=61, n_theta=8,
             rstar_ext=14.0, dt_rule=1, courant=0.5)


def oracle_params(orc, params, r0):
    kw = {k: v for k, v in params.items() if k not in ("prec", "wave_capacity")}
    return orc.params(**kw, r0=r0)


@pytest.mark.parametrize("m", [2, 1])
def test_cotangent_mode_matches_oracle_adjoint(orc, m):
    params = dict(SMALL, m=m)
    n, r0 = 30, 8.0
    amps = inputs.amplitudes(n, seed=5005)
    gw = np.random.default_rng(12).standard_normal((n, 8, 2))
    p = oracle_params(orc, params, r0)
    ga_o, gr_o, _ = orc.adjoint(p, orc.orbit_source(p), gw, amps=amps)
    with TeukSolver(dict(params, prec="fp64", wave_capacity=n + 1)) as s:
        s.set_source(r0, amps)
        ga, gr, _ = s.adjoint(n, step0=0, grad_wave=gw)
        assert s.time()[0] == 0  # cotangent mode does not touch the state
    assert rel(ga, ga_o) <= 1e-11
    assert gr == pytest.approx(gr_o, rel=1e-11)


def test_fp64_df_instance_adjoint_matches_oracle(orc):
    # double-float instances: FP64 co-state on the double-float coefficient tables
    params = dict(SMALL, m=2)
    n, r0 = 30, 8.0
    amps = inputs.amplitudes(n, seed=5005)
    gw = np.random.default_rng(12).standard_normal((n, 8, 2))
    p = oracle_params(orc, params, r0)
    ga_o, gr_o, _ = orc.adjoint(p, orc.orbit_source(p), gw, amps=amps)
    with TeukSolver(dict(params, prec="fp64_df", wave_capacity=n + 1)) as s:
        s.set_source(r0, amps)
        ga, gr, _ = s.adjoint(n, step0=0, grad_wave=gw)
    assert rel(ga, ga_o) <= 1e-11
    assert gr == pytest.approx(gr_o, rel=1e-11)


# FP32 instances run the co-state in compensated FP32.  Against the oracle's FP64
# adjoint (cotangent mode: no forward run, so only the FP32 rounding of the coefficient
# tables and of the co-state arithmetic separate them) the gradients agree to ~1e-6
# relative (measured up to 9.4e-7 for dL/dA and 3.1e-6 for dL/dr0 on these grids); the
# bounds leave a factor of ~10.
@pytest.mark.parametrize("prec", ["fp32_kahan", "fp32"])
@pytest.mark.parametrize("m", [2, 1])
def test_fp32_costate_matches_oracle_adjoint(orc, prec, m):
    params = dict(SMALL, m=m, n_rstar=201, n_theta=16, rstar_min=-20.0, rstar_max=40.0,
                  rstar_ext=11.0)
    n, r0 = 200, 8.0
    amps = inputs.amplitudes(n, seed=5005)
    gw = np.random.default_rng(12).standard_normal((n, 16, 2))
    p = oracle_params(orc, params, r0)
    ga_o, gr_o, _ = orc.adjoint(p, orc.orbit_source(p), gw, amps=amps)
    with TeukSolver(dict(params, prec=prec, wave_capacity=n + 1)) as s:
        s.set_source(r0, amps)
        ga, gr, _ = s.adjoint(n, step0=0, grad_wave=gw)
    assert rel(ga, ga_o) <= 1e-5
    assert gr == pytest.approx(gr_o, rel=3e-5)


def _host_loss(s, n):
    w, first = s.extract(cap=n + 1)
    assert first == 0
    return s.geometry()["r_ext"] ** 6 * np.sum(w[1:] ** 2), w


@pytest.mark.parametrize("prec", ["fp64", "fp32_kahan"])
def test_builtin_loss_checkpointing_is_exact(orc, prec):
    params = dict(SMALL, m=2, n_rstar=301, n_theta=32, rstar_min=-20.0, rstar_max=60.0,
                  rstar_ext=12.0)
    n, r0 = 300, 8.0
    amps = inputs.amplitudes(n, seed=5005)
    res = {}
    for ck in (0, 100, 64, 1):
        with TeukSolver(dict(params, prec=prec)) as s:
            s.set_source(r0, amps)
            res[ck] = s.adjoint(n, step0=0, ckpt_every=ck)
            assert s.time()[0] == n
    for ck in (100, 64, 1):  # recomputing from checkpoints reproduces the stored sweep bit for bit
        assert np.array_equal(res[ck][0], res[0][0])
        assert res[ck][1] == res[0][1] and res[ck][2] == res[0][2]
    if prec == "fp64":
        # and the result is the oracle's adjoint of the oracle's loss
        p = oracle_params(orc, params, r0)
        src = orc.orbit_source(p)
        _, wo = orc.run(p, None, n, src, amps=amps)
        rext = orc.r_ext(p)
        ga_o, gr_o, _ = orc.adjoint(p, src, 2 * rext ** 6 * wo[1:], amps=amps)
        assert rel(res[0][0], ga_o) <= 1e-10
        assert res[0][1] == pytest.approx(gr_o, rel=1e-10)
        assert res[0][2] == pytest.approx(rext ** 6 * np.sum(wo[1:] ** 2), rel=1e-12)


def _fd_loss(params, r0, amps, n):
    with TeukSolver(dict(params, prec="fp64", wave_capacity=n + 1)) as s:
        s.set_source(r0, amps)
        s.step(n)
        return _host_loss(s, n)[0]


def test_gradients_vs_central_differences_small():
    params = dict(SMALL, m=2, n_rstar=201, n_theta=16, rstar_min=-20.0, rstar_max=40.0,
                  rstar_ext=11.0)
    n, r0, h = 200, 8.0, 1e-6
    amps = inputs.amplitudes(n, seed=7)
    with TeukSolver(dict(params, prec="fp64")) as s:
        s.set_source(r0, amps)
        ga, gr, L = s.adjoint(n, step0=0, ckpt_every=50)
    assert L == pytest.approx(_fd_loss(params, r0, amps, n), rel=1e-13)
    for k in (0, 57, 120, 199):
        ap, am = amps.copy(), amps.copy()
        ap[k] += h
        am[k] -= h
        fd = (_fd_loss(params, r0, ap, n) - _fd_loss(params, r0, am, n)) / (2 * h)
        assert ga[k] == pytest.approx(fd, rel=1e-6, abs=1e-9 * abs(L))
    fdr = (_fd_loss(params, r0 + h, amps, n) - _fd_loss(params, r0 - h, amps, n)) / (2 * h)
    assert gr == pytest.approx(fdr, rel=1e-5)


def test_adjoint_workload_4096x128_full_size():
    # the full adjoint workload (4096 x 128 grid, 10000 steps, checkpoint every 100) in
    # FP64; gradients checked by central differences (h = 1e-6) at sampled steps and for
    # r0.  In 10000 steps of dt = 2e-3 the signal travels ~20 M, so the loss is taken at a
    # near-zone probe r* = 12.5 (the particle sits at r* = 11.5); at r* = 300 it is 0.
    cfg = inputs.ADJOINT_4096x128
    params, n, r0 = dict(cfg["params"], rstar_ext=12.5), cfg["steps"], cfg["r0"]
    amps = inputs.amplitudes(n, seed=cfg["amp_seed"])
    with TeukSolver(dict(params, prec="fp64")) as s:
        s.set_source(r0, amps)
        ga, gr, L = s.adjoint(n, step0=0, ckpt_every=cfg["ckpt_every"])
    assert L > 0 and np.all(np.isfinite(ga))
    h = 1e-6
    for k in (0, 4999, 9876):
        ap, am = amps.copy(), amps.copy()
        ap[k] += h
        am[k] -= h
        fd = (_fd_loss(params, r0, ap, n) - _fd_loss(params, r0, am, n)) / (2 * h)
        assert ga[k] == pytest.approx(fd, rel=1e-5, abs=1e-8 * abs(L))
    fdr = (_fd_loss(params, r0 + h, amps, n) - _fd_loss(params, r0 - h, amps, n)) / (2 * h)
    assert gr == pytest.approx(fdr, rel=1e-5)


def test_fp32_kahan_gradient_full_size_close_to_fp64():
    # the full adjoint workload on an FP32-Kahan instance (compensated FP32 co-state)
    # against the FP64 instance: measured 2.8e-7 (dL/dA), 1.5e-6 (dL/dr0), 3.2e-7 (loss)
    cfg = inputs.ADJOINT_4096x128
    params, n, r0 = dict(cfg["params"], rstar_ext=12.5), cfg["steps"], cfg["r0"]
    amps = inputs.amplitudes(n, seed=cfg["amp_seed"])
    res = {}
    for prec in ("fp64", "fp32_kahan"):
        with TeukSolver(dict(params, prec=prec)) as s:
            s.set_source(r0, amps)
            res[prec] = s.adjoint(n, step0=0, ckpt_every=cfg["ckpt_every"])
    assert rel(res["fp32_kahan"][0], res["fp64"][0]) <= 3e-6
    assert res["fp32_kahan"][1] == pytest.approx(res["fp64"][1], rel=2e-5)
    assert res["fp32_kahan"][2] == pytest.approx(res["fp64"][2], rel=3e-6)


def test_autograd_function_matches_builtin_adjoint():
    import torch

    from paper_1001_3631_gb300.autograd import TeukWaveformFn, psi_loss
    params = dict(SMALL, m=2, n_rstar=201, n_theta=16, rstar_min=-20.0, rstar_max=40.0,
                  rstar_ext=11.0)
    n, r0 = 150, 8.0
    amps0 = inputs.amplitudes(n, seed=3)
    with TeukSolver(dict(params, prec="fp64", wave_capacity=n + 1)) as s:
        amps = torch.tensor(amps0, dtype=torch.float64, requires_grad=True)
        r0t = torch.tensor(r0, dtype=torch.float64, requires_grad=True)
        w = TeukWaveformFn.apply(amps, r0t, s, n)
        L = psi_loss(s, w)
        L.backward()
        s.set_source(r0, amps0)
        s.set_state(np.zeros(s.shape()), 0)
        ga, gr, Lb = s.adjoint(n, step0=0, ckpt_every=0)
    assert float(L.detach()) == pytest.approx(Lb, rel=1e-13)
    assert rel(amps.grad.numpy(), ga) <= 1e-12
    assert float(r0t.grad) == pytest.approx(gr, rel=1e-12)


def test_autograd_two_applies_on_one_solver_then_one_backward():
    """Each apply's backward differentiates its own problem even when a later apply on
    the same solver has replaced the source: L = f(A1, r1) + f(A2, r2)."""
    import torch

    from paper_1001_3631_gb300.autograd import TeukWaveformFn, psi_loss
    params = dict(SMALL, m=2, n_rstar=121, n_theta=8, rstar_min=-20.0, rstar_max=40.0,
                  rstar_ext=11.0)
    n = 60
    a1, a2 = inputs.amplitudes(n, seed=31), inputs.amplitudes(n, seed=32)
    with TeukSolver(dict(params, prec="fp64", wave_capacity=n + 1)) as s:
        A1 = torch.tensor(a1, dtype=torch.float64, requires_grad=True)
        A2 = torch.tensor(a2, dtype=torch.float64, requires_grad=True)
        r1 = torch.tensor(8.0, dtype=torch.float64, requires_grad=True)
        r2 = torch.tensor(9.5, dtype=torch.float64, requires_grad=True)
        L = psi_loss(s, TeukWaveformFn.apply(A1, r1, s, n)) + psi_loss(s, TeukWaveformFn.apply(A2, r2, s, n))
        L.backward()
        ref = []
        for a, r in ((a1, 8.0), (a2, 9.5)):
            s.set_source(r, a)
            s.set_state(np.zeros(s.shape()), 0)
            ref.append(s.adjoint(n, step0=0, ckpt_every=0))
    assert rel(A1.grad.numpy(), ref[0][0]) <= 1e-12
    assert rel(A2.grad.numpy(), ref[1][0]) <= 1e-12
    assert float(r1.grad) == pytest.approx(ref[0][1], rel=1e-12)
    assert float(r2.grad) == pytest.approx(ref[1][1], rel=1e-12)


@pytest.mark.parametrize("prec", ["fp64", "fp32_kahan"])
def test_checkpointed_loss_function_matches_waveform_function(prec):
    """TeukPsiLossFn (checkpointed forward, segment recomputation in the reverse sweep)
    gives the loss and gradients of TeukWaveformFn followed by psi_loss, scaled by the
    incoming gradient."""
    import torch

    from paper_1001_3631_gb300.autograd import TeukPsiLossFn, TeukWaveformFn, psi_loss
    params = dict(SMALL, m=2, n_rstar=201, n_theta=16, rstar_min=-20.0, rstar_max=40.0,
                  rstar_ext=11.0)
    n, r0 = 230, 8.0
    amps0 = inputs.amplitudes(n, seed=4)
    with TeukSolver(dict(params, prec=prec, wave_capacity=n + 1)) as s:
        A = torch.tensor(amps0, dtype=torch.float64, requires_grad=True)
        R = torch.tensor(r0, dtype=torch.float64, requires_grad=True)
        L = TeukPsiLossFn.apply(A, R, s, n, 50)
        (3.0 * L).backward()
        A2 = torch.tensor(amps0, dtype=torch.float64, requires_grad=True)
        R2 = torch.tensor(r0, dtype=torch.float64, requires_grad=True)
        L2 = psi_loss(s, TeukWaveformFn.apply(A2, R2, s, n))
        (3.0 * L2).backward()
    tol = 1e-12 if prec == "fp64" else 1e-6
    assert float(L.detach()) == pytest.approx(float(L2.detach()), rel=tol)
    assert rel(A.grad.numpy(), A2.grad.numpy()) <= tol
    assert float(R.grad) == pytest.approx(float(R2.grad), rel=max(tol, 1e-12))


@pytest.mark.parametrize("nth", [400, 600])
@pytest.mark.parametrize("prec,tol", [("fp64", 1e-11), ("fp32_kahan", 1e-5)])
def test_tall_columns_use_the_large_block_kernels(orc, prec, tol, nth):
    # n_theta = 400 / 600: blocks of 416 / 608 threads, the reverse-step kernels built for
    # columns of up to 512 / 1024 rows (their shared memory exceeds the default 48 KB)
    params = dict(SMALL, m=2, n_rstar=24, n_theta=nth, rstar_min=-10.0, rstar_max=20.0,
                  rstar_ext=12.0)
    n, r0 = 6, 6.0
    amps = inputs.amplitudes(n, seed=5)
    gw = np.random.default_rng(3).standard_normal((n, nth, 2))
    p = oracle_params(orc, params, r0)
    ga_o, gr_o, _ = orc.adjoint(p, orc.orbit_source(p), gw, amps=amps)
    with TeukSolver(dict(params, prec=prec, wave_capacity=n + 1)) as s:
        s.set_source(r0, amps)
        ga, gr, _ = s.adjoint(n, step0=0, grad_wave=gw)
        s.sync()
    assert rel(ga, ga_o) <= tol
    assert gr == pytest.approx(gr_o, rel=10 * tol)
