"""Moving particle (sampled eccentric / inclined path) through the C ABI against the
oracle's moving-source run, element by element, in every precision and launch form;
a circular path against the circular-orbit source; argument errors."""
import numpy as np
import pytest

from paper_1001_3631_gb300 import TeukError, TeukSolver, inputs

pytestmark = pytest.mark.gpu

TOL = {"fp64": 1e-12, "fp64_df": 1e-12, "fp32_kahan": 1e-6, "fp32": 1e-5}

# (params, path) -- ragged grids; both pole parities; a Keplerian inclined path and a
# fast synthetic one that sweeps across many blocks within the run.  The extraction
# radius lies in the region the particle sweeps, so that the waveform of these short
# runs carries the source's signal (further out it is still the pre-arrival precursor,
# ~1e-60, below the FP32 range of the double-float path).
CASES = [
    (dict(s=-2, m=3, a=0.7, rstar_min=-20.0, rstar_max=40.0, n_rstar=151, n_theta=33,
          rstar_ext=12.0, dt_rule=1, courant=0.5), "kepler"),
    (dict(s=-2, m=2, a=0.9, rstar_min=-10.0, rstar_max=30.0, n_rstar=197, n_theta=12,
          rstar_ext=10.3, dt_rule=1, courant=0.5), "fast"),
    (dict(s=1, m=1, a=0.5, rstar_min=-10.0, rstar_max=30.0, n_rstar=97, n_theta=300,
          rstar_ext=11.0, dt_rule=1, courant=0.5), "kepler"),
]


def rel(a, b):
    nb = np.linalg.norm(b)
    return np.linalg.norm(a - b) / (nb if nb > 0 else 1.0)


def path(kind, n_samples, dt):
    if kind == "kepler":
        return inputs.eccentric_trajectory(n_samples, dt, semi_latus=8.0, ecc=0.5, incl=0.6,
                                           chi0=1.5, amp_sigma=0.1)
    t = 0.5 * dt * np.arange(n_samples)
    return np.stack([9.0 + 4.0 * np.sin(9.0 * t), 1.5 + 0.6 * np.sin(7.0 * t), 0.3 * t,
                     1.0 + 0.2 * np.cos(5.0 * t)], axis=1)


def oracle(orc, params, traj, nsteps, u0=None, step0=0):
    kw = {k: v for k, v in params.items() if k not in ("prec", "wave_capacity")}
    return orc.run_trajectory(orc.params(**kw), traj, u0, nsteps, step0=step0)


def gpu(params, prec, traj, steps, u0=None, strip=0, persistent=False, step0=0):
    with TeukSolver(dict(params, prec=prec)) as s:
        s.set_tiling(strip, 0 if persistent else 1)
        s.set_trajectory(traj)
        if u0 is not None or step0:
            s.set_state(np.zeros(s.shape()) if u0 is None else u0, step0)
        for n in steps:
            s.step(n)
        u = s.get_state()
        w, first = s.extract()
        s.sync()
    return u, w, first


@pytest.mark.parametrize("prec", ["fp64", "fp64_df", "fp32_kahan", "fp32"])
@pytest.mark.parametrize("case", range(len(CASES)))
def test_moving_source_against_oracle(orc, case, prec):
    params, kind = CASES[case]
    with TeukSolver(dict(params, prec="fp64")) as s:
        dt = s.geometry()["dt"]
    nsteps = 120
    # samples end in the middle of step 100 (no corrector source there), so the last
    # steps run without a source
    traj = path(kind, 201, dt)
    uo, wo = oracle(orc, params, traj, nsteps)
    assert np.abs(wo[-1]).max() > 1e-6 * np.abs(uo).max()
    for strip in (0, 5):
        u, w, first = gpu(params, prec, traj, [nsteps], strip=strip)
        assert first == 0
        assert rel(u, uo) <= TOL[prec], (strip, rel(u, uo))
        assert rel(w, wo) <= TOL[prec], (strip, rel(w, wo))


@pytest.mark.parametrize("prec", ["fp64", "fp32_kahan"])
def test_moving_source_launch_forms_agree_bitwise(orc, prec):
    params, kind = CASES[0]
    with TeukSolver(dict(params, prec="fp64")) as s:
        dt = s.geometry()["dt"]
    traj = path(kind, 160, dt)
    u0 = inputs.random_state(params["n_theta"], params["n_rstar"], seed=5)
    ref = gpu(params, prec, traj, [37, 23], u0=u0, step0=3, strip=7)
    for strip, persistent in ((0, False), (16, True), (0, True)):
        got = gpu(params, prec, traj, [37, 23], u0=u0, step0=3, strip=strip, persistent=persistent)
        assert np.array_equal(got[0], ref[0]) and np.array_equal(got[1], ref[1])
    # and the oracle from the same start (step 3: samples 6 and 7 first)
    uo, _ = oracle(orc, params, traj, 60, u0=u0, step0=3)
    assert rel(ref[0], uo) <= TOL[prec]


def test_batched_mix_of_moving_and_circular_sources(orc):
    insts = [CASES[0][0], CASES[1][0], dict(CASES[0][0], m=2, n_rstar=130)]
    dts = []
    for p in insts:
        with TeukSolver(dict(p, prec="fp64")) as s:
            dts.append(s.geometry()["dt"])
    trajs = [path("kepler", 120, dts[0]), path("fast", 120, dts[1]), None]
    n = 50
    with TeukSolver([dict(p, prec="fp64") for p in insts]) as s:
        s.set_tiling(0, 1)
        for k, tr in enumerate(trajs):
            if tr is None:
                s.set_source(8.0, instance=k)
            else:
                s.set_trajectory(tr, instance=k)
        s.step(n)
        got = [s.get_state(k) for k in range(3)]
        s.sync()
    for k, tr in enumerate(trajs):
        p = insts[k]
        if tr is None:
            kw = {q: v for q, v in p.items()}
            op = orc.params(**kw, r0=8.0)
            uo, _ = orc.run(op, None, n, orc.orbit_source(op))
        else:
            uo, _ = oracle(orc, p, tr, n)
        assert rel(got[k], uo) <= 1e-12, k


@pytest.mark.parametrize("prec,tol", [("fp64", 1e-13), ("fp32_kahan", 1e-6)])
def test_circular_path_equals_circular_orbit_source(orc, prec, tol):
    params = CASES[0][0]
    r0 = 7.5
    kw = dict(params)
    ob = orc.orbit(orc.params(**kw, r0=r0))
    n = 80
    amps = inputs.amplitudes(n, seed=9)
    with TeukSolver(dict(params, prec=prec)) as s:
        dt = s.geometry()["dt"]
        s.set_source(r0, amps)
        s.step(n)
        u_ref = s.get_state()
        t = 0.5 * dt * np.arange(2 * n)
        traj = np.stack([np.full(2 * n, r0), np.full(2 * n, 0.5 * np.pi),
                         ob["Omega"] * t + ob["phi0"], np.repeat(amps, 2)], axis=1)
        s.set_trajectory(traj)
        s.set_state(np.zeros(s.shape()), 0)
        s.step(n)
        u = s.get_state()
        s.sync()
    assert rel(u, u_ref) <= tol


def test_paper_scale_grid_eccentric_orbit(orc):
    ps = inputs.PAPER_SCALE_16384x256["params"]
    with TeukSolver(dict(ps, prec="fp64")) as s:
        dt = s.geometry()["dt"]
    traj = inputs.eccentric_trajectory(9, dt, semi_latus=10.0, ecc=0.4, incl=0.3, chi0=1.0)
    u0 = inputs.smooth_state(ps["n_theta"], ps["n_rstar"], seed=12)
    uo, wo = oracle(orc, ps, traj, 4, u0=u0)
    for prec in ("fp64", "fp32_kahan"):
        u, w, _ = gpu(ps, prec, traj, [4], u0=u0)
        # the source window only: the field there is dominated by the deposited source
        d = u - uo
        assert rel(u, uo) <= TOL[prec] and rel(w, wo) <= TOL[prec], prec
        assert np.abs(d).max() <= 1e3 * TOL[prec] * np.abs(uo).max()


def test_trajectory_argument_errors():
    params = CASES[0][0]
    with TeukSolver(dict(params, prec="fp64")) as s:
        dt = s.geometry()["dt"]
        good = path("kepler", 10, dt)
        bad = []
        b = good.copy(); b[3, 0] = 1.0; bad.append(b)            # inside the horizon
        b = good.copy(); b[2, 1] = 0.0; bad.append(b)            # on the pole
        b = good.copy(); b[4, 0] = 1e4; bad.append(b)            # off the radial grid
        b = good.copy(); b[1, 3] = np.nan; bad.append(b)         # not finite
        for b in bad:
            with pytest.raises(TeukError) as e:
                s.set_trajectory(b)
            assert e.value.status == 1
        with pytest.raises(TeukError):
            s.set_trajectory(np.zeros((0, 4)))
        s.set_trajectory(good)
        s.step(3)
        with pytest.raises(TeukError) as e:
            s.adjoint(3)
        assert e.value.status == 1
        s.set_source(8.0)        # the circular orbit replaces the path
        s.step(2)
        s.sync()
