"""Pins of the oracle's moving-particle source (a sampled eccentric or inclined orbit:
the circular-orbit source of the synthetic problem with the Gaussian centred on the
particle and the phase of its azimuth, Sec. 2 and Eq. 1's source term).

Independent of the oracle's code: a 40-digit brute-force stepper fed with a source
evaluated from its definition in mpmath; the reduction to the circular-orbit source;
the exact phase rotation e^{-i m alpha} of a turned azimuth; no source once the samples
end; and the theta-mirror symmetry of the s = 0 equation."""
import mpmath as mp
import numpy as np
import pytest

import derive
from paper_1001_3631_gb300 import inputs
from test_oracle_scheme import _brute_force


def rel(a, b):
    return np.linalg.norm(a - b) / np.linalg.norm(b)


def cplx(u):
    return u[0] + 1j * u[1], u[2] + 1j * u[3]


GRID = dict(n_rstar=120, n_theta=16, rstar_min=-20.0, rstar_max=40.0, rstar_ext=30.0,
            dt_rule=1, courant=0.5)


def test_circular_trajectory_is_the_orbit_source(orc):
    p = orc.params(s=-2, m=3, a=0.7, r0=7.0, **GRID)
    g, ob = orc.grid(p), orc.orbit(p)
    n = 40
    amps = inputs.amplitudes(n, seed=3)
    t = 0.5 * g["dt"] * np.arange(2 * n)
    traj = np.stack([np.full(2 * n, 7.0), np.full(2 * n, 0.5 * np.pi), ob["Omega"] * t + ob["phi0"],
                     np.repeat(amps, 2)], axis=1)
    u0 = inputs.smooth_state(16, 120, seed=4)
    u_ref, w_ref = orc.run(p, u0, n, orc.orbit_source(p), amps=amps)
    u, w = orc.run_trajectory(p, traj, u0, n)
    assert rel(u, u_ref) <= 1e-13 and rel(w, w_ref) <= 1e-13


@pytest.mark.parametrize("m", [2, 3])
def test_bruteforce_moving_source_tiny_grid(orc, m):
    M, a, s = 1.0, 0.6, -2
    nr, nth, dt, nsteps = 7, 4, 0.01, 3
    rs_min, rs_max = -4.0, 8.0
    sig_r, sig_t = 0.3, 0.12       # the 8 sigma cut keeps 2 columns and 1-2 rows
    rng = np.random.default_rng(31 + m)
    u0 = rng.standard_normal((4, nth, nr))
    # the particle crosses columns and rows during the three steps
    traj = np.array([[4.2 + 0.35 * k, 1.3 + 0.11 * k, 0.4 + 0.9 * k, 1.0 + 0.05 * (-1) ** k]
                     for k in range(2 * nsteps)])
    p = orc.params(M=M, a=a, s=s, m=m, rstar_min=rs_min, rstar_max=rs_max, n_rstar=nr,
                   n_theta=nth, dt=dt, rstar_ext=0.0, sigma_r_abs=sig_r, sigma_th_abs=sig_t)
    u, _ = orc.run_trajectory(p, traj, u0, nsteps)
    with mp.workdps(40):
        drs = (mp.mpf(rs_max) - rs_min) / (nr - 1)
        dth = mp.pi / nth
        rplus = M + mp.sqrt(M * M - a * a)

        def r_of(rs):
            y = mp.findroot(lambda yy: derive.tortoise_of_x(M, a, mp.e ** yy) - rs, mp.mpf(0))
            return rplus + mp.e ** y

        cut = []

        def tau(n, half, j, i):
            r_p, th_p, phi_p, A = [mp.mpf(v) for v in traj[2 * n + (0 if half else 1)]]
            rs_p = derive.tortoise_of_x(M, a, r_p - rplus)
            rs = rs_min + (i + (mp.mpf(1) / 2 if half else 0)) * drs
            th = (j + mp.mpf(1) / 2) * dth
            dr, dt_ = rs - rs_p, th - th_p
            cut.append(min(abs(abs(dr) / (8 * sig_r) - 1), abs(abs(dt_) / (8 * sig_t) - 1)))
            if abs(dr) > 8 * sig_r or abs(dt_) > 8 * sig_t:
                return mp.mpc(0)
            G = mp.e ** (-(dr ** 2 / sig_r ** 2 + dt_ ** 2 / sig_t ** 2) / 2) / (2 * mp.pi * sig_r * sig_t)
            r = r_of(rs)
            D = r * r - 2 * M * r + a * a
            Sig2 = (r * r + a * a) ** 2 - a * a * D * mp.sin(th) ** 2
            pref = 4 * mp.pi * D * (r * r + a * a * mp.cos(th) ** 2) / (Sig2 * r ** 3)
            return A * mp.expj(-m * phi_p) * pref * G

        ref = _brute_force(M, a, s, m, rs_min, rs_max, nr, nth, dt, u0, 0, 0, None, None, None,
                           nsteps, taus=tau)
    assert min(cut) > 1e-6          # no node on the cut, where rounding could decide
    assert np.abs(u - ref).max() <= 1e-13 * np.abs(ref).max()
    # the source did enter: without it the result differs
    u_free, _ = orc.run(p, u0, nsteps)
    assert np.abs(u_free - ref).max() > 1e-6 * np.abs(ref).max()


def test_turned_azimuth_rotates_the_solution(orc):
    p = orc.params(s=-2, m=2, a=0.9, **GRID)
    g = orc.grid(p)
    n = 30
    traj = inputs.eccentric_trajectory(2 * n, g["dt"], semi_latus=9.0, ecc=0.3, incl=0.4)
    alpha = 0.77
    turned = traj.copy()
    turned[:, 2] += alpha
    u1, w1 = orc.run_trajectory(p, traj, None, n)
    u2, w2 = orc.run_trajectory(p, turned, None, n)
    F1, P1 = cplx(u1)
    F2, P2 = cplx(u2)
    rot = np.exp(-1j * 2 * alpha)
    assert rel(F2, rot * F1) <= 1e-13 and rel(P2, rot * P1) <= 1e-13
    assert np.abs(F1).max() > 0


@pytest.mark.parametrize("n_samples", [20, 21])
def test_no_source_after_the_last_sample(orc, n_samples):
    p = orc.params(s=-2, m=2, a=0.9, **GRID)
    g = orc.grid(p)
    traj = inputs.eccentric_trajectory(n_samples, g["dt"], semi_latus=9.0, ecc=0.3, incl=0.4)
    u, _ = orc.run_trajectory(p, traj, None, 20)
    # sample 2n feeds Eq. (13) of step n and sample 2n + 1 Eq. (14): 20 samples cover
    # 10 steps; 21 samples add the predictor source of step 10
    half = orc.run_trajectory(p, traj[:20], None, 10)[0]
    if n_samples == 20:
        ref, _ = orc.run(p, half, 10, step0=10)
    else:
        one = np.concatenate([traj, np.zeros((1, 4))])
        one[21] = traj[20]
        one[21, 3] = 0.0           # a corrector sample of amplitude 0 is no source
        ref = orc.run_trajectory(p, one, half, 1, step0=10)[0]
        ref, _ = orc.run(p, ref, 9, step0=11)
    assert np.array_equal(u, ref)


def test_theta_mirror_symmetry_at_zero_spin(orc):
    # s = 0: every coefficient is even under theta -> pi - theta, cot odd, so a particle
    # at pi - theta_p gives the mirrored field
    p = orc.params(s=0, m=2, a=0.8, **GRID)
    g = orc.grid(p)
    n = 30
    traj = inputs.eccentric_trajectory(2 * n, g["dt"], semi_latus=9.0, ecc=0.3, incl=0.5)
    mirrored = traj.copy()
    mirrored[:, 1] = np.pi - traj[:, 1]
    u1, _ = orc.run_trajectory(p, traj, None, n)
    u2, _ = orc.run_trajectory(p, mirrored, None, n)
    assert rel(u2, u1[:, ::-1, :]) <= 1e-12
    assert rel(u1, u1[:, ::-1, :]) > 1e-3      # the inclined orbit is not symmetric itself
