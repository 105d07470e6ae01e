"""Pins of the oracle's geometry and source: Eq. (2) tortoise coordinate, its
inversion, the grid, the synthetic source and the extraction interpolation.

Each check compares the oracle with something it does not contain: a numeric
derivative of its r*(r) against Eq. (2), the Schwarzschild textbook limit,
Kepler's law, Eq. (3), the Gaussian's normalisation, finite differences."""
import math

import mpmath as mp
import numpy as np
import pytest

import derive


@pytest.mark.parametrize("a", [0.0, 0.3, 0.7, 0.9, 0.99])
def test_tortoise_derivative_is_eq2(orc, a):
    # Eq. (2): dr*/dr = (r^2 + a^2)/Delta, checked by a numeric derivative of the oracle's r*(r).
    M = 1.0
    rp = M + math.sqrt(M * M - a * a)
    for r in [rp + 1e-3, rp + 0.5, 3.0, 10.0, 123.0]:
        h = 1e-6 * max(1.0, r - rp) if r - rp > 1e-2 else 1e-7
        d = (orc.rstar_of_r(M, a, r + h) - orc.rstar_of_r(M, a, r - h)) / (2 * h)
        Delta = r * r - 2 * M * r + a * a
        assert d == pytest.approx((r * r + a * a) / Delta, rel=1e-6)
        # and the test's own closed form (mpmath) agrees with the oracle's value
        assert orc.rstar_of_r(M, a, r) == pytest.approx(float(derive.tortoise_closed_form(M, a, r)),
                                                        rel=1e-13, abs=1e-12)


def test_tortoise_schwarzschild_limit(orc):
    # a = 0: the textbook r* = r + 2M ln(r/2M - 1)
    for M in [1.0, 2.5]:
        for r in [2.0 * M + 1e-4, 3.0 * M, 10.0 * M, 500.0 * M]:
            with mp.workdps(40):
                exact = float(mp.mpf(r) + 2 * M * mp.log(mp.mpf(r) / (2 * M) - 1))
            assert orc.rstar_of_r(M, 0.0, r) == pytest.approx(exact, rel=1e-13, abs=1e-12)


@pytest.mark.parametrize("a", [0.0, 0.5, 0.9, 0.99])
def test_tortoise_inversion_roundtrip(orc, a):
    M = 1.0
    rp = M + math.sqrt(M * M - a * a)
    rm = M - math.sqrt(M * M - a * a)
    for rs in [-200.0, -50.0, -3.0, 0.0, 12.783, 140.0, 800.0]:
        x = orc.x_of_rstar(M, a, rs)
        assert x > 0
        assert x * (x + rp - rm) > 0.0          # Delta > 0, even at r* = -200
        back = orc.lib().orc_rstar_of_x(M, a, x)
        assert abs(back - rs) <= 4e-14 * max(1.0, abs(rs))
        # independent inversion with mpmath at 40 digits
        with mp.workdps(40):
            y = mp.findroot(lambda yy: derive.tortoise_of_x(M, a, mp.e**yy) - rs, mp.log(x))
            assert x == pytest.approx(float(mp.e**y), rel=1e-12)


def test_grid_and_time_step_rules(orc):
    p = orc.params(n_rstar=800, n_theta=64, rstar_min=-50.0, rstar_max=150.0, courant=0.5,
                   dt_rule=0)
    g = orc.grid(p)
    assert g["drs"] == pytest.approx(200.0 / 799.0, rel=1e-15)
    assert g["dth"] == pytest.approx(math.pi / 64, rel=1e-15)
    assert g["dt"] == pytest.approx(0.5 * 200.0 / 799.0, rel=1e-15)
    p.dt_rule = 1
    assert orc.grid(p)["dt"] == pytest.approx(0.5 * (math.pi / 64) / (2 + 2 + 2), rel=1e-15)
    p.dt = 0.01
    assert orc.grid(p)["dt"] == 0.01
    # extraction bracket: r*_ext = 140 -> (140 + 50)/dr* = 759.05
    g = orc.grid(p)
    assert g["i_e"] == 759 and g["f_e"] == pytest.approx(0.05, abs=1e-12)


def test_extraction_is_linear_interpolation(orc):
    # A state linear in r* is reproduced exactly at r*_ext; a node hit exactly uses weights (1, 0).
    p = orc.params(n_rstar=41, n_theta=4, rstar_min=-10.0, rstar_max=30.0, rstar_ext=17.3)
    rs = -10.0 + np.arange(41) * 1.0
    u = np.zeros((4, 4, 41))
    for j in range(4):
        u[0, j] = 2.0 * rs + j
        u[1, j] = -rs
    _, w = orc.run(p, u, nsteps=0)
    for j in range(4):
        assert w[0, j, 0] == pytest.approx(2 * 17.3 + j, rel=1e-14)
        assert w[0, j, 1] == pytest.approx(-17.3, rel=1e-14)
    p.rstar_ext = 17.0
    _, w = orc.run(p, u, nsteps=0)
    assert w[0, 2, 0] == 2 * 17.0 + 2


def test_orbit_frequency_and_phase(orc):
    # a = 0: Kepler, Omega = r0^{-3/2}; phi0 = 0
    p = orc.params(a=0.0, r0=10.0)
    ob = orc.orbit(p)
    assert ob["Omega"] == pytest.approx(10.0 ** -1.5, rel=1e-15)
    assert ob["phi0"] == 0.0
    # Kerr prograde circular orbit (Bardeen-Press-Teukolsky): Omega = 1/(r0^{3/2} + a) at M = 1
    p = orc.params(a=0.9, r0=8.0)
    ob = orc.orbit(p)
    assert ob["Omega"] == pytest.approx(1.0 / (8.0 ** 1.5 + 0.9), rel=1e-15)
    # phi0(r0) is the Eq. (3) shift: d phi0/d r0 = a/Delta(r0), and phi0 -> 0 as r0 -> infinity
    h = 1e-5
    pp = orc.params(a=0.9, r0=8.0 + h)
    pm = orc.params(a=0.9, r0=8.0 - h)
    fd = (orc.orbit(pp)["phi0"] - orc.orbit(pm)["phi0"]) / (2 * h)
    assert fd == pytest.approx(0.9 / (64.0 - 16.0 + 0.81), rel=1e-8)
    assert ob["dphi0_dr0"] == pytest.approx(0.9 / (64.0 - 16.0 + 0.81), rel=1e-14)
    far = orc.params(a=0.9, r0=1e8, rstar_max=2e8, rstar_ext=10.0)
    assert abs(orc.orbit(far)["phi0"]) < 1e-8
    # r-derivative of Omega by finite differences
    fdO = (orc.orbit(pp)["Omega"] - orc.orbit(pm)["Omega"]) / (2 * h)
    assert ob["dOmega_dr0"] == pytest.approx(fdO, rel=1e-8)


def test_source_profile_normalisation_and_prefactor(orc):
    # P = [4 pi (r^2 + a^2 cos^2) Delta / (Sigma^2 r^3)] * G, G a unit-mass Gaussian.
    p = orc.params(n_rstar=801, n_theta=128, rstar_min=-50.0, rstar_max=150.0, a=0.9, r0=10.0,
                   rstar_ext=140.0)
    src = orc.orbit_source(p)
    g, ob = orc.grid(p), orc.orbit(p)
    th = (np.arange(128) + 0.5) * g["dth"]
    rs = -50.0 + np.arange(801) * g["drs"]
    # recover G by dividing out the prefactor, computed here from Eq. (1)'s right-hand side
    # and the tau conversion, then check its grid integral and its centre.
    a = 0.9
    G = np.zeros((128, 801))
    for i in range(801):
        x = orc.x_of_rstar(1.0, a, rs[i])
        r = g["rp"] + x
        Delta = x * (x + g["rp"] - g["rm"])
        Sig2 = (r * r + a * a) ** 2 - a * a * Delta * np.sin(th) ** 2
        pref = 4 * np.pi * (r * r + a * a * np.cos(th) ** 2) * Delta / (Sig2 * r ** 3)
        G[:, i] = src.P_int[:, i].real / pref
    assert np.abs(src.P_int.imag).max() == 0.0
    assert G.sum() * g["drs"] * g["dth"] == pytest.approx(1.0, rel=1e-6)
    jc, ic = np.unravel_index(np.argmax(G), G.shape)
    assert abs(rs[ic] - ob["rstar0"]) <= g["drs"] and abs(th[jc] - np.pi / 2) <= g["dth"]
    # truncated at 8 sigma
    far = np.abs(rs - ob["rstar0"]) > 8 * ob["sigma_r"] + 1e-12
    assert np.all(src.P_int[:, far] == 0)


def test_source_profile_r0_derivative(orc):
    h = 1e-5
    kw = dict(n_rstar=201, n_theta=32, rstar_min=-20.0, rstar_max=60.0, a=0.7, r0=9.0,
              rstar_ext=50.0)
    src = orc.orbit_source(orc.params(**kw))
    sp_ = orc.orbit_source(orc.params(**dict(kw, r0=9.0 + h)))
    sm_ = orc.orbit_source(orc.params(**dict(kw, r0=9.0 - h)))
    fd = (sp_.P_int - sm_.P_int) / (2 * h)
    scale = np.abs(src.dP_int).max()
    assert np.abs(fd - src.dP_int).max() <= 1e-6 * scale
    fdh = (sp_.P_half - sm_.P_half) / (2 * h)
    assert np.abs(fdh - src.dP_half).max() <= 1e-6 * scale
