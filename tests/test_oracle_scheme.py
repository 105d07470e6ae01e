"""Pins of the oracle's time step (Eqs. 13-14 with the boundary treatment of Sec. 2.2).

Independent of the oracle: a 40-digit brute-force stepper whose coefficients come
from sympy's derivation of Eq. (1); superposition (the scheme is linear);
second-order convergence to a manufactured solution whose source is Eq. (1)
applied by sympy; the radial CFL limit of Lax-Wendroff; and the adjoint checked
by the dot-product identity and by finite differences."""
import math

import mpmath as mp
import numpy as np
import pytest

import derive


# --------------------------------------------------------------------------
# brute force: Eqs. (13)-(14) at 40 digits on a tiny grid
# --------------------------------------------------------------------------

def _brute_force(M, a, s, m, rs_min, rs_max, nr, nth, dt, u0, omega, phase0, P_int, P_half,
                 amps, nsteps, taus=None):
    """taus (optional): taus(n, half, j, i) -> the source at step n, half node i+1/2
    (half = 1, Eq. 13) or node i (half = 0, Eq. 14), replacing A_n e^{-i(omega t + phase0)} P."""
    co = derive.mpmath_coefficients(M, a, s, m)
    drs = (mp.mpf(rs_max) - rs_min) / (nr - 1)
    dth = mp.pi / nth
    ghost = 1 if abs(m + s) % 2 == 0 else -1

    def r_of(rs):
        y = mp.findroot(lambda yy: derive.tortoise_of_x(M, a, mp.e ** yy) - rs, mp.mpf(0))
        return M + mp.sqrt(M * M - a * a) + mp.e ** y

    def b_of(rr, tt):
        return mp.sqrt(-co["xx"](rr, tt)).real

    def coef(rs, tt):
        rr = r_of(rs)
        b = b_of(rr, tt)
        D = rr * rr - 2 * M * rr + a * a
        db = mp.diff(lambda x: b_of(x, tt), rr) * D / (rr * rr + a * a)   # db/dr* (Eq. 2)
        ct = co["t"](rr, tt)
        pst = -co["x"](rr, tt)
        return dict(b=b, ct=ct, Pst=ct * b + pst - b * db, w=-co["hh"](rr, tt),
                    wcot=-co["h"](rr, tt), qV=-co["0"](rr, tt))

    th = [(j + mp.mpf(1) / 2) * dth for j in range(nth)]
    ci = [[coef(rs_min + i * drs, th[j]) for i in range(nr)] for j in range(nth)]
    ch = [[coef(rs_min + (i + mp.mpf(1) / 2) * drs, th[j]) for i in range(nr - 1)]
          for j in range(nth)]
    Phi = [[mp.mpc(u0[0, j, i], u0[1, j, i]) for i in range(nr)] for j in range(nth)]
    Pi = [[mp.mpc(u0[2, j, i], u0[3, j, i]) for i in range(nr)] for j in range(nth)]

    def row(F, jj):
        if jj < 0:
            return [ghost * v for v in F[0]]
        if jj >= nth:
            return [ghost * v for v in F[nth - 1]]
        return F[jj]

    def S_Pi(k, Fb_m, Fb, Fb_p, Pb, dF, tau):
        D2 = (Fb_p - 2 * Fb + Fb_m) / dth ** 2
        D1 = (Fb_p - Fb_m) / (2 * dth)
        return -k["ct"] * Pb + k["Pst"] * dF + k["w"] * D2 + k["wcot"] * D1 + k["qV"] * Fb + tau

    for n in range(nsteps):
        A = amps[n] if amps is not None else 1
        t = n * mp.mpf(dt)
        ep = A * mp.expj(-(omega * t + phase0))
        ec = A * mp.expj(-(omega * (t + mp.mpf(dt) / 2) + phase0))
        hF = [[None] * (nr - 1) for _ in range(nth)]
        hP = [[None] * (nr - 1) for _ in range(nth)]
        for j in range(nth):
            Fm, F0, Fp = row(Phi, j - 1), Phi[j], row(Phi, j + 1)
            for i in range(nr - 1):
                k = ch[j][i]
                Fb = (F0[i + 1] + F0[i]) / 2
                Pb = (Pi[j][i + 1] + Pi[j][i]) / 2
                dF = (F0[i + 1] - F0[i]) / drs
                dP = (Pi[j][i + 1] - Pi[j][i]) / drs
                sp_ = S_Pi(k, (Fm[i + 1] + Fm[i]) / 2, Fb, (Fp[i + 1] + Fp[i]) / 2, Pb, dF,
                           taus(n, 1, j, i) if taus else
                           ep * mp.mpc(P_half[j, i].real, P_half[j, i].imag))
                hF[j][i] = Fb - mp.mpf(dt) / 2 * (k["b"] * dF - Pb)
                hP[j][i] = Pb - mp.mpf(dt) / 2 * (-k["b"] * dP - sp_)
        nF = [[mp.mpc(0)] * nr for _ in range(nth)]
        nP = [[mp.mpc(0)] * nr for _ in range(nth)]
        for j in range(nth):
            Hm, H0, Hp = row(hF, j - 1), hF[j], row(hF, j + 1)
            for i in range(1, nr - 1):
                k = ci[j][i]
                Fb = (H0[i] + H0[i - 1]) / 2
                Pb = (hP[j][i] + hP[j][i - 1]) / 2
                dF = (H0[i] - H0[i - 1]) / drs
                dP = (hP[j][i] - hP[j][i - 1]) / drs
                sp_ = S_Pi(k, (Hm[i] + Hm[i - 1]) / 2, Fb, (Hp[i] + Hp[i - 1]) / 2, Pb, dF,
                           taus(n, 0, j, i) if taus else
                           ec * mp.mpc(P_int[j, i].real, P_int[j, i].imag))
                nF[j][i] = Phi[j][i] - mp.mpf(dt) * (k["b"] * dF - Pb)
                nP[j][i] = Pi[j][i] - mp.mpf(dt) * (-k["b"] * dP - sp_)
        Phi, Pi = nF, nP
    out = np.zeros((4, nth, nr))
    for j in range(nth):
        for i in range(nr):
            out[0, j, i], out[1, j, i] = float(Phi[j][i].real), float(Phi[j][i].imag)
            out[2, j, i], out[3, j, i] = float(Pi[j][i].real), float(Pi[j][i].imag)
    return out


@pytest.mark.parametrize("m", [2, 3])
def test_bruteforce_tiny_grid(orc, m):
    M, a, s = 1.0, 0.6, -2
    nr, nth, dt, nsteps = 7, 4, 0.01, 3
    rng = np.random.default_rng(17 + m)
    u0 = rng.standard_normal((4, nth, nr))
    P_int = rng.standard_normal((nth, nr)) + 1j * rng.standard_normal((nth, nr))
    P_half = rng.standard_normal((nth, nr - 1)) + 1j * rng.standard_normal((nth, nr - 1))
    amps = [1.1, 0.9, 1.05]
    p = orc.params(M=M, a=a, s=s, m=m, rstar_min=-4.0, rstar_max=8.0, n_rstar=nr, n_theta=nth,
                   dt=dt, rstar_ext=0.0, r0=5.0)
    src = orc.Source(0.37, 0.2, P_int, P_half)
    u, _ = orc.run(p, u0, nsteps, src, amps=np.array(amps))
    with mp.workdps(40):
        ref = _brute_force(M, a, s, m, -4.0, 8.0, nr, nth, dt, u0, 0.37, 0.2, P_int, P_half,
                           amps, nsteps)
    assert np.abs(u - ref).max() <= 1e-13 * np.abs(ref).max()


# --------------------------------------------------------------------------
# linearity / superposition
# --------------------------------------------------------------------------

def test_superposition_and_scaling(orc):
    p = orc.params(n_rstar=120, n_theta=16, rstar_min=-20.0, rstar_max=40.0, rstar_ext=30.0,
                   r0=7.0, a=0.8, m=3)
    rng = np.random.default_rng(5)
    nth, nr = 16, 120
    mk = lambda: (rng.standard_normal((nth, nr)) + 1j * rng.standard_normal((nth, nr)),
                  rng.standard_normal((nth, nr - 1)) + 1j * rng.standard_normal((nth, nr - 1)))
    (A1, B1), (A2, B2) = mk(), mk()
    s1 = orc.Source(0.2, 0.1, A1, B1)
    s2 = orc.Source(0.2, 0.1, A2, B2)
    s12 = orc.Source(0.2, 0.1, A1 + A2, B1 + B2)
    s3 = orc.Source(0.2, 0.1, 2.5 * A1, 2.5 * B1)
    u0 = rng.standard_normal((4, nth, nr))
    n = 40
    u1, w1 = orc.run(p, None, n, s1)
    u2, w2 = orc.run(p, None, n, s2)
    u12, w12 = orc.run(p, None, n, s12)
    u3, _ = orc.run(p, None, n, s3)
    uh, _ = orc.run(p, u0, n, None)
    uf, _ = orc.run(p, u0, n, s1)
    sc = np.abs(u12).max()
    assert np.abs(u12 - (u1 + u2)).max() <= 1e-13 * sc
    assert np.abs(w12 - (w1 + w2)).max() <= 1e-13 * np.abs(w12).max()
    assert np.abs(u3 - 2.5 * u1).max() <= 1e-13 * np.abs(u3).max()
    assert np.abs(uf - (uh + u1)).max() <= 1e-13 * np.abs(uf).max()


# --------------------------------------------------------------------------
# manufactured solution: second-order convergence in (dr*, dtheta, dt)
# --------------------------------------------------------------------------

@pytest.mark.parametrize("m", [2, 1])
def test_manufactured_solution_second_order(orc, m):
    M, a, s = 1.0, 0.5, -2
    omega0, rc, ell, T = 0.3, 10.0, 3.0, 1.5
    fQ, fPhi, fPi = derive.mms_source(M, a, s, m, omega0, rc, ell)
    rp = M + math.sqrt(M * M - a * a)

    def r_nodes(rs):
        with mp.workdps(30):
            return np.array([rp + float(mp.e ** mp.findroot(
                lambda yy: derive.tortoise_of_x(M, a, mp.e ** yy) - mp.mpf(float(x)),
                (-100, 10), solver="illinois")) for x in rs])

    errs = []
    for lev in range(3):
        nr, nth, nsteps = 120 * 2 ** lev + 1, 16 * 2 ** lev, 100 * 2 ** lev
        rs = np.linspace(-20.0, 40.0, nr)
        rsh = 0.5 * (rs[1:] + rs[:-1])
        th = (np.arange(nth) + 0.5) * np.pi / nth
        ri, rh = r_nodes(rs), r_nodes(rsh)
        R, TH = np.meshgrid(ri, th)
        RS, _ = np.meshgrid(rs, th)
        RH, THh = np.meshgrid(rh, th)
        RSH, _ = np.meshgrid(rsh, th)
        P_int = fQ(R, RS, TH) + 0j
        P_half = fQ(RH, RSH, THh) + 0j
        u0 = np.zeros((4, nth, nr))
        F0 = fPhi(0.0, RS, TH) + 0j
        Pi0 = fPi(0.0, R, RS, TH) + 0j
        u0[0], u0[1], u0[2], u0[3] = F0.real, F0.imag, Pi0.real, Pi0.imag
        p = orc.params(M=M, a=a, s=s, m=m, rstar_min=-20.0, rstar_max=40.0, n_rstar=nr,
                       n_theta=nth, dt=T / nsteps, rstar_ext=0.0, r0=6.0)
        u, _ = orc.run(p, u0, nsteps, orc.Source(omega0, 0.0, P_int, P_half), wave=False)
        FT = fPhi(T, RS, TH) + 0j
        errs.append(np.abs(u[0] + 1j * u[1] - FT).max())
    r1, r2 = errs[0] / errs[1], errs[1] / errs[2]
    assert 3.5 < r1 < 4.5 and 3.5 < r2 < 4.5, errs


# --------------------------------------------------------------------------
# stability: the radial CFL limit and the literal Courant rule
# --------------------------------------------------------------------------

@pytest.mark.parametrize("a,rs_min,rs_max,nth", [(0.0, 10.0, 60.0, 4), (0.9, -5.0, 20.0, 8)])
def test_radial_cfl_limit(orc, a, rs_min, rs_max, nth):
    # Lax-Wendroff for d_t u + b d_r* u is stable iff b dt/dr* <= 1.  With s = m = 0
    # and a coarse angular grid the angular terms are benign, so the limit seen is the
    # radial one: C b_max = 0.97 grows no more than C b_max = 0.90 does (Phi = Psi/r^3
    # itself grows when the field moves inward), C b_max = 1.03 grows without bound.
    nr = 101
    base = dict(s=0, m=0, a=a, rstar_min=rs_min, rstar_max=rs_max, n_rstar=nr, n_theta=nth,
                rstar_ext=rs_min + 1.0, dt_rule=0)
    p = orc.params(**base)
    g = orc.grid(p)
    bmax = 0.0
    for i in range(2 * nr - 1):
        x = orc.x_of_rstar(1.0, a, rs_min + 0.5 * i * g["drs"])
        for j in range(nth):
            bmax = max(bmax, orc.coeffs(p, x, (j + 0.5) * g["dth"])["b"])
    rng = np.random.default_rng(3)
    u0 = rng.standard_normal((4, nth, nr))
    growth = {}
    for f in (0.90, 0.97, 1.03):
        p = orc.params(**dict(base, courant=f / bmax))
        u, _ = orc.run(p, u0, int(400 * 0.97 / f), None, wave=False)
        growth[f] = np.abs(u).max() / np.abs(u0).max()
    assert growth[0.97] < 2.0 * growth[0.90], growth
    assert growth[1.03] > 1e6 * growth[0.97], growth


def test_literal_courant_rule_is_unstable_on_the_single_mode_grid(orc):
    # dt = 0.5 dr* (rule 0) on the 800 x 64 grid: the explicitly integrated angular
    # terms (pole potential up to (|m|+|s|)^2/sin^2) make the step amplify by orders of
    # magnitude; this is why dt_rule 1 exists.
    p = orc.params(dt_rule=0, courant=0.5)
    u, _ = orc.run(p, None, 200, orc.orbit_source(p), wave=False)
    assert not np.isfinite(np.abs(u).max()) or np.abs(u).max() > 1e50
    p = orc.params(dt_rule=1, courant=0.5)
    u, _ = orc.run(p, None, 200, orc.orbit_source(p), wave=False)
    assert np.abs(u).max() < 1.0


# --------------------------------------------------------------------------
# adjoint
# --------------------------------------------------------------------------

@pytest.mark.parametrize("m", [2, 3])
def test_adjoint_dot_product(orc, m):
    p = orc.params(n_rstar=24, n_theta=6, rstar_min=-10.0, rstar_max=20.0, rstar_ext=15.0,
                   r0=6.0, a=0.9, m=m, dt=0.05)
    rng = np.random.default_rng(11)
    x = rng.standard_normal((4, 6, 24))
    y = rng.standard_normal((4, 6, 24))
    lhs = np.sum(orc.apply_K(p, x) * y)
    rhs = np.sum(x * orc.apply_KT(p, y))
    assert abs(lhs - rhs) <= 1e-13 * (np.abs(orc.apply_K(p, x)).sum() * np.abs(y).max())


def _loss(orc, p, amps, nsteps):
    src = orc.orbit_source(p)
    _, w = orc.run(p, None, nsteps, src, amps=amps)
    re = orc.r_ext(p)
    return np.sum(re ** 6 * (w[1:, :, 0] ** 2 + w[1:, :, 1] ** 2)), w


@pytest.mark.parametrize("m", [2, 1])
def test_adjoint_gradients_vs_finite_differences(orc, m):
    nsteps = 30
    kw = dict(n_rstar=60, n_theta=8, rstar_min=-10.0, rstar_max=30.0, rstar_ext=14.0, r0=8.0,
              a=0.7, m=m, dt_rule=1, courant=0.5)
    p = orc.params(**kw)
    rng = np.random.default_rng(5005)
    amps = 1.0 + 0.1 * rng.standard_normal(nsteps)
    L, w = _loss(orc, p, amps, nsteps)
    re = orc.r_ext(p)
    gwave = 2.0 * re ** 6 * w[1:]                 # dL/dW for L = sum r_ext^6 |W|^2
    ga, gr, _ = orc.adjoint(p, orc.orbit_source(p), gwave, amps=amps)
    h = 1e-6
    for k in [0, 7, 18, 29]:
        ap, am = amps.copy(), amps.copy()
        ap[k] += h
        am[k] -= h
        fd = (_loss(orc, p, ap, nsteps)[0] - _loss(orc, p, am, nsteps)[0]) / (2 * h)
        # L is quadratic in A: central differences are exact up to rounding
        assert ga[k] == pytest.approx(fd, rel=1e-7, abs=1e-9 * abs(L) / h * 1e-6)
    Lp = _loss(orc, orc.params(**dict(kw, r0=8.0 + h)), amps, nsteps)[0]
    Lm = _loss(orc, orc.params(**dict(kw, r0=8.0 - h)), amps, nsteps)[0]
    assert gr == pytest.approx((Lp - Lm) / (2 * h), rel=1e-6)
