"""Pins of the oracle's radiated fluxes (energy, linear momentum, angular momentum about
the spin axis; the recoil of Sec. 2.2) against closed forms and symmetries:

- a windowed monochromatic mode g''(t) (g = s(t) e^{-i w t}, s = sin^2(pi t / T)), whose
  time integrals are g' and g: the rates, the radiated totals and dJz/dt = m w s^2 / 2 ...
  within the trapezoid rule's error;
- records linear in t, for which the trapezoid sums have exact closed forms;
- two modes m, m+1: the x-y momentum is the product of their integrals (Fourier
  orthogonality of the azimuth integral), and zero for modes m, m+2;
- a rotation about the spin axis by alpha rotates (Px, Py) by alpha and leaves E, Pz,
  Jz unchanged; a reflection through the equatorial plane flips Pz only (any spin);
- far from the hole the spin drops out (the Kerr factor of psi_4 and the phi~ shift tend
  to 1 and 0)."""
import numpy as np
import pytest

NTH = 8


def _params(orc, m, a=0.0, dt=0.005, rstar_ext=17.0):
    return orc.params(s=-2, m=m, a=a, n_rstar=60, n_theta=NTH, rstar_min=-10.0,
                      rstar_max=max(30.0, 2.0 * rstar_ext), rstar_ext=rstar_ext, dt=dt)


def _rec(z):
    """complex [k][n_theta] -> records [k][n_theta][2]"""
    return np.stack([z.real, z.imag], axis=-1)


def _weights():
    dth = np.pi / NTH
    th = (np.arange(NTH) + 0.5) * dth
    return th, np.sin(th) * dth


def _window(T, w, t):
    """g = s e^{-iwt} with s = sin^2(pi t/T): g, g', g''"""
    k = np.pi / T
    s, s1, s2 = np.sin(k * t) ** 2, k * np.sin(2 * k * t), 2 * k * k * np.cos(2 * k * t)
    E = np.exp(-1j * w * t)
    return s * E, (s1 - 1j * w * s) * E, (s2 - 2j * w * s1 - w * w * s) * E


def test_windowed_monochromatic_mode(orc):
    T, w, m, dt = 20.0, 1.5, 2, 0.005
    nrec = int(round(T / dt)) + 1
    t = np.arange(nrec) * dt
    g, g1, g2 = _window(T, w, t)
    A = np.random.default_rng(1).standard_normal(NTH) + 1j * np.random.default_rng(2).standard_normal(NTH)
    out = orc.radiated_flux([_params(orc, m, dt=dt)], [_rec(g2[:, None] * A[None, :])])
    th, wj = _weights()
    S0 = (wj * np.abs(A) ** 2).sum()
    Sz = (wj * np.cos(th) * np.abs(A) ** 2).sum()
    dE = 0.5 * S0 * np.abs(g1) ** 2
    tol = 1e-4
    assert np.abs(out[:, 0] - dE).max() <= tol * dE.max()
    assert np.abs(out[:, 3] - 0.5 * Sz * np.abs(g1) ** 2).max() <= tol * dE.max()
    # one mode: no momentum in the equatorial plane (exactly, up to rounding)
    assert np.abs(out[:, 1:3]).max() <= 1e-13 * dE.max()
    # dJz/dt = m/2 S0 Im(conj(g') g) = m w s^2 S0 / 2 > 0: the prograde mode carries +Jz
    dJ = 0.5 * m * S0 * np.imag(np.conj(g1) * g)
    assert np.abs(out[:, 4] - dJ).max() <= tol * dJ.max() and dJ.max() > 0
    # totals over the window: int |g'|^2 = pi^2/(2T) + 3 w^2 T/8, int s^2 = 3T/8
    E_T = 0.5 * S0 * (np.pi ** 2 / (2 * T) + 3 * w * w * T / 8)
    J_T = 0.5 * m * S0 * w * 3 * T / 8
    assert abs(out[-1, 5] - E_T) <= tol * E_T
    assert abs(out[-1, 9] - J_T) <= tol * J_T


def test_records_linear_in_time_are_integrated_exactly(orc):
    m, dt, nrec = 3, 0.01, 301
    t = np.arange(nrec) * dt
    al, be = 0.7 - 0.2j, -0.3 + 1.1j
    A = np.linspace(0.5, 1.5, NTH) * np.exp(0.3j * np.arange(NTH))
    out = orc.radiated_flux([_params(orc, m, dt=dt)], [_rec((al + be * t)[:, None] * A[None, :])])
    th, wj = _weights()
    S0 = (wj * np.abs(A) ** 2).sum()
    N = al * t + be * t * t / 2                              # trapezoid: exact for linear
    H = al * t * t / 2 + be / 2 * (t ** 3 / 3 + dt * dt * t / 6)   # exact for quadratics
    assert np.allclose(out[:, 0], 0.5 * S0 * np.abs(N) ** 2, rtol=1e-12, atol=1e-14)
    assert np.allclose(out[:, 4], 0.5 * m * S0 * np.imag(np.conj(N) * H), rtol=1e-11, atol=1e-13)


def test_adjacent_modes_carry_momentum_in_the_plane(orc):
    T, dt = 20.0, 0.005
    nrec = int(round(T / dt)) + 1
    t = np.arange(nrec) * dt
    rng = np.random.default_rng(5)
    A = rng.standard_normal(NTH) + 1j * rng.standard_normal(NTH)
    B = rng.standard_normal(NTH) + 1j * rng.standard_normal(NTH)
    _, g1a, g2a = _window(T, 1.0, t)
    _, g1b, g2b = _window(T, 1.6, t)
    th, wj = _weights()
    for m2, adjacent in ((3, True), (4, False)):
        out = orc.radiated_flux([_params(orc, 2, dt=dt), _params(orc, m2, dt=dt)],
                                [_rec(g2a[:, None] * A[None, :]), _rec(g2b[:, None] * B[None, :])])
        Pp = out[:, 1] + 1j * out[:, 2]
        dE = 0.5 * (wj * np.abs(A) ** 2).sum() * np.abs(g1a) ** 2 + \
            0.5 * (wj * np.abs(B) ** 2).sum() * np.abs(g1b) ** 2
        assert np.abs(out[:, 0] - dE).max() <= 1e-4 * dE.max()
        if adjacent:
            # dPx + i dPy = 1/2 sum_j w_j sin th_j N_m conj(N_{m+1})
            want = 0.5 * (wj * np.sin(th) * A * np.conj(B)).sum() * g1a * np.conj(g1b)
            assert np.abs(Pp - want).max() <= 1e-4 * np.abs(want).max()
            assert np.abs(want).max() > 0.05 * dE.max()
        else:
            assert np.abs(Pp).max() <= 1e-13 * dE.max()


def _random_modes(orc, ms, a, nrec=200, seed=11):
    rng = np.random.default_rng(seed)
    ps = [_params(orc, m, a=a, dt=0.01) for m in ms]
    t = np.arange(nrec) * 0.01
    ws = []
    for m in ms:
        prof = rng.standard_normal(NTH) + 1j * rng.standard_normal(NTH)
        wv = 0.6 + 0.4 * rng.random()
        ws.append(_rec(np.sin(3 * t)[:, None] ** 2 * np.exp(-1j * m * wv * t)[:, None] * prof[None, :]))
    return ps, ws


@pytest.mark.parametrize("a", [0.0, 0.9])
def test_rotation_about_the_spin_axis(orc, a):
    ms = [1, 2, 3]
    ps, ws = _random_modes(orc, ms, a)
    out = orc.radiated_flux(ps, ws)
    alpha = 0.83
    rot = []
    for m, W in zip(ms, ws):
        z = (W[..., 0] + 1j * W[..., 1]) * np.exp(-1j * m * alpha)   # the field rotated by +alpha
        rot.append(_rec(z))
    o2 = orc.radiated_flux(ps, rot)
    sc = np.abs(out).max(axis=0)
    for q in (0, 3, 4, 5, 8, 9):
        assert np.abs(o2[:, q] - out[:, q]).max() <= 1e-12 * sc[q]
    for q in (1, 6):
        P, P2 = out[:, q] + 1j * out[:, q + 1], o2[:, q] + 1j * o2[:, q + 1]
        assert np.abs(P2 - np.exp(1j * alpha) * P).max() <= 1e-12 * np.abs(P).max()
        assert np.abs(P).max() > 1e-3 * sc[0 if q == 1 else 5]


@pytest.mark.parametrize("a", [0.0, 0.9])
def test_reflection_through_the_equatorial_plane(orc, a):
    ms = [-1, 0, 1, 2]
    ps, ws = _random_modes(orc, ms, a, seed=4)
    out = orc.radiated_flux(ps, ws)
    o2 = orc.radiated_flux(ps, [W[:, ::-1, :] for W in ws])
    sc = np.abs(out).max(axis=0)
    for q in range(10):
        sign = -1.0 if q in (3, 8) else 1.0
        assert np.abs(o2[:, q] - sign * out[:, q]).max() <= 1e-12 * sc.max()
    assert sc[3] > 1e-3 * sc[0]


def test_spin_drops_out_far_from_the_hole(orc):
    ms = [2, 3]
    res = []
    for a in (0.0, 0.9):
        rng = np.random.default_rng(9)
        ps = [_params(orc, m, a=a, dt=0.01, rstar_ext=1.0e6) for m in ms]
        ws = [rng.standard_normal((50, NTH, 2)) for _ in ms]
        res.append(orc.radiated_flux(ps, ws))
    sc = np.abs(res[0]).max(axis=0)
    # Kerr factor 1 + O(a^2/r^2) ~ 1e-12, phi~ shift -a/r ~ 1e-6 (rotates Px, Py only)
    for q in (0, 3, 4, 5, 8, 9):
        assert np.abs(res[1][:, q] - res[0][:, q]).max() <= 1e-10 * sc[q]
    for q in (1, 2, 6, 7):
        assert np.abs(res[1][:, q] - res[0][:, q]).max() <= 1e-5 * sc[q]


def test_cumulative_totals_integrate_the_rates(orc):
    """Records linear in t give polynomial rates (quartic energy rate), whose trapezoid
    sums have a closed form: the exact integral plus the terminating Euler-Maclaurin
    corrections h^2/12 [f'] - h^4/720 [f''']."""
    m, dt, nrec = 3, 0.01, 301
    t = np.arange(nrec) * dt
    al, be = 0.7 - 0.2j, -0.3 + 1.1j
    A = np.linspace(0.5, 1.5, NTH)
    out = orc.radiated_flux([_params(orc, m, dt=dt)], [_rec((al + be * t)[:, None] * A[None, :])])
    _, wj = _weights()
    S0 = (wj * A ** 2).sum()
    P = np.polynomial.Polynomial
    Nr, Ni = P([0.0, al.real, be.real / 2]), P([0.0, al.imag, be.imag / 2])
    f = 0.5 * S0 * (Nr * Nr + Ni * Ni)                   # dE/dt, degree 4
    F, f1, f3 = f.integ(), f.deriv(1), f.deriv(3)
    want = F(t) - F(0) + dt * dt / 12 * (f1(t) - f1(0)) - dt ** 4 / 720 * (f3(t) - f3(0))
    assert np.allclose(out[:, 5], want, rtol=1e-12, atol=1e-15)


def test_momentum_direction_follows_the_phi_shift_of_eq3(orc):
    """With a profile only on two rows mirror to each other about the equator, the spin
    scales every quantity by one common factor and turns the x-y momentum by -shift
    (e^{i m phi~} = e^{i m (phi + shift)}), the shift of Eq. (3) at the extraction radius;
    the shift is the orbit phase phi0 of a particle at that radius (pinned by
    d phi0 / d r0 = a / Delta)."""
    T, dt = 20.0, 0.005
    nrec = int(round(T / dt)) + 1
    t = np.arange(nrec) * dt
    _, _, g2a = _window(T, 1.0, t)
    _, _, g2b = _window(T, 1.7, t)
    A = np.zeros(NTH, complex)
    B = np.zeros(NTH, complex)
    A[2], A[NTH - 3], B[2], B[NTH - 3] = 1.0 + 0.5j, 0.3 - 1.0j, -0.7 + 0.2j, 0.9 + 0.4j
    res = {}
    for a in (0.0, 0.9):
        ps = [_params(orc, 2, a=a, dt=dt), _params(orc, 3, a=a, dt=dt)]
        res[a] = orc.radiated_flux(ps, [_rec(g2a[:, None] * A[None, :]), _rec(g2b[:, None] * B[None, :])])
    p9 = _params(orc, 2, a=0.9, dt=dt)
    r_ext = orc.orbit(p9)["r_ext"]
    shift = orc.orbit(orc.params(s=-2, m=2, a=0.9, n_rstar=60, n_theta=NTH, rstar_min=-10.0,
                                 rstar_max=30.0, rstar_ext=17.0, r0=r_ext))["phi0"]
    assert shift < -0.01
    kappa = res[0.9][-1, 5] / res[0.0][-1, 5]
    assert 0.5 < kappa < 1.0
    for q in (0, 3, 4, 5, 8, 9):
        assert np.allclose(res[0.9][:, q], kappa * res[0.0][:, q], rtol=1e-11,
                           atol=1e-12 * np.abs(res[0.0][:, q]).max())
    P0 = res[0.0][:, 1] + 1j * res[0.0][:, 2]
    P9 = res[0.9][:, 1] + 1j * res[0.9][:, 2]
    assert np.abs(P9 - kappa * np.exp(-1j * shift) * P0).max() <= 1e-11 * np.abs(P0).max()
