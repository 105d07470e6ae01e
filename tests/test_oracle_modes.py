"""Pins of the oracle's sum over modes (the field of Eqs. 3-4 at the extraction radius):
a discrete Fourier transform over a uniform azimuth grid (numpy's FFT, independent of
the summation) recovers each mode's r^3 e^{i m shift} W_m, with the shift of Eq. (3)
that the circular-orbit phase phi0 also uses (pinned there by d phi0/d r0 = a/Delta)."""
import numpy as np
import pytest


@pytest.mark.parametrize("a", [0.0, 0.9])
def test_fourier_transform_over_phi_recovers_each_mode(orc, a):
    ms = [-3, -2, -1, 0, 1, 2, 3]
    ps = [orc.params(s=-2, m=m, a=a, n_rstar=60, n_theta=8, rstar_min=-10.0, rstar_max=30.0,
                     rstar_ext=17.0, dt=0.004) for m in ms]
    rng = np.random.default_rng(8)
    waves = [rng.standard_normal((5, 8, 2)) for _ in ms]
    L = 16
    phi = 2 * np.pi * np.arange(L) / L
    h = orc.mode_sum(ps, waves, phi)
    F = np.fft.fft(h, axis=2) / L          # F[q] = sum over modes with m = q (mod L)
    r_ext = orc.orbit(ps[0])["r_ext"]
    shift = orc.orbit(orc.params(s=-2, m=2, a=a, n_rstar=60, n_theta=8, rstar_min=-10.0,
                                 rstar_max=30.0, rstar_ext=17.0, r0=r_ext))["phi0"]
    if a == 0.0:
        assert shift == 0.0
    for m, W in zip(ms, waves):
        want = r_ext ** 3 * np.exp(1j * m * shift) * (W[..., 0] + 1j * W[..., 1])
        assert np.abs(F[:, :, m % L] - want).max() <= 1e-12 * np.abs(want).max()
    # the extraction radius is r(r*_ext) of Eq. (2)
    assert abs(orc.rstar_of_r(1.0, a, r_ext) - 17.0) < 1e-12


def test_single_axisymmetric_mode_is_r_cubed_times_the_record(orc):
    p = orc.params(s=-2, m=0, a=0.5, n_rstar=60, n_theta=8, rstar_min=-10.0, rstar_max=30.0,
                   rstar_ext=17.0, dt=0.004)
    W = np.random.default_rng(2).standard_normal((3, 8, 2))
    h = orc.mode_sum([p], [W], [0.0, 1.0, 4.0])
    r3 = orc.orbit(p)["r_ext"] ** 3
    for l in range(3):
        assert np.allclose(h[:, :, l], r3 * (W[..., 0] + 1j * W[..., 1]), rtol=1e-15, atol=0)
