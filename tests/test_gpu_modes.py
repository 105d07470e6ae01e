"""Waveform summed over modes (Eqs. 3-4) on the GPU against the oracle: the modes
m = -3..3 of one particle on a circular orbit (each with its own phase e^{-im(Omega t +
phi0)}), run as instances of one batched context with a shared time step."""
import numpy as np
import pytest

from paper_1001_3631_gb300 import TeukError, TeukSolver, inputs

pytestmark = pytest.mark.gpu

MS = [-3, -2, -1, 0, 1, 2, 3]
BASE = dict(s=-2, a=0.9, rstar_min=-10.0, rstar_max=30.0, n_rstar=120, n_theta=16,
            rstar_ext=13.0, dt=0.004)


def rel(a, b):
    return np.linalg.norm(a - b) / np.linalg.norm(b)


@pytest.mark.parametrize("prec,tol", [("fp64", 1e-12), ("fp32_kahan", 1e-6)])
def test_mode_sum_against_oracle(orc, prec, tol):
    n = 60
    u0 = inputs.smooth_state(16, 120, seed=3)
    with TeukSolver([dict(BASE, m=m, prec=prec) for m in MS]) as s:
        for k in range(len(MS)):
            s.set_source(7.0, instance=k)
            s.set_state(u0, 0, instance=k)
        s.step(n)
        phi = np.linspace(0.0, 2 * np.pi, 9)
        h = s.mode_sum(phi, 10, n - 9)       # time levels 10 .. 60
        s.sync()
    ps, waves = [], []
    for m in MS:
        p = orc.params(**dict(BASE, m=m), r0=7.0)
        _, w = orc.run(p, u0, n, orc.orbit_source(p))
        ps.append(p)
        waves.append(w[10:])
    ho = orc.mode_sum(ps, waves, phi)
    assert h.shape == ho.shape == (n - 9, 16, 9)
    assert rel(h, ho) <= tol


def test_mode_sum_argument_errors():
    with TeukSolver([dict(BASE, m=2, prec="fp64"), dict(BASE, m=3, prec="fp64", dt=0.003)]) as s:
        s.step(3)
        with pytest.raises(TeukError) as e:          # not one problem: different steps
            s.mode_sum([0.0], 0, 4)
        assert e.value.status == 1
    with TeukSolver([dict(BASE, m=2, prec="fp64"), dict(BASE, m=3, prec="fp64")]) as s:
        s.step(3)
        with pytest.raises(TeukError):               # level 4 is not held yet
            s.mode_sum([0.0], 0, 5)
        assert s.mode_sum([0.0, 1.0], 1, 3).shape == (3, 16, 2)
        assert s.mode_sum([0.0], 0, 0).shape == (0, 16, 1)
        s.sync()
