"""Radiated energy, momentum and Jz fluxes (the recoil of Sec. 2.2) on the GPU against the
oracle: the modes of one particle on a circular orbit run as instances of one context,
their fluxes from the records (chunked time scans, per-record sums over a block per chunk
and group of rows) compared with the oracle's plain record-by-record integrals, end to
end (oracle run + oracle fluxes) and on the same records; ragged chunks, many records
and chunks, and the argument errors."""
import numpy as np
import pytest

from paper_1001_3631_gb300 import TeukError, TeukSolver, inputs

pytestmark = pytest.mark.gpu

BASE = dict(s=-2, a=0.9, rstar_min=-10.0, rstar_max=30.0, n_rstar=120, n_theta=16,
            rstar_ext=13.0, dt=0.004)


def _close(g, o, tol):
    """every column within tol of that quantity's largest magnitude"""
    sc = np.abs(o).max(axis=0)
    assert np.all(sc > 0)
    assert np.all(np.abs(g - o).max(axis=0) <= tol * sc), (np.abs(g - o).max(axis=0) / sc)


def _oracle_modes(orc, ms, u0, n, base=BASE, r0=7.0):
    ps, waves = [], []
    for m in ms:
        p = orc.params(**dict(base, m=m), r0=r0)
        _, w = orc.run(p, u0, n, orc.orbit_source(p))
        ps.append(p)
        waves.append(w)
    return ps, waves


def test_flux_end_to_end_against_oracle(orc):
    ms = [-1, 0, 1, 2, 3]
    n = 400
    u0 = inputs.smooth_state(16, 120, seed=5)
    with TeukSolver([dict(BASE, m=m, prec="fp64") for m in ms]) as s:
        for k in range(len(ms)):
            s.set_source(7.0, instance=k)
            s.set_state(u0, 0, instance=k)
        s.step(n)
        g = s.radiated_flux(0, n + 1)
        g_late = s.radiated_flux(150, n - 149)      # totals from record 150
        s.sync()
    ps, waves = _oracle_modes(orc, ms, u0, n)
    o = orc.radiated_flux(ps, waves)
    assert g.shape == o.shape == (n + 1, 10)
    _close(g, o, 1e-11)
    o_late = orc.radiated_flux(ps, [w[150:] for w in waves])
    _close(g_late, o_late, 1e-11)
    assert np.all(g[0] == 0.0)                     # nothing integrated at the first record
    # adjacent modes radiate momentum in the plane; the field is not mirror-symmetric
    assert np.abs(g[:, 1:3]).max() > 1e-6 * np.abs(g[:, 0]).max()


def test_flux_on_fp32_kahan_records_same_records(orc):
    ms = [1, 2, 3, 5]                               # 3 has a partner, 5 has none
    n = 257
    u0 = inputs.smooth_state(16, 120, seed=6)
    with TeukSolver([dict(BASE, m=m, prec="fp32_kahan") for m in ms]) as s:
        for k in range(len(ms)):
            s.set_source(7.0, instance=k)
            s.set_state(u0, 0, instance=k)
        s.step(n)
        recs = [s.extract(instance=k)[0] for k in range(len(ms))]
        g = s.radiated_flux(0, n + 1)
        s.sync()
    ps = [orc.params(**dict(BASE, m=m), r0=7.0) for m in ms]
    _close(g, orc.radiated_flux(ps, recs), 1e-11)


def test_flux_many_records_and_chunks(orc):
    """8 modes x 128 rows and 12 001 records: 152 chunks of 79 records (the chain of
    chunk starts longer than its eight-load batches), 4 row groups of 32."""
    ms = list(range(-2, 6))
    base = dict(s=-2, a=0.6, rstar_min=-10.0, rstar_max=30.0, n_rstar=48, n_theta=128,
                rstar_ext=9.0, dt=0.001, wave_capacity=16384)
    n = 12000
    with TeukSolver([dict(base, m=m, prec="fp64") for m in ms]) as s:
        for k in range(len(ms)):
            s.set_source(6.0, instance=k)
        s.step(n)
        recs = [s.extract(instance=k)[0] for k in range(len(ms))]
        g = s.radiated_flux(0, n + 1)
        s.sync()
    ps = [orc.params(**{k: v for k, v in base.items() if k != "wave_capacity"}, m=m, r0=6.0)
          for m in ms]
    assert all(r.shape[0] == n + 1 for r in recs)
    _close(g, orc.radiated_flux(ps, recs), 1e-10)


def test_flux_edge_cases_and_errors(orc):
    with TeukSolver([dict(BASE, m=2, prec="fp64"), dict(BASE, m=3, prec="fp64")]) as s:
        for k in range(2):
            s.set_source(7.0, instance=k)
        s.step(5)
        assert s.radiated_flux(0, 0).shape == (0, 10)
        one = s.radiated_flux(3, 1)
        assert np.all(one == 0.0)                     # a single record: nothing integrated
        two = s.radiated_flux(4, 2)
        assert two.shape == (2, 10) and np.all(np.isfinite(two))
        with pytest.raises(TeukError):                # level 6 is not held yet
            s.radiated_flux(0, 7)
        s.sync()
    with TeukSolver([dict(BASE, m=2, prec="fp64"), dict(BASE, m=2, prec="fp64")]) as s:
        s.step(2)
        with pytest.raises(TeukError) as e:           # the same mode twice
            s.radiated_flux(0, 3)
        assert e.value.status == 1
    with TeukSolver([dict(BASE, m=2, prec="fp64"), dict(BASE, m=3, prec="fp64", a=0.5)]) as s:
        s.step(2)
        with pytest.raises(TeukError):                # not one problem
            s.radiated_flux(0, 3)
