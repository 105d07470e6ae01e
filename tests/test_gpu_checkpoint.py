"""Checkpoint / resume (teuk_save_state / teuk_load_state): a run saved after 20 steps and
resumed in a fresh context steps on bit for bit like the run that was saved (state and
waveform records), in every precision and for a batched context; a file of another
problem, or no saved state at all, is refused with TEUK_EINVAL and changes nothing."""
import numpy as np
import pytest

from paper_1001_3631_gb300 import TeukError, TeukSolver, inputs

pytestmark = pytest.mark.gpu

PARAMS = dict(s=-2, m=2, a=0.9, rstar_min=-20.0, rstar_max=60.0, n_rstar=333, n_theta=40,
              rstar_ext=30.0, dt_rule=1, courant=0.5)


def start(params, u0):
    s = TeukSolver(params)
    n = len(params) if isinstance(params, list) else 1
    for k in range(n):
        s.set_source(8.0, inputs.amplitudes(80, seed=4), instance=k)
        s.set_state(u0, 0, instance=k)
    return s


@pytest.mark.parametrize("prec", ["fp64", "fp64_df", "fp32_kahan", "fp32"])
def test_resume_from_saved_state_is_bitwise(prec, tmp_path):
    u0 = inputs.smooth_state(40, 333, seed=6)
    f = str(tmp_path / "ck.bin")
    with start(dict(PARAMS, prec=prec), u0) as a:
        a.step(20)
        a.save_state(f)
        a.step(15)
        ua = a.get_state()
        wa, fa = a.extract()
        a.sync()
    with start(dict(PARAMS, prec=prec), np.zeros_like(u0)) as b:
        b.load_state(f)
        assert b.time()[0] == 20
        b.step(15)
        ub = b.get_state()
        wb, fb = b.extract()
        b.sync()
    assert np.array_equal(ua, ub)
    # the resumed run holds the records from step 20 on; they equal the saved run's
    assert fb == 20 and np.array_equal(wb, wa[fb - fa:])


def test_resume_batched_context(tmp_path):
    u0 = inputs.smooth_state(40, 333, seed=7)
    ps = [dict(PARAMS, prec="fp32_kahan"), dict(PARAMS, m=3, prec="fp32_kahan")]
    with start(ps, u0) as a:
        a.step(10)
        for k in range(2):
            a.save_state(str(tmp_path / ("k%d" % k)), instance=k)
        a.step(12)
        ua = [a.get_state(instance=k) for k in range(2)]
        a.sync()
    with start(ps, np.zeros_like(u0)) as b:
        for k in range(2):
            b.load_state(str(tmp_path / ("k%d" % k)), instance=k)
        b.step(12)
        ub = [b.get_state(instance=k) for k in range(2)]
        b.sync()
    assert all(np.array_equal(x, y) for x, y in zip(ua, ub))


def test_load_refuses_another_problem_or_a_bad_file(tmp_path):
    u0 = inputs.smooth_state(40, 333, seed=8)
    f = str(tmp_path / "ck.bin")
    with start(dict(PARAMS, prec="fp64"), u0) as a:
        a.step(3)
        a.save_state(f)
    bad = tmp_path / "bad.bin"
    bad.write_bytes(b"not a state")
    for other in (dict(PARAMS, prec="fp64", m=3), dict(PARAMS, prec="fp32_kahan"),
                  dict(PARAMS, prec="fp64", n_theta=41)):
        with TeukSolver(other) as b:
            before = b.get_state()
            for path in (f, str(bad), str(tmp_path / "missing.bin")):
                with pytest.raises(TeukError) as e:
                    b.load_state(path)
                assert e.value.status == 1
            assert np.array_equal(b.get_state(), before) and b.time()[0] == 0
