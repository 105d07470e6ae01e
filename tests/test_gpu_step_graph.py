"""Per-step launches replayed from the cached CUDA graphs of 64 steps (teuk_step_n with
n >= 64 on a single instance) equal one direct launch per step bit for bit, across a
graph's end, after the state or the time level is replaced (the step base is re-read),
after the source changes (the graph is captured again) and from either buffer parity."""
import numpy as np
import pytest

from paper_1001_3631_gb300 import TeukSolver, inputs

pytestmark = pytest.mark.gpu

PARAMS = dict(s=-2, m=2, a=0.9, rstar_min=-20.0, rstar_max=60.0, n_rstar=300, n_theta=32,
              rstar_ext=30.0, dt_rule=1, courant=0.5)


def run(prec, chunks, u0, changes=None):
    with TeukSolver(dict(PARAMS, prec=prec)) as s:
        s.set_source(8.0, inputs.amplitudes(600, seed=1))
        s.set_state(u0, 5)
        for i, n in enumerate(chunks):
            if changes and i in changes:
                changes[i](s)
            if n > 0:
                s.step(n)
            else:
                for _ in range(-n):   # -n single-step calls: direct launches
                    s.step(1)
        u = s.get_state()
        w, first = s.extract()
        s.sync()
        return u, w, first


@pytest.mark.parametrize("prec", ["fp32_kahan", "fp64", "fp64_df", "fp32"])
def test_graph_replay_equals_direct_launches(prec):
    u0 = inputs.smooth_state(32, 300, seed=2)
    ref = run(prec, [-1, -150, -71], u0)
    got = run(prec, [1, 150, 71], u0)   # odd start parity, 2 graphs + 22, 1 graph + 7
    assert got[2] == ref[2]
    assert np.array_equal(got[0], ref[0]) and np.array_equal(got[1], ref[1])


def test_graph_follows_state_time_and_source_changes():
    u0 = inputs.smooth_state(32, 300, seed=3)
    u1 = inputs.smooth_state(32, 300, seed=4)
    changes = {1: lambda s: s.set_state(u1, 40),
               2: lambda s: s.set_source(9.0, inputs.amplitudes(600, seed=7))}
    ref = run("fp32_kahan", [-70, -130, -65], u0, changes)
    got = run("fp32_kahan", [70, 130, 65], u0, changes)
    assert got[2] == ref[2]
    assert np.array_equal(got[0], ref[0]) and np.array_equal(got[1], ref[1])


def test_graph_follows_tiling_changes():
    # a new strip length, then the default again, between graph replays: each change
    # captures a new graph, and the results stay those of direct launches
    u0 = inputs.smooth_state(32, 300, seed=5)
    ref = run("fp32_kahan", [-70, -70, -70], u0)
    changes = {1: lambda s: s.set_instance_tiling(0, 9), 2: lambda s: s.set_instance_tiling(0, 0)}
    got = run("fp32_kahan", [70, 70, 70], u0, changes)
    assert got[2] == ref[2]
    assert np.array_equal(got[0], ref[0]) and np.array_equal(got[1], ref[1])
