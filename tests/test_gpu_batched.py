"""Batched persistent kernel: many uneven instances in one launch (CUDA graph replay),
checked bit for bit against the one-kernel-per-step path, against the oracle, and for
its bounded waits (a completion flag that is never published must surface as
TEUK_ETIMEOUT, not a hang)."""
import numpy as np
import pytest

from paper_1001_3631_gb300 import TeukError, TeukSolver, inputs

pytestmark = pytest.mark.gpu

INST = [  # uneven grids, both pole parities, different spins, orbits and start levels
    dict(params=dict(s=-2, m=2, a=0.9, rstar_min=-10.0, rstar_max=30.0, n_rstar=97, n_theta=12,
                     rstar_ext=20.0, dt_rule=1, courant=0.5), r0=6.0, step0=0),
    dict(params=dict(s=-2, m=3, a=0.7, rstar_min=-20.0, rstar_max=40.0, n_rstar=151, n_theta=33,
                     rstar_ext=35.0, dt_rule=1, courant=0.5), r0=8.0, step0=11),
    dict(params=dict(s=-2, m=1, a=0.0, rstar_min=-10.0, rstar_max=30.0, n_rstar=64, n_theta=8,
                     rstar_ext=29.9, dt_rule=1, courant=0.5), r0=7.0, step0=3),
    dict(params=dict(s=-2, m=4, a=0.5, rstar_min=-30.0, rstar_max=90.0, n_rstar=400, n_theta=64,
                     rstar_ext=40.0, dt_rule=1, courant=0.5), r0=9.0, step0=0),
]


def rel(a, b):
    nb = np.linalg.norm(b)
    return np.linalg.norm(a - b) / (nb if nb > 0 else 1.0)


def run_single(inst, prec, steps, strip, persistent=False):
    with TeukSolver(dict(inst["params"], prec=prec)) as s:
        s.set_tiling(strip, 0 if persistent else 1)
        s.set_source(inst["r0"], inputs.amplitudes(100, seed=inst["step0"] + 1))
        u0 = inputs.random_state(inst["params"]["n_theta"], inst["params"]["n_rstar"], seed=2)
        s.set_state(u0, inst["step0"])
        for n in steps:
            s.step(n)
        u = s.get_state()
        w, first = s.extract()
        s.sync()
    return u, w, first


def run_batched(prec, steps, strip, stream=None):
    with TeukSolver([dict(i["params"], prec=prec) for i in INST], stream=stream) as s:
        s.set_tiling(strip, 1)
        for k, inst in enumerate(INST):
            s.set_source(inst["r0"], inputs.amplitudes(100, seed=inst["step0"] + 1), instance=k)
            u0 = inputs.random_state(inst["params"]["n_theta"], inst["params"]["n_rstar"], seed=2)
            s.set_state(u0, inst["step0"], instance=k)
        for n in steps:
            s.step(n)
        out = []
        for k in range(len(INST)):
            w, first = s.extract(instance=k)
            out.append((s.get_state(k), w, first))
        s.sync()
        launches = s.kernel_launches()
    return out, launches


@pytest.mark.parametrize("prec,graph", [("fp64", True), ("fp32_kahan", True), ("fp64", False)])
def test_batched_equals_per_step_launches_bitwise(prec, graph):
    # the persistent launch is captured in a CUDA graph (on the context's private stream)
    # and replayed on the caller's stream: a side stream or the legacy default stream
    import torch
    stream = torch.cuda.Stream() if graph else None
    steps = [37, 5, 1]
    res, launches = run_batched(prec, steps, 8, stream)
    for k, inst in enumerate(INST):
        u, w, first = run_single(inst, prec, steps, 8)
        assert first == res[k][2] == inst["step0"]
        assert np.array_equal(u, res[k][0]), k
        assert np.array_equal(w, res[k][1]), k


def test_batched_fp64_matches_oracle(orc):
    steps = [20, 7]
    res, _ = run_batched("fp64", steps, 0)
    for k, inst in enumerate(INST):
        p = orc.params(**inst["params"], r0=inst["r0"])
        u0 = inputs.random_state(inst["params"]["n_theta"], inst["params"]["n_rstar"], seed=2)
        uo, wo = orc.run(p, u0, sum(steps), orc.orbit_source(p),
                         amps=inputs.amplitudes(100, seed=inst["step0"] + 1), step0=inst["step0"])
        assert rel(res[k][0], uo) <= 1e-12
        assert rel(res[k][1], wo) <= 1e-12


def test_single_instance_through_the_persistent_kernel():
    inst = INST[3]
    a = run_single(inst, "fp32_kahan", [9, 4], 16, persistent=False)
    b = run_single(inst, "fp32_kahan", [9, 4], 16, persistent=True)
    assert np.array_equal(a[0], b[0]) and np.array_equal(a[1], b[1])


def test_bounded_wait_gives_up_and_reports_timeout():
    with TeukSolver([dict(i["params"], prec="fp64") for i in INST[:2]]) as s:
        s.set_tiling(4, 1)
        # item 0 of the first step never publishes its completion; its neighbours'
        # waits run out after 20000 polls (a few ms) instead of hanging
        s.set_fault_injection(skip_release_item=0, spin_limit=20000)
        s.step(3)
        with pytest.raises(TeukError) as e:
            s.sync()
        assert e.value.status == 5  # TEUK_ETIMEOUT
        # the context stays usable: clear the injection, reset the state, run again
        s.set_fault_injection(-1, 0)
        for k, inst in enumerate(INST[:2]):
            s.set_state(np.zeros((4, inst["params"]["n_theta"], inst["params"]["n_rstar"])), 0,
                        instance=k)
            s.set_source(inst["r0"], instance=k)
        s.step(3)
        s.sync()
        assert np.abs(s.get_state(1)).max() > 0


def test_ring_wait_times_out_and_context_recovers():
    # a column that is never copied into the step kernel's ring: the blocks waiting for
    # it give up after about a second and the status says so; nothing faults or hangs
    inst = INST[0]
    with TeukSolver(dict(inst["params"], prec="fp32_kahan")) as s:
        s.set_source(inst["r0"])
        s.step(2)
        s.sync()
        s.set_fill_fault(column=7)
        s.step(3)
        with pytest.raises(TeukError) as e:
            s.sync()
        assert e.value.status == 5  # TEUK_ETIMEOUT
        # cleared and reset, the context steps normally again (equal to a fresh run)
        s.set_fill_fault(-1)
        u0 = inputs.random_state(inst["params"]["n_theta"], inst["params"]["n_rstar"], seed=4)
        s.set_state(u0, 0)
        s.step(3)
        s.sync()
        u = s.get_state()
    with TeukSolver(dict(inst["params"], prec="fp32_kahan")) as s2:
        s2.set_source(inst["r0"])
        s2.set_state(u0, 0)
        s2.step(3)
        assert np.array_equal(s2.get_state(), u)


def test_autotune_keeps_results_and_state(tmp_path):
    with TeukSolver([dict(i["params"], prec="fp32_kahan") for i in INST]) as s:
        for k, inst in enumerate(INST):
            s.set_source(inst["r0"], instance=k)
        s.step(4)
        before = [s.get_state(k) for k in range(len(INST))]
        wb = [s.extract(instance=k)[0] for k in range(len(INST))]
        chosen = s.autotune(trial_steps=3, cache_path=str(tmp_path / "tune.json"))
        # valid strips (grids this small may take one-column strips)
        assert len(chosen) == len(INST)
        assert all(1 <= c <= i["params"]["n_rstar"] - 2 for c, i in zip(chosen, INST))
        for k in range(len(INST)):
            assert np.array_equal(s.get_state(k), before[k])
            assert np.array_equal(s.extract(instance=k)[0], wb[k])
        # a second solver reads the cached table without timing
        with TeukSolver([dict(i["params"], prec="fp32_kahan") for i in INST]) as s2:
            assert s2.autotune(cache_path=str(tmp_path / "tune.json")) == chosen
        # time levels and buffers were restored: two more steps equal an untuned run
        s.step(2)
        with TeukSolver([dict(i["params"], prec="fp32_kahan") for i in INST]) as s3:
            for k, inst in enumerate(INST):
                s3.set_source(inst["r0"], instance=k)
            s3.step(6)
            for k in range(len(INST)):
                assert np.array_equal(s3.get_state(k), s.get_state(k))


def test_autotune_single_instance_keeps_results_and_state(tmp_path):
    # one instance stepped per launch: candidates are timed on a scratch copy
    inst = INST[3]
    with TeukSolver(dict(inst["params"], prec="fp32_kahan")) as s:
        s.set_source(inst["r0"])
        s.step(4)
        before = s.get_state()
        wb = s.extract()[0]
        chosen = s.autotune(trial_steps=3, cache_path=str(tmp_path / "tune.json"))
        assert len(chosen) == 1 and 1 <= chosen[0] <= inst["params"]["n_rstar"] - 2
        assert np.array_equal(s.get_state(), before)
        assert np.array_equal(s.extract()[0], wb)
        s.step(3)
        u = s.get_state()
    with TeukSolver(dict(inst["params"], prec="fp32_kahan")) as s2:
        s2.set_source(inst["r0"])
        s2.step(7)
        assert np.array_equal(s2.get_state(), u)


def test_batched_uneven_workload_128_instances(orc):
    # the full 128-instance workload (8 modes x 16 orbits, uneven grids), a few steps in
    # FP32-Kahan; three instances are re-run alone (bitwise) and against the oracle
    insts = inputs.batched_uneven()
    assert len(insts) == 128
    with TeukSolver([dict(i["params"], prec="fp32_kahan") for i in insts]) as s:
        for k, inst in enumerate(insts):
            s.set_source(inst["r0"], instance=k)
        s.step(3)
        s.sync()
        picks = [0, 77, 127]
        got = {k: s.get_state(k) for k in picks}
        wav = {k: s.extract(instance=k)[0] for k in picks}
    for k in picks:
        inst = insts[k]
        with TeukSolver(dict(inst["params"], prec="fp32_kahan")) as s1:
            s1.set_source(inst["r0"])
            s1.step(3)
            assert np.array_equal(s1.get_state(), got[k])
        p = orc.params(**inst["params"], r0=inst["r0"])
        uo, wo = orc.run(p, None, 3, orc.orbit_source(p))
        assert rel(got[k], uo) <= 1e-6


@pytest.mark.parametrize("prec", ["fp64", "fp32_kahan"])
def test_batched_block_size_classes_up_to_1024_rows(prec):
    # one context with columns of 8, 300, 600 and 1024 rows: the persistent kernels built
    # for blocks of up to 256, 512 and 1024 rows in one replayed graph, each instance
    # bitwise equal to its own run
    tall = [dict(params=dict(s=-2, m=m, a=0.6, rstar_min=-10.0, rstar_max=20.0, n_rstar=nr, n_theta=nth,
                             rstar_ext=15.0, dt_rule=1, courant=0.5), r0=6.0, step0=k)
            for k, (m, nr, nth) in enumerate(((2, 90, 8), (1, 40, 300), (3, 30, 600), (2, 24, 1024)))]
    steps = [9, 4]
    with TeukSolver([dict(i["params"], prec=prec) for i in tall]) as s:
        for k, inst in enumerate(tall):
            s.set_source(inst["r0"], inputs.amplitudes(100, seed=k + 1), instance=k)
            u0 = inputs.random_state(inst["params"]["n_theta"], inst["params"]["n_rstar"], seed=5 + k)
            s.set_state(u0, inst["step0"], instance=k)
        for n in steps:
            s.step(n)
        got = [(s.get_state(k), s.extract(instance=k)) for k in range(len(tall))]
        s.sync()
    for k, inst in enumerate(tall):
        with TeukSolver(dict(inst["params"], prec=prec)) as s:
            s.set_source(inst["r0"], inputs.amplitudes(100, seed=k + 1))
            u0 = inputs.random_state(inst["params"]["n_theta"], inst["params"]["n_rstar"], seed=5 + k)
            s.set_state(u0, inst["step0"])
            for n in steps:
                s.step(n)
            u = s.get_state()
            w, first = s.extract()
            s.sync()
        assert got[k][1][1] == first
        assert np.array_equal(got[k][0], u), k
        assert np.array_equal(got[k][1][0], w), k
