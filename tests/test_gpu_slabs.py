"""Slab instances (teuk_params.slab_col0 / slab_ncols) on the GPU: the grid split into
r* slabs that are stepped one step at a time with their halo columns exchanged
(teuk_slab_export / teuk_slab_import) reproduce the unsplit run bit for bit -- states,
and the waveform records of the slab that holds the extraction radius.  Three slabs in
one process on one GPU (device-to-device halo copies), and two processes on the same GPU
exchanging through gloo (the multi-rank driver, its kernels never waiting on each
other)."""
import os
import socket

import numpy as np
import pytest
import torch.multiprocessing as mp

from paper_1001_3631_gb300 import TeukError, TeukSolver, inputs, slabs

pytestmark = pytest.mark.gpu

GRIDS = [
    dict(s=-2, m=2, a=0.9, rstar_min=-50.0, rstar_max=150.0, n_rstar=800, n_theta=64,
         rstar_ext=14.2, dt_rule=1, courant=0.5),
    dict(s=-2, m=3, a=0.7, rstar_min=-10.0, rstar_max=30.0, n_rstar=97, n_theta=33,
         rstar_ext=4.3, dt_rule=1, courant=0.5),
]
STEPS = 30


def set_src(s, moving):
    if moving:   # an eccentric, inclined path (per-step source tables in local columns)
        traj = inputs.eccentric_trajectory(2 * STEPS + 2, s.time()[1], semi_latus=7.0, ecc=0.5, incl=0.5)
        s.set_trajectory(traj)
    else:
        s.set_source(8.0, inputs.amplitudes(STEPS, seed=4))


def unsplit(params, prec, u0, moving=False):
    with TeukSolver(dict(params, prec=prec, wave_capacity=STEPS + 1)) as s:
        set_src(s, moving)
        s.set_state(u0, 0)
        s.step(STEPS)
        u = s.get_state()
        w, first = s.extract(cap=STEPS + 1)
        s.sync()
    return u, w


@pytest.mark.parametrize("prec,g,moving", [(p, g, False) for p in ("fp64", "fp32_kahan", "fp64_df")
                                           for g in range(len(GRIDS))] +
                         [("fp64", 0, True), ("fp32_kahan", 0, True)])
def test_three_slabs_on_one_gpu_equal_the_unsplit_run(prec, g, moving):
    import torch
    params = GRIDS[g]
    nr, nth = params["n_rstar"], params["n_theta"]
    u0 = inputs.smooth_state(nth, nr, seed=23)
    ref_u, ref_w = unsplit(params, prec, u0, moving)
    parts = slabs.partition(nr, 3)
    sv = []
    for c0, n in parts:
        s = TeukSolver(dict(params, prec=prec, wave_capacity=STEPS + 1, slab_col0=c0, slab_ncols=n))
        set_src(s, moving)
        s.set_state(np.ascontiguousarray(u0[:, :, c0 - 1:c0 + n + 1]), 0)
        sv.append(s)
    nb = sv[0].halo_bytes()
    buf = [[torch.empty(nb, dtype=torch.uint8, device="cuda") for _ in range(2)] for _ in sv]
    for _ in range(STEPS):
        for s in sv:
            s.step(1)
        for k, s in enumerate(sv):          # each slab's end columns out ...
            s.slab_export(0, buf[k][0].data_ptr())
            s.slab_export(1, buf[k][1].data_ptr())
        for k, s in enumerate(sv):          # ... into the neighbours' halos
            if k > 0:
                s.slab_import(0, buf[k - 1][1].data_ptr())
            if k < len(sv) - 1:
                s.slab_import(1, buf[k + 1][0].data_ptr())
    owners = 0
    for (c0, n), s in zip(parts, sv):
        u = s.get_state()
        assert np.array_equal(u[:, :, 1:1 + n], ref_u[:, :, c0:c0 + n])
        try:
            w, first = s.extract(cap=STEPS + 1)
        except TeukError:
            continue                        # the extraction radius lies in another slab
        owners += 1
        assert first == 0 and np.array_equal(w, ref_w)
        s.sync()
    assert owners == 1
    for s in sv:
        s.close()


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _rank(rank, world, port, out):
    import torch
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    torch.cuda.set_device(0)
    params = dict(GRIDS[0], prec="fp32_kahan", wave_capacity=STEPS + 1)
    u0 = inputs.smooth_state(64, 800, seed=29)
    st = slabs.SlabStepper(params, rank, world, host_exchange=True)
    st.solver.set_source(8.0)
    st.solver.set_state(np.ascontiguousarray(u0[:, :, st.col0 - 1:st.col0 + st.ncols + 1]), 0)
    st.step(STEPS)
    owned = np.ascontiguousarray(st.owned(st.solver.get_state()))
    st.solver.sync()
    st.solver.close()
    gathered = [None] * world if rank == 0 else None
    dist.gather_object(owned, gathered, dst=0)
    if rank == 0:
        with TeukSolver(params) as s:
            s.set_source(8.0)
            s.set_state(u0, 0)
            s.step(STEPS)
            full = s.get_state()
        out["equal"] = bool(np.array_equal(np.concatenate(gathered, axis=2), full[:, :, 1:799]))
    dist.destroy_process_group()


@pytest.mark.timeout(300)
def test_two_rank_slab_driver_over_gloo_equals_the_unsplit_run():
    ctx = mp.get_context("spawn")
    out = ctx.Manager().dict()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, out)) for r in range(2)]
    for q in procs:
        q.start()
    for q in procs:
        q.join(280)
        assert q.exitcode == 0
    assert out["equal"]


def test_slab_argument_errors():
    params = GRIDS[1]
    for col0, n in ((0, 10), (90, 10), (5, 1)):
        with pytest.raises(TeukError):
            TeukSolver(dict(params, slab_col0=col0, slab_ncols=n))
    with TeukSolver(dict(params)) as s:   # not a slab
        with pytest.raises(TeukError):
            s.slab_export(0, 0)
    with TeukSolver(dict(params, slab_col0=10, slab_ncols=20)) as s:
        with pytest.raises(TeukError):
            s.set_resident(1)
        with pytest.raises(TeukError):
            s.adjoint(5, grad_wave=np.zeros((5, 33, 2)))
