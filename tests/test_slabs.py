"""The r* slab decomposition on CPU ranks (gloo): the partition covers the interior
columns once, and the oracle stepped slab by slab -- each rank advancing only its own
columns plus one halo column per side, the halos exchanged point to point after every
step -- reproduces the unsplit oracle bit for bit (the stencil of Eqs. 13-14 reaches one
column in r*).  No GPU is used."""
import os
import socket

import numpy as np
import pytest
import torch.multiprocessing as mp

from paper_1001_3631_gb300 import inputs, slabs

PARAMS = dict(s=-2, m=3, a=0.7, rstar_min=-10.0, rstar_max=30.0, n_rstar=61, n_theta=8,
              rstar_ext=14.0, dt_rule=1, courant=0.5)
STEPS = 40


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def test_partition_covers_the_interior_columns_once():
    for nr, n in ((61, 2), (61, 3), (800, 7), (16384, 8), (9, 3)):
        parts = slabs.partition(nr, n)
        cols = [c for c0, k in parts for c in range(c0, c0 + k)]
        assert cols == list(range(1, nr - 1))
        sizes = [k for _, k in parts]
        assert max(sizes) - min(sizes) <= 1 and min(sizes) >= 2
    with pytest.raises(ValueError):
        slabs.partition(7, 3)


def _worker(rank, world, port, out):
    import torch
    import torch.distributed as dist

    from oracle import teuk_oracle as orc
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    p = orc.params(**PARAMS, r0=8.0)
    src = orc.orbit_source(p)
    nr, nth = PARAMS["n_rstar"], PARAMS["n_theta"]
    u0 = inputs.smooth_state(nth, nr, seed=17)
    c0, n = slabs.partition(nr, world)[rank]
    lo, hi = c0 - 1, c0 + n            # the columns this rank holds: owned plus halos
    keep = np.zeros(nr, bool)
    keep[lo:hi + 1] = True
    u = np.where(keep[None, None, :], u0, 0.0)
    for k in range(STEPS):
        # the oracle advances the whole array; only the held columns carry data, and the
        # owned ones depend on nothing else
        u, _ = orc.run(p, u, 1, src, step0=k, wave=False)
        u = np.where(keep[None, None, :], u, 0.0)
        sl = torch.from_numpy(np.ascontiguousarray(u[:, :, c0]))
        sr = torch.from_numpy(np.ascontiguousarray(u[:, :, c0 + n - 1]))
        rl, rr = torch.empty_like(sl), torch.empty_like(sr)
        slabs.exchange(sl, sr, rl, rr, rank, world)
        if rank > 0:
            u[:, :, lo] = rl.numpy()
        if rank < world - 1:
            u[:, :, hi] = rr.numpy()
    owned = np.ascontiguousarray(u[:, :, c0:c0 + n])
    gathered = [None] * world if rank == 0 else None
    dist.gather_object(owned, gathered, dst=0)
    if rank == 0:
        full, _ = orc.run(p, u0, STEPS, src, wave=False)
        joined = np.concatenate(gathered, axis=2)
        out["equal"] = bool(np.array_equal(joined, full[:, :, 1:nr - 1]))
        out["ends_zero"] = bool(not full[:, :, 0].any() and not full[:, :, -1].any())
        out["max_abs"] = float(np.abs(full).max())
    dist.destroy_process_group()


@pytest.mark.timeout(240)
@pytest.mark.parametrize("world", [2, 3])
def test_oracle_slabs_on_gloo_ranks_equal_the_unsplit_run(world):
    ctx = mp.get_context("spawn")
    manager = ctx.Manager()
    out = manager.dict()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, world, port, out)) for r in range(world)]
    for q in procs:
        q.start()
    for q in procs:
        q.join(200)
        assert q.exitcode == 0
    assert out["max_abs"] > 0
    assert out["ends_zero"]
    assert out["equal"]
