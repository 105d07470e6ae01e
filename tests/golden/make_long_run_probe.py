"""Writes long_run_8192x128_probe.npz: the oracle's waveform records of the long-run
workload (s = -2, m = 2, a = 0.99, N_r* = 8192 over r* in [-200, 800], N_theta = 128,
circular orbit at r0 = 8, zero initial data, dt rule 1 at Courant factor 0.5) at every
1000th step of 100 000, at the near-zone probe r* = 30 and at the stated extraction
radius r* = 400.

Calls only the oracle (oracle/teuk_oracle.c); about 45 minutes on one core.  The file is
read by the benchmark's precision sweep and by a GPU test, which compare the GPU paths
with these records."""
import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

from oracle import teuk_oracle as orc  # noqa: E402

PARAMS = dict(s=-2, m=2, M=1.0, a=0.99, rstar_min=-200.0, rstar_max=800.0, n_rstar=8192,
              n_theta=128, courant=0.5, dt_rule=1, r0=8.0)
STEPS, EVERY = 100000, 1000
PROBES = (30.0, 400.0)


def main(out=os.path.join(HERE, "long_run_8192x128_probe.npz")):
    t0 = time.time()
    p = orc.params(**PARAMS, rstar_ext=PROBES[0])
    src = orc.orbit_source(p)
    g = orc.grid(p)
    u = np.zeros((4, p.n_theta, p.n_rstar))
    rec = {r: np.zeros((STEPS // EVERY + 1, p.n_theta, 2)) for r in PROBES}
    # the extraction of each probe radius: linear between the bracketing nodes
    ext = []
    for r in PROBES:
        pr = orc.params(**PARAMS, rstar_ext=r)
        gr = orc.grid(pr)
        ext.append((r, gr["i_e"], gr["f_e"]))

    def record(k):
        for r, ie, fe in ext:
            rec[r][k] = ((1.0 - fe) * u[0:2, :, ie] + fe * u[0:2, :, ie + 1]).T

    record(0)
    for k in range(1, STEPS // EVERY + 1):
        u, _ = orc.run(p, u, EVERY, src, step0=(k - 1) * EVERY, wave=False)
        record(k)
        print("step %d  %.0f s" % (k * EVERY, time.time() - t0), flush=True)
    np.savez_compressed(out, steps=np.arange(0, STEPS + 1, EVERY), dt=g["dt"],
                        probe30=rec[30.0], probe400=rec[400.0], params=repr(PARAMS))


if __name__ == "__main__":
    main()
