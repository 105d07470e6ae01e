"""Writes paper_scale_16384x256_probe.npz: the oracle's run of the paper-scale single mode
(s = -2, m = 2, a = 0.9, N_r* = 16384 over r* in [-200, 800], N_theta = 256, circular
orbit at r0 = 8, zero initial data, dt rule 1 at Courant factor 0.5) for 4000 steps: the
waveform at the near-zone probe r* = 12 every 100 steps, and the final state at every
512th r* column (the stated extraction radius r* = 700 is not reached in 4000 steps).

Calls only the oracle (oracle/teuk_oracle.c); about 20 minutes on one core.  Read by the
benchmark's accuracy leg, which states the error of every GPU path against it."""
import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

from oracle import teuk_oracle as orc  # noqa: E402

PARAMS = dict(s=-2, m=2, M=1.0, a=0.9, rstar_min=-200.0, rstar_max=800.0, n_rstar=16384,
              n_theta=256, courant=0.5, dt_rule=1, r0=8.0)
STEPS, EVERY, PROBE, COL_EVERY = 4000, 100, 12.0, 512


def main(out=os.path.join(HERE, "paper_scale_16384x256_probe.npz")):
    t0 = time.time()
    p = orc.params(**PARAMS, rstar_ext=PROBE)
    src = orc.orbit_source(p)
    g = orc.grid(p)
    ie, fe = g["i_e"], g["f_e"]
    u = np.zeros((4, p.n_theta, p.n_rstar))
    rec = np.zeros((STEPS // EVERY + 1, p.n_theta, 2))
    for k in range(1, STEPS // EVERY + 1):
        u, _ = orc.run(p, u, EVERY, src, step0=(k - 1) * EVERY, wave=False)
        rec[k] = ((1.0 - fe) * u[0:2, :, ie] + fe * u[0:2, :, ie + 1]).T
        print("step %d  %.0f s" % (k * EVERY, time.time() - t0), flush=True)
    cols = np.arange(0, p.n_rstar, COL_EVERY)
    np.savez_compressed(out, steps=np.arange(0, STEPS + 1, EVERY), dt=g["dt"], probe12=rec,
                        final_cols=cols, final_state=u[:, :, cols], params=repr(PARAMS))


if __name__ == "__main__":
    main()
