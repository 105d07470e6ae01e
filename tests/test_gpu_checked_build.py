"""The checked build (libteuk_check.so, TEUK_CHECK: every global-memory index of the time
loop's kernels tested against its buffer, failures reported as TEUK_EBOUNDS instead of a
trap).  Tiny grids (N_r* 8..20, N_theta 4..8) in every precision and launch form are
compared element by element with the oracle and must raise no check; the self-test
submits an out-of-range index to the check without addressing memory and must come back
as TEUK_EBOUNDS.  Each case runs in a child process that loads the checked library."""
import json
import os
import subprocess
import sys

import pytest

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

CHILD = r'''
import json, sys
import numpy as np
sys.path.insert(0, ROOT)
from paper_1001_3631_gb300 import TeukError, TeukSolver, _lib, inputs
from oracle import teuk_oracle as orc
assert _lib.load().teuk_checked_build() == 1
out = {}
grids = [dict(s=-2, m=2, a=0.9, rstar_min=-10.0, rstar_max=20.0, n_rstar=8, n_theta=4, rstar_ext=8.0),
         dict(s=-2, m=3, a=0.5, rstar_min=-10.0, rstar_max=20.0, n_rstar=13, n_theta=5, rstar_ext=-10.0),
         dict(s=-1, m=1, a=0.3, rstar_min=-10.0, rstar_max=20.0, n_rstar=20, n_theta=8, rstar_ext=20.0)]
for gi, g in enumerate(grids):
    g = dict(g, dt_rule=1, courant=0.5)
    nth, nr = g["n_theta"], g["n_rstar"]
    u0 = inputs.random_state(nth, nr, seed=40 + gi)
    p = orc.params(**g, r0=4.0 + 0.5 * gi)
    uo, wo = orc.run(p, u0, 7, orc.orbit_source(p))
    for prec in ("fp64", "fp64_df", "fp32_kahan", "fp32"):
        for mode in ("per_step", "resident", "batched"):
            try:
                if mode == "batched":
                    s = TeukSolver([dict(g, prec=prec), dict(g, prec=prec)])
                else:
                    s = TeukSolver(dict(g, prec=prec))
                if mode == "resident":
                    try:
                        s.set_resident(1)
                    except TeukError:
                        s.close()
                        continue
                s.set_source(p.r0)
                s.set_state(u0, 0)
                s.step(3)
                s.step(4)
                u = s.get_state()
                w, _ = s.extract()
                s.sync()
                e = float(np.linalg.norm(u - uo) / np.linalg.norm(uo))
                ew = float(np.linalg.norm(w - wo) / max(np.linalg.norm(wo), 1e-300))
                out["%d/%s/%s" % (gi, prec, mode)] = [e, ew]
                s.close()
            except TeukError as ex:
                out["%d/%s/%s" % (gi, prec, mode)] = ["error", ex.status]
    # the adjoint and a moving particle on the same grid (FP64 and FP32-Kahan)
    for prec in ("fp64", "fp32_kahan"):
        with TeukSolver(dict(g, prec=prec, wave_capacity=9)) as s:
            s.set_source(p.r0, inputs.amplitudes(8, seed=3))
            try:
                s.adjoint(8, step0=0, grad_wave=np.ones((8, nth, 2)))
                s.sync()
                out["%d/%s/adjoint" % (gi, prec)] = "ok"
            except TeukError as ex:
                out["%d/%s/adjoint" % (gi, prec)] = ["error", ex.status]
s = TeukSolver(dict(grids[0], dt_rule=1, courant=0.5, prec="fp64"))
s.check_selftest()
try:
    s.sync()
    out["selftest"] = "no error"
except TeukError as ex:
    out["selftest"] = ex.status
s.close()
print("RESULT " + json.dumps(out))
'''


def test_checked_build_runs_clean_and_reports_a_failed_check():
    env = dict(os.environ, TEUK_LIB_VARIANT="check")
    r = subprocess.run([sys.executable, "-c", "ROOT = %r\n" % ROOT + CHILD], env=env, cwd=ROOT,
                       capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr[-3000:]
    line = [x for x in r.stdout.splitlines() if x.startswith("RESULT ")][-1]
    out = json.loads(line[len("RESULT "):])
    assert out.pop("selftest") == 7   # TEUK_EBOUNDS
    ran = 0
    for key, v in out.items():
        assert v != "error" and not (isinstance(v, list) and v[0] == "error"), (key, v)
        if isinstance(v, list):
            tol = 1e-12 if ("fp64" in key) else (1e-6 if "kahan" in key else 2e-5)
            assert v[0] <= tol and v[1] <= tol, (key, v)
            ran += 1
    assert ran >= 3 * 4 * 2   # every grid and precision in at least two launch forms
