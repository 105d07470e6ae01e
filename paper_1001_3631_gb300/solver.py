"""TeukSolver: a thin Python handle over the C ABI (include/teuk.h).

It marshals numpy arrays and torch streams into the C calls; the time loop, the
source and the extraction all run in the library's CUDA kernels."""
from __future__ import annotations

import ctypes
import json
import os

import numpy as np

from . import _lib
from ._lib import TEUK_FP32, TEUK_FP32_KAHAN, TEUK_FP64, TEUK_FP64_DF, check, ptr

PREC = {"fp64": TEUK_FP64, "fp32": TEUK_FP32, "fp32_kahan": TEUK_FP32_KAHAN, "fp64_df": TEUK_FP64_DF,
        TEUK_FP64: TEUK_FP64, TEUK_FP32: TEUK_FP32, TEUK_FP32_KAHAN: TEUK_FP32_KAHAN,
        TEUK_FP64_DF: TEUK_FP64_DF}

PARAM_DEFAULTS = dict(s=-2, m=2, M=1.0, a=0.9, rstar_min=-50.0, rstar_max=150.0, n_rstar=800,
                      n_theta=64, courant=0.5, dt_rule=1, dt=0.0, rstar_ext=140.0,
                      prec="fp64", wave_capacity=0, slab_col0=0, slab_ncols=0)


def make_params(**kw) -> _lib.teuk_params:
    d = dict(PARAM_DEFAULTS)
    for k, v in kw.items():
        if k not in d:
            raise KeyError("unknown parameter %r" % k)
        d[k] = v
    d["prec"] = PREC[d["prec"]]
    return _lib.teuk_params(**d)


_ALLOC_HOOKS = None   # the ctypes callbacks in force (kept alive while installed)


def set_allocator(alloc=None, free=None):
    """Route the device memory of contexts created from now on through Python callables
    alloc(bytes, stream_handle) -> device pointer (0 on failure) and free(ptr, stream_handle)
    (teuk_set_allocator); set_allocator() restores cudaMallocAsync.  Contexts keep the
    allocator they were created with."""
    global _ALLOC_HOOKS
    lib = _lib.load()
    if alloc is None and free is None:
        check(lib.teuk_set_allocator(None, None, None), None)
        _ALLOC_HOOKS = None
        return

    def _a(nbytes, stream, user):
        try:
            return int(alloc(int(nbytes), int(stream or 0))) or None
        except Exception:
            return None

    def _f(ptr, stream, user):
        try:
            free(int(ptr), int(stream or 0))
        except Exception:
            pass

    hooks = (_lib.ALLOC_FN(_a), _lib.FREE_FN(_f), alloc, free)
    check(lib.teuk_set_allocator(ctypes.cast(hooks[0], ctypes.c_void_p),
                                 ctypes.cast(hooks[1], ctypes.c_void_p), None), None)
    _ALLOC_HOOKS = hooks


def use_torch_allocator(enable=True):
    """Device memory of new contexts from torch's caching allocator (one pool with torch)."""
    if not enable:
        set_allocator()
        return
    import torch

    set_allocator(lambda n, st: torch.cuda.caching_allocator_alloc(n, stream=st),
                  lambda p, st: torch.cuda.caching_allocator_delete(p))


def _stream_handle(stream):
    if stream is None:
        import torch
        return torch.cuda.current_stream().cuda_stream
    if isinstance(stream, int):
        return stream
    return stream.cuda_stream


class TeukSolver:
    """One context of one or more instances (see teuk_create)."""

    def __init__(self, params, stream=None):
        if isinstance(params, dict):
            params = [params]
        plist = [p if isinstance(p, _lib.teuk_params) else make_params(**p) for p in params]
        self.n = len(plist)
        arr = (_lib.teuk_params * self.n)(*plist)
        self.params = plist
        self._stream = stream
        h = ctypes.c_void_p()
        lib = _lib.load()
        st = lib.teuk_create(arr, self.n, ctypes.c_void_p(_stream_handle(stream)), ctypes.byref(h))
        check(st, None)
        self.ctx = h
        self._steps_per_launch = 1

    # -- lifetime
    def close(self):
        if getattr(self, "ctx", None):
            _lib.load().teuk_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    # -- calls
    def set_source(self, r0, amps=None, instance=0, sigma_rstar_cells=4.0, sigma_theta_cells=4.0,
                   sigma_rstar_abs=0.0, sigma_theta_abs=0.0):
        orb = _lib.teuk_orbit(r0, sigma_rstar_cells, sigma_theta_cells, sigma_rstar_abs,
                              sigma_theta_abs)
        a = None if amps is None else np.ascontiguousarray(amps, dtype=np.float64)
        check(_lib.load().teuk_set_source(self.ctx, instance, ctypes.byref(orb), ptr(a),
                                          0 if a is None else a.size), self.ctx)

    def set_trajectory(self, traj, instance=0, sigma_rstar_cells=4.0, sigma_theta_cells=4.0,
                       sigma_rstar_abs=0.0, sigma_theta_abs=0.0):
        """Moving particle: traj [n_samples][4] = {r_p, theta_p, phi_p, A} at t = k dt/2
        (step n takes samples 2n and 2n + 1)."""
        orb = _lib.teuk_orbit(0.0, sigma_rstar_cells, sigma_theta_cells, sigma_rstar_abs,
                              sigma_theta_abs)
        t = np.ascontiguousarray(traj, dtype=np.float64).reshape(-1, 4)
        check(_lib.load().teuk_set_trajectory(self.ctx, instance, ctypes.byref(orb), ptr(t),
                                              t.shape[0]), self.ctx)

    def shape(self, instance=0):
        p = self.params[instance]
        return (4, p.n_theta, p.slab_ncols + 2 if p.slab_ncols > 0 else p.n_rstar)

    # -- slabs (teuk_params.slab_ncols > 0): halo columns, device to device
    def halo_bytes(self, instance=0):
        b = ctypes.c_int64(0)
        check(_lib.load().teuk_slab_halo_bytes(self.ctx, instance, ctypes.byref(b)), self.ctx)
        return b.value

    def slab_export(self, side, dev_ptr, instance=0):
        check(_lib.load().teuk_slab_export(self.ctx, instance, side, ctypes.c_void_p(dev_ptr)), self.ctx)

    def slab_import(self, side, dev_ptr, instance=0):
        check(_lib.load().teuk_slab_import(self.ctx, instance, side, ctypes.c_void_p(dev_ptr)), self.ctx)

    def set_state(self, u, step0=0, instance=0):
        u = np.ascontiguousarray(u, dtype=np.float64)
        assert u.shape == self.shape(instance)
        check(_lib.load().teuk_set_state(self.ctx, instance, ptr(u), step0), self.ctx)

    def get_state(self, instance=0):
        u = np.empty(self.shape(instance))
        check(_lib.load().teuk_get_state(self.ctx, instance, ptr(u)), self.ctx)
        return u

    def step(self, n):
        check(_lib.load().teuk_step_n(self.ctx, int(n)), self.ctx)

    def extract(self, cap=None, instance=0, scalar=False):
        """Returns (records [k][n_theta][2], first_step[, scalar [k][2]])."""
        p = self.params[instance]
        step, _ = self.time(instance)
        if cap is None:
            cap = step + 1
        out = np.empty((cap, p.n_theta, 2))
        sc = np.empty((cap, 2)) if scalar else None
        nw, first = ctypes.c_int64(0), ctypes.c_int64(0)
        check(_lib.load().teuk_extract(self.ctx, instance, ptr(out), ptr(sc), cap,
                                       ctypes.byref(nw), ctypes.byref(first)), self.ctx)
        k = nw.value
        if scalar:
            return out[:k], first.value, sc[:k]
        return out[:k], first.value

    def mode_sum(self, phi, first, n_records):
        """Psi = sum_m e^{i m phi~} r^3 Phi_m at the extraction radius over the instances
        (modes of one problem) for time levels first .. first + n_records - 1 and the
        azimuths phi: complex array [n_records][n_theta][len(phi)]."""
        ph = np.ascontiguousarray(np.atleast_1d(phi), dtype=np.float64)
        nth = self.params[0].n_theta
        out = np.empty((n_records, nth, ph.size, 2))
        check(_lib.load().teuk_mode_sum(self.ctx, ptr(ph), ph.size, int(first), int(n_records),
                                        ptr(out)), self.ctx)
        return out[..., 0] + 1j * out[..., 1]

    def radiated_flux(self, first, n_records):
        """Energy, linear momentum and Jz carried off by the field of the instances (distinct
        modes of one problem), from the records first .. first + n_records - 1: array
        [n_records][10] = dE/dt, dPx/dt, dPy/dt, dPz/dt, dJz/dt, E, Px, Py, Pz, Jz (totals
        from `first`; the recoil velocity is -P / M_total)."""
        out = np.empty((int(n_records), 10))
        check(_lib.load().teuk_radiated_flux(self.ctx, int(first), int(n_records), ptr(out)),
              self.ctx)
        return out

    def adjoint(self, n, step0=0, grad_wave=None, ckpt_every=100, instance=0):
        """Returns (grad_amps [n], grad_r0, loss).  ckpt_every (built-in loss only): K > 0
        recomputes each K-step segment's records from a state checkpoint in the reverse
        sweep; 0 keeps every record's cotangent instead (no recomputation)."""
        gw = None if grad_wave is None else np.ascontiguousarray(grad_wave, dtype=np.float64)
        ga = np.zeros(n)
        gr, loss = ctypes.c_double(0.0), ctypes.c_double(0.0)
        check(_lib.load().teuk_adjoint_n(self.ctx, instance, step0, n, ckpt_every, ptr(gw),
                                         ptr(ga), ctypes.byref(gr), ctypes.byref(loss)), self.ctx)
        return ga, gr.value, loss.value

    def sync(self):
        check(_lib.load().teuk_sync(self.ctx), self.ctx)

    def save_state(self, path, instance=0):
        """Checkpoint: parameters, time level and the current level's planes, bit for bit."""
        check(_lib.load().teuk_save_state(self.ctx, instance, os.fsencode(path)), self.ctx)

    def load_state(self, path, instance=0):
        """Resume from save_state's file (the same problem; clears the waveform records)."""
        check(_lib.load().teuk_load_state(self.ctx, instance, os.fsencode(path)), self.ctx)

    def check_selftest(self):
        """Checked builds: make the next sync report TEUK_EBOUNDS (no memory is addressed)."""
        check(_lib.load().teuk_check_selftest(self.ctx), self.ctx)

    def time(self, instance=0):
        s, dt = ctypes.c_int64(0), ctypes.c_double(0.0)
        check(_lib.load().teuk_get_time(self.ctx, instance, ctypes.byref(s), ctypes.byref(dt)),
              self.ctx)
        return s.value, dt.value

    def geometry(self, instance=0):
        """dict(drs, dth, dt, rp, rm, r_ext, i_e, f_e) of one instance."""
        out = np.zeros(8)
        check(_lib.load().teuk_get_geometry(self.ctx, instance, ptr(out)), self.ctx)
        return dict(drs=out[0], dth=out[1], dt=out[2], rp=out[3], rm=out[4], r_ext=out[5],
                    i_e=int(out[6]), f_e=out[7])

    def set_tiling(self, strip=0, steps_per_launch=1):
        """strip: r* columns per thread block (0 = automatic); steps_per_launch 0 sends a
        single-instance context through the persistent batched kernel."""
        check(_lib.load().teuk_set_tiling(self.ctx, strip, steps_per_launch), self.ctx)
        self._steps_per_launch = steps_per_launch

    def set_resident(self, halo=1, blocks_per_sm=1):
        """Resident launches (one cooperative launch per step() call, the grid held in
        shared memory, boundary columns exchanged every ``halo`` steps, the column runs cut
        for ``blocks_per_sm`` blocks per SM); halo 0 turns them off."""
        check(_lib.load().teuk_set_resident_shape(self.ctx, int(halo), int(blocks_per_sm)), self.ctx)

    def set_blocked(self, steps=2, blocks_per_sm=1):
        """Blocked launches (each launch advances ``steps`` steps of the grid held in shared
        memory, halos from the previous launch's output, no exchange); 0 turns them off."""
        check(_lib.load().teuk_set_blocked(self.ctx, int(steps), int(blocks_per_sm)), self.ctx)

    def kernel_launches(self):
        return _lib.load().teuk_kernel_launches(self.ctx)

    def set_instance_tiling(self, instance, strip):
        check(_lib.load().teuk_set_instance_tiling(self.ctx, instance, strip), self.ctx)

    def set_fill_fault(self, column=-1, instance=0):
        check(_lib.load().teuk_set_fill_fault(self.ctx, instance, column), self.ctx)

    def set_fault_injection(self, skip_release_item=-1, spin_limit=0):
        check(_lib.load().teuk_set_fault_injection(self.ctx, skip_release_item, spin_limit),
              self.ctx)

    def autotune(self, trial_steps=10, cache_path=None):
        """Strip length per instance from a cached table keyed by (GPU, launch mode, n_theta,
        precision, n_rstar bucket); entries missing from the table are timed by
        teuk_autotune.  A negative entry -v (single instance stepped per call) selects
        resident launches with halo v % 16 and v // 16 + 1 blocks per SM.  The launch mode is "step" for one instance stepped one launch per
        step, and for contexts that run the persistent kernels a signature of the whole
        set of instances (their best strips depend on one another)."""
        import hashlib

        import torch
        path = cache_path or os.environ.get("TEUK_TUNE_CACHE") or os.path.join(
            os.path.expanduser("~"), ".cache", "teuk_gb300", "tune.json")
        gpu = torch.cuda.get_device_name()
        if self.n == 1 and self._steps_per_launch != 0:
            mode = "step"
        else:
            shapes = sorted((p.n_rstar, p.n_theta, p.prec) for p in self.params)
            mode = "batch:" + hashlib.sha1(repr(shapes).encode()).hexdigest()[:12]
        keys = ["%s|%s|%d|%d|%d" % (gpu, mode, p.n_theta, p.prec, int(np.ceil(np.log2(p.n_rstar))))
                for p in self.params]
        table = {}
        if os.path.exists(path):
            try:
                with open(path) as f:
                    table = json.load(f)
            except (OSError, ValueError):
                table = {}
        if all(k in table for k in keys):
            for i, k in enumerate(keys):
                v = int(table[k])
                if v < 0:   # resident launches: halo (-v) % 16, (-v) // 16 + 1 blocks per SM
                    self.set_resident((-v) % 16, (-v) // 16 + 1)
                else:
                    self.set_instance_tiling(i, v)
                    if self.n == 1 and self._steps_per_launch != 0:
                        self.set_resident(0)
            return [int(table[k]) for k in keys]
        chosen = np.zeros(self.n, dtype=np.int32)
        check(_lib.load().teuk_autotune(self.ctx, trial_steps, chosen.ctypes.data_as(ctypes.c_void_p)),
              self.ctx)
        for k, c in zip(keys, chosen):
            table[k] = int(c)
        try:
            os.makedirs(os.path.dirname(path), exist_ok=True)
            tmp = path + ".tmp%d" % os.getpid()
            with open(tmp, "w") as f:
                json.dump(table, f, indent=1, sort_keys=True)
            os.replace(tmp, path)
        except OSError:
            pass
        return [int(c) for c in chosen]
