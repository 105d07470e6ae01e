"""ctypes wrapper of the plain FP64 C oracle (``teuk_oracle.c``).

TEST INFRASTRUCTURE ONLY: imported by the tests, the smoke check and the
CPU-baseline leg of the benchmark, never by the product path.  It shares no
code with the CUDA library.

Arrays:
  state  u      float64 [4][n_theta][n_rstar]  = {Phi_R, Phi_I, Pi_R, Pi_I}  (Eq. 9)
  wave          float64 [records][n_theta][2]   Phi at r*_ext, (re, im)
  profiles      complex128 [n_theta][n_rstar] (integer nodes), [n_theta][n_rstar-1] (half nodes)
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "teuk_oracle.c")
_LIB = os.path.join(_HERE, "libteuk_oracle.so")


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (-O2, no contraction, no fast-math)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + ".tmp%d" % os.getpid()
        subprocess.check_call(["gcc", "-std=c11", "-O2", "-ffp-contract=off", "-fno-fast-math",
                               "-shared", "-fPIC", "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


class Params(ctypes.Structure):
    """Problem statement (Eq. 1 parameters, grid, Courant rule, orbit, extraction)."""

    _fields_ = [
        ("s", ctypes.c_int), ("m", ctypes.c_int),
        ("M", ctypes.c_double), ("a", ctypes.c_double),
        ("rstar_min", ctypes.c_double), ("rstar_max", ctypes.c_double),
        ("n_rstar", ctypes.c_int), ("n_theta", ctypes.c_int),
        ("courant", ctypes.c_double), ("dt_rule", ctypes.c_int), ("dt", ctypes.c_double),
        ("rstar_ext", ctypes.c_double), ("r0", ctypes.c_double),
        ("sigma_r_cells", ctypes.c_double), ("sigma_th_cells", ctypes.c_double),
        ("sigma_r_abs", ctypes.c_double), ("sigma_th_abs", ctypes.c_double),
    ]


_lib = None


def lib():
    global _lib
    if _lib is None:
        _lib = ctypes.CDLL(build())
        D, I, P = ctypes.c_double, ctypes.c_int, ctypes.c_void_p
        L = ctypes.c_int64
        pp = ctypes.POINTER(Params)
        _lib.orc_rstar_of_x.restype = D
        _lib.orc_rstar_of_x.argtypes = [D, D, D]
        _lib.orc_x_of_rstar.restype = D
        _lib.orc_x_of_rstar.argtypes = [D, D, D]
        _lib.orc_coeffs.restype = None
        _lib.orc_coeffs.argtypes = [pp, D, D, P]
        _lib.orc_grid.restype = I
        _lib.orc_grid.argtypes = [pp, P]
        _lib.orc_orbit.restype = I
        _lib.orc_orbit.argtypes = [pp, P]
        _lib.orc_orbit_profile.restype = I
        _lib.orc_orbit_profile.argtypes = [pp, P, P, P, P]
        _lib.orc_run.restype = I
        _lib.orc_run.argtypes = [pp, D, D, P, P, P, L, L, L, P, P]
        _lib.orc_run_traj.restype = I
        _lib.orc_run_traj.argtypes = [pp, P, L, L, L, P, P]
        _lib.orc_apply_K.restype = I
        _lib.orc_apply_K.argtypes = [pp, P, P]
        _lib.orc_apply_KT.restype = I
        _lib.orc_apply_KT.argtypes = [pp, P, P]
        _lib.orc_theta_apply.restype = I
        _lib.orc_theta_apply.argtypes = [pp, P, P]
        _lib.orc_adjoint.restype = I
        _lib.orc_adjoint.argtypes = [pp, D, D, P, P, P, P, D, D, P, L, L, L, P, P, P, P]
    return _lib


DEFAULTS = dict(s=-2, m=2, M=1.0, a=0.9, rstar_min=-50.0, rstar_max=150.0, n_rstar=800,
                n_theta=64, courant=0.5, dt_rule=1, dt=0.0, rstar_ext=140.0, r0=10.0,
                sigma_r_cells=4.0, sigma_th_cells=4.0, sigma_r_abs=0.0, sigma_th_abs=0.0)


def params(**kw) -> Params:
    d = dict(DEFAULTS)
    for k, v in kw.items():
        if k not in d:
            raise KeyError(k)
        d[k] = v
    return Params(**d)


def _ptr(a):
    return None if a is None else a.ctypes.data_as(ctypes.c_void_p)


def _check(st):
    if st != 0:
        raise ValueError("oracle returned status %d" % st)


def rstar_of_r(M, a, r):
    rp = M + np.sqrt(M * M - a * a)
    return lib().orc_rstar_of_x(M, a, r - rp)


def x_of_rstar(M, a, rstar):
    return lib().orc_x_of_rstar(M, a, rstar)


def coeffs(p: Params, x: float, theta: float) -> dict:
    out = np.zeros(12)
    lib().orc_coeffs(ctypes.byref(p), x, theta, _ptr(out))
    names = ["b", "w", "bbr", "ct_re", "ct_im", "pst_re", "pst_im", "Pst_re", "Pst_im",
             "q_re", "q_im", "V"]
    return dict(zip(names, out))


def grid(p: Params) -> dict:
    out = np.zeros(7)
    _check(lib().orc_grid(ctypes.byref(p), _ptr(out)))
    return dict(drs=out[0], dth=out[1], dt=out[2], rp=out[3], rm=out[4], i_e=int(out[5]),
                f_e=out[6])


def orbit(p: Params) -> dict:
    out = np.zeros(10)
    _check(lib().orc_orbit(ctypes.byref(p), _ptr(out)))
    keys = ["Omega", "phi0", "rstar0", "r_ext", "dOmega_dr0", "dphi0_dr0", "drstar0_dr0",
            "sigma_r", "sigma_th", "x0"]
    return dict(zip(keys, out))


class Source:
    """tau = A_n exp(-i (omega t + phase0)) P with P at integer / half nodes."""

    def __init__(self, omega, phase0, P_int, P_half, dP_int=None, dP_half=None,
                 domega=0.0, dphase0=0.0):
        self.omega, self.phase0 = float(omega), float(phase0)
        self.P_int = np.ascontiguousarray(P_int, dtype=np.complex128)
        self.P_half = np.ascontiguousarray(P_half, dtype=np.complex128)
        nth, nr = self.P_int.shape
        self.dP_int = (np.zeros_like(self.P_int) if dP_int is None
                       else np.ascontiguousarray(dP_int, dtype=np.complex128))
        self.dP_half = (np.zeros_like(self.P_half) if dP_half is None
                        else np.ascontiguousarray(dP_half, dtype=np.complex128))
        self.domega, self.dphase0 = float(domega), float(dphase0)


def orbit_source(p: Params) -> Source:
    """The synthetic circular-orbit source of the problem statement."""
    nth, nr = p.n_theta, p.n_rstar
    P_int = np.zeros((nth, nr), np.complex128)
    P_half = np.zeros((nth, nr - 1), np.complex128)
    dP_int = np.zeros_like(P_int)
    dP_half = np.zeros_like(P_half)
    _check(lib().orc_orbit_profile(ctypes.byref(p), _ptr(P_int), _ptr(P_half), _ptr(dP_int),
                                   _ptr(dP_half)))
    ob = orbit(p)
    m = p.m
    return Source(m * ob["Omega"], m * ob["phi0"], P_int, P_half, dP_int, dP_half,
                  m * ob["dOmega_dr0"], m * ob["dphi0_dr0"])


def run(p: Params, u0=None, nsteps=1, source: Source | None = None, amps=None, step0=0,
        wave=True):
    """Evolve ``nsteps`` steps; returns (u, wave) with wave [nsteps+1][n_theta][2]."""
    nth, nr = p.n_theta, p.n_rstar
    u = np.zeros((4, nth, nr)) if u0 is None else np.array(u0, dtype=np.float64, copy=True)
    assert u.shape == (4, nth, nr)
    w = np.zeros((nsteps + 1, nth, 2)) if wave else None
    a = None if amps is None else np.ascontiguousarray(amps, dtype=np.float64)
    na = 0 if a is None else a.size
    if source is None:
        _check(lib().orc_run(ctypes.byref(p), 0.0, 0.0, None, None, _ptr(a), na, step0, nsteps,
                             _ptr(u), _ptr(w)))
    else:
        _check(lib().orc_run(ctypes.byref(p), source.omega, source.phase0, _ptr(source.P_int),
                             _ptr(source.P_half), _ptr(a), na, step0, nsteps, _ptr(u), _ptr(w)))
    return u, w


def run_trajectory(p: Params, traj, u0=None, nsteps=1, step0=0, wave=True):
    """Evolve with the moving-particle source: traj [n_samples][4] = {r_p, theta_p,
    phi_p, A} at t = k dt/2 (step n takes samples 2n and 2n + 1).  Returns (u, wave)."""
    nth, nr = p.n_theta, p.n_rstar
    u = np.zeros((4, nth, nr)) if u0 is None else np.array(u0, dtype=np.float64, copy=True)
    assert u.shape == (4, nth, nr)
    w = np.zeros((nsteps + 1, nth, 2)) if wave else None
    t = np.ascontiguousarray(traj, dtype=np.float64).reshape(-1, 4)
    _check(lib().orc_run_traj(ctypes.byref(p), _ptr(t), t.shape[0], step0, nsteps, _ptr(u),
                              _ptr(w)))
    return u, w


def mode_sum(ps, waves, phi):
    """The field of Eqs. (3)-(4) at the extraction radius summed over modes:
    out[k][j][l] = r_ext^3 sum_i e^{i m_i phi~_l} W_i[k][j] with
    phi~ = phi + a/(r_+ - r_-) ln((r_ext - r_+)/(r_ext - r_-)) (Eq. 3); ps: the modes'
    parameters (same s, M, a, grid in theta, extraction radius), waves: their records
    [k][n_theta][2].  Complex [k][n_theta][len(phi)]."""
    g = grid(ps[0])
    r_ext = orbit(ps[0])["r_ext"]
    a, rp, rm = ps[0].a, g["rp"], g["rm"]
    shift = a / (rp - rm) * np.log((r_ext - rp) / (r_ext - rm))
    phi = np.atleast_1d(np.asarray(phi, dtype=np.float64))
    out = np.zeros(waves[0].shape[:2] + (phi.size,), np.complex128)
    for p, W in zip(ps, waves):
        Wc = W[..., 0] + 1j * W[..., 1]
        out += np.exp(1j * p.m * (phi + shift))[None, None, :] * Wc[:, :, None]
    return r_ext ** 3 * out


def radiated_flux(ps, waves):
    """Energy, linear momentum and angular momentum about the spin axis carried off by
    the field of several modes, from their waveform records at the extraction radius
    (the recoil of Sec. 2.2: the momentum the waves carry away; the system's kick
    velocity is -P / M_total).  Flux formulas from outside the paper (Teukolsky and
    Press 1974, Kinnersley tetrad; the same integrals in terms of psi_4 as in the
    numerical-relativity literature, with psi_4 of that tetrad):

      Psi = rho^-4 psi_4 for s = -2, rho^-1 = r - i a cos(theta)   (Teukolsky 1973)
      r psi_4 = Phi e^{i m phi~} (r / (r - i a cos theta))^4          (Eq. 4, Psi = e^{i m phi~} r^3 Phi)
      phi~ = phi + a/(r_+ - r_-) ln((r - r_+)/(r - r_-))            (Eq. 3 at the radius)
      N(t) = int_{t_0}^t r psi_4 dt',  H(t) = int_{t_0}^t N dt'      (t_0: the first record)
      dE/dt  =  1/(4 pi) oint |N|^2 dOmega
      dP/dt  =  1/(4 pi) oint n |N|^2 dOmega,  n = (sin th cos ph, sin th sin ph, cos th)
      dJz/dt = -1/(4 pi) Re oint conj(N) d_phi H dOmega

    Written out plainly: the time integrals by the trapezoid rule over the records
    (uniform step dt), the field summed over modes on a uniform azimuth grid fine
    enough to integrate every product exactly, theta by the midpoint rule of the
    waveform sum (weights sin(theta_j) dtheta), and E, P, Jz as trapezoid integrals of
    the rates from the first record.  ps: the modes' parameters (one problem: same s,
    M, a, theta grid, time step and extraction radius), waves: their records
    [k][n_theta][2], one record a time step.
    Returns [k][10]: dE/dt, dPx/dt, dPy/dt, dPz/dt, dJz/dt, E, Px, Py, Pz, Jz."""
    g = grid(ps[0])
    r = orbit(ps[0])["r_ext"]
    a, rp, rm, dt = ps[0].a, g["rp"], g["rm"], g["dt"]
    nth = ps[0].n_theta
    shift = a / (rp - rm) * np.log((r - rp) / (r - rm))
    dth = np.pi / nth
    th = (np.arange(nth) + 0.5) * dth
    ms = [p.m for p in ps]
    nrec = waves[0].shape[0]
    # r psi_4 of each mode, still without its azimuthal factor
    kerr = (r / (r - 1j * a * np.cos(th))) ** 4
    C = [(W[..., 0] + 1j * W[..., 1]) * kerr[None, :] for W in waves]
    # N and H: trapezoid rule from the first record, one record after the other
    N = [np.zeros((nrec, nth), np.complex128) for _ in ms]
    H = [np.zeros((nrec, nth), np.complex128) for _ in ms]
    for i in range(len(ms)):
        for k in range(1, nrec):
            N[i][k] = N[i][k - 1] + 0.5 * dt * (C[i][k - 1] + C[i][k])
            H[i][k] = H[i][k - 1] + 0.5 * dt * (N[i][k - 1] + N[i][k])
    # azimuth grid: |N|^2 times e^{+-i phi} holds harmonics up to (m_max - m_min + 1)
    L = 2 * (max(ms) - min(ms)) + 4
    ph = 2.0 * np.pi * np.arange(L) / L
    eph = [np.exp(1j * m * (ph + shift))[None, :] for m in ms]   # e^{i m phi~} on the grid
    dA = (np.sin(th) * dth)[:, None] * (2.0 * np.pi / L)          # dOmega of each (j, l)
    nx = np.sin(th)[:, None] * np.cos(ph)[None, :]
    ny = np.sin(th)[:, None] * np.sin(ph)[None, :]
    nz = np.cos(th)[:, None] * np.ones(L)[None, :]
    rates = np.zeros((nrec, 5))
    for k in range(nrec):
        Nf = np.zeros((nth, L), np.complex128)      # N(theta_j, phi_l) at record k
        dHf = np.zeros((nth, L), np.complex128)     # d_phi H
        for i, m in enumerate(ms):
            Nf += N[i][k][:, None] * eph[i]
            dHf += 1j * m * H[i][k][:, None] * eph[i]
        I2 = np.abs(Nf) ** 2
        rates[k, 0] = (I2 * dA).sum() / (4.0 * np.pi)
        rates[k, 1] = (nx * I2 * dA).sum() / (4.0 * np.pi)
        rates[k, 2] = (ny * I2 * dA).sum() / (4.0 * np.pi)
        rates[k, 3] = (nz * I2 * dA).sum() / (4.0 * np.pi)
        rates[k, 4] = -(np.real(np.conj(Nf) * dHf) * dA).sum() / (4.0 * np.pi)
    out = np.zeros((nrec, 10))
    out[:, :5] = rates
    for k in range(1, nrec):
        out[k, 5:] = out[k - 1, 5:] + 0.5 * dt * (rates[k - 1] + rates[k])
    return out


def apply_K(p: Params, x):
    y = np.zeros_like(x)
    _check(lib().orc_apply_K(ctypes.byref(p), _ptr(np.ascontiguousarray(x)), _ptr(y)))
    return y


def apply_KT(p: Params, y):
    x = np.zeros_like(y)
    _check(lib().orc_apply_KT(ctypes.byref(p), _ptr(np.ascontiguousarray(y)), _ptr(x)))
    return x


def adjoint(p: Params, source: Source, gwave, amps=None, step0=0):
    """Reverse sweep: returns (grad_amps [nsteps], grad_r0, lambda0 [4][nth][nr])."""
    gwave = np.ascontiguousarray(gwave, dtype=np.float64)
    nsteps = gwave.shape[0]
    ga = np.zeros(nsteps)
    gr = ctypes.c_double(0.0)
    lam0 = np.zeros((4, p.n_theta, p.n_rstar))
    a = None if amps is None else np.ascontiguousarray(amps, dtype=np.float64)
    na = 0 if a is None else a.size
    _check(lib().orc_adjoint(ctypes.byref(p), source.omega, source.phase0, _ptr(source.P_int),
                             _ptr(source.P_half), _ptr(source.dP_int), _ptr(source.dP_half),
                             source.domega, source.dphase0, _ptr(a), na, step0, nsteps,
                             _ptr(gwave), _ptr(ga), ctypes.byref(gr), _ptr(lam0)))
    return ga, gr.value, lam0


def theta_apply(p: Params, F):
    """Theta_h applied to one complex column F[n_theta] (with the angular ghosts)."""
    F = np.ascontiguousarray(F, dtype=np.complex128)
    out = np.zeros_like(F)
    _check(lib().orc_theta_apply(ctypes.byref(p), _ptr(F), _ptr(out)))
    return out


def r_ext(p: Params) -> float:
    return orbit(p)["r_ext"]
