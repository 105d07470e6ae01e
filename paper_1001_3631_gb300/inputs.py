"""Seeded synthetic inputs shared by the tests and the benchmark.

This module holds none of the method's arithmetic: only the problem statements
of the named workloads (grid, spin, mode, orbit, step counts) and seeded random
initial data / amplitudes, generated from index coordinates."""
from __future__ import annotations

import numpy as np

# Named workloads (sizes of the paper-style runs; all sources are the synthetic
# smeared circular orbit, all data synthetic).
SINGLE_MODE_800x64 = dict(
    params=dict(s=-2, m=2, M=1.0, a=0.9, rstar_min=-50.0, rstar_max=150.0, n_rstar=800,
                n_theta=64, courant=0.5, dt_rule=1, rstar_ext=140.0),
    r0=10.0, steps=2000)
PAPER_SCALE_16384x256 = dict(
    params=dict(s=-2, m=2, M=1.0, a=0.9, rstar_min=-200.0, rstar_max=800.0, n_rstar=16384,
                n_theta=256, courant=0.5, dt_rule=1, rstar_ext=700.0),
    r0=8.0, steps=20000)
LONG_RUN_8192x128 = dict(
    params=dict(s=-2, m=2, M=1.0, a=0.99, rstar_min=-200.0, rstar_max=800.0, n_rstar=8192,
                n_theta=128, courant=0.5, dt_rule=1, rstar_ext=400.0),
    r0=8.0, steps=100000)
ADJOINT_4096x128 = dict(
    params=dict(s=-2, m=2, M=1.0, a=0.7, rstar_min=-200.0, rstar_max=800.0, n_rstar=4096,
                n_theta=128, courant=0.5, dt_rule=1, rstar_ext=300.0),
    r0=9.0, steps=10000, amp_seed=5005, ckpt_every=100)


def batched_uneven(seed=3003, n_modes=8, n_orbits=16):
    """8 modes (m = 1..8) x 16 orbits: r0 ~ U[6, 20], a ~ U[0, 0.95] per orbit, per
    instance N_r* ~ U{2048, 4096, 8192, 16384}, N_theta ~ U{64, 128, 256}."""
    rng = np.random.default_rng(seed)
    orbits = [(float(rng.uniform(6.0, 20.0)), float(rng.uniform(0.0, 0.95)))
              for _ in range(n_orbits)]
    out = []
    for m in range(1, n_modes + 1):
        for (r0, a) in orbits:
            nr = int(rng.choice([2048, 4096, 8192, 16384]))
            nth = int(rng.choice([64, 128, 256]))
            out.append(dict(params=dict(s=-2, m=m, M=1.0, a=a, rstar_min=-200.0, rstar_max=800.0,
                                        n_rstar=nr, n_theta=nth, courant=0.5, dt_rule=1,
                                        rstar_ext=700.0), r0=r0))
    return out


def eccentric_trajectory(n_samples, dt, semi_latus=10.0, ecc=0.4, incl=0.3, chi0=0.0,
                         amp_sigma=0.0, seed=6006):
    """Samples {r_p, theta_p, phi_p, A} at t = k dt/2, k = 0 .. n_samples - 1, of a
    synthetic eccentric, inclined particle path: a Keplerian ellipse
    r = p / (1 + e cos chi) (Kepler's equation for the anomaly, unit mass) on a plane
    tilted by ``incl`` about the x axis, with A ~ N(1, amp_sigma^2) per sample.  An
    input shape for the moving-source path, not a Kerr geodesic."""
    t = 0.5 * dt * np.arange(n_samples, dtype=np.float64)
    a_sm = semi_latus / (1.0 - ecc * ecc)
    mean_motion = a_sm ** -1.5
    E0 = 2.0 * np.arctan(np.sqrt((1.0 - ecc) / (1.0 + ecc)) * np.tan(0.5 * chi0))
    Mn = E0 - ecc * np.sin(E0) + mean_motion * t
    E = Mn.copy()
    for _ in range(50):   # Newton on Kepler's equation E - e sin E = M
        E = E - (E - ecc * np.sin(E) - Mn) / (1.0 - ecc * np.cos(E))
    chi = 2.0 * np.arctan2(np.sqrt(1.0 + ecc) * np.sin(0.5 * E), np.sqrt(1.0 - ecc) * np.cos(0.5 * E))
    r = a_sm * (1.0 - ecc * np.cos(E))
    x, y, z = np.cos(chi), np.sin(chi) * np.cos(incl), np.sin(chi) * np.sin(incl)
    theta = np.arccos(np.clip(z, -1.0, 1.0))
    phi = np.unwrap(np.arctan2(y, x))
    A = np.ones(n_samples)
    if amp_sigma > 0:
        A += amp_sigma * np.random.default_rng(seed).standard_normal(n_samples)
    return np.stack([r, theta, phi, A], axis=1)


def amplitudes(n, seed=5005, sigma=0.1):
    """Per-step source amplitudes A_n ~ N(1, sigma^2)."""
    return 1.0 + sigma * np.random.default_rng(seed).standard_normal(n)


def smooth_state(n_theta, n_rstar, seed=1001, n_bumps=3):
    """Random smooth initial data in u-layout [4][n_theta][n_rstar]: a sum of
    Gaussian bumps in the normalised radial index times sin^4 of the normalised
    angular index, with random complex weights, zero at both radial ends."""
    rng = np.random.default_rng(seed)
    x = np.arange(n_rstar) / (n_rstar - 1)
    y = (np.arange(n_theta) + 0.5) / n_theta
    ang = np.sin(np.pi * y) ** 4
    u = np.zeros((4, n_theta, n_rstar))
    for _ in range(n_bumps):
        c, w = rng.uniform(0.2, 0.8), rng.uniform(0.03, 0.1)
        prof = np.exp(-((x - c) / w) ** 2)
        for k in range(4):
            u[k] += rng.standard_normal() * np.outer(ang, prof)
    u[:, :, 0] = 0.0
    u[:, :, -1] = 0.0
    return u


def random_state(n_theta, n_rstar, seed=7):
    """Unstructured random initial data in u-layout (exercises every lane and row)."""
    return np.random.default_rng(seed).standard_normal((4, n_theta, n_rstar))
