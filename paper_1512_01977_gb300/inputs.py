"""Seeded synthetic initial fields and workload lists.

This module builds inputs only: density and velocity fields with the shapes of
the paper's validation cases, and the random mixes of solves used for the
batched and served workloads.  It holds none of the method's arithmetic (no
EOS, no lattice, no update); coexistence densities and temperatures arrive as
plain numbers from the caller.  Both the CUDA path and the CPU oracle take
their inputs from here.

Fields are float64 numpy arrays of shape (nr, nz): index [j, k] is the node at
z_k = k + 1/2, r_j = j + 1/2 (row-major, z contiguous).
"""
import math

import numpy as np


def grid(nz, nr):
    """Node coordinates (Z, R), each of shape (nr, nz)."""
    z = np.arange(nz) + 0.5
    r = np.arange(nr) + 0.5
    Z, R = np.meshgrid(z, r)
    return Z, R


def tanh_profile(d, R, rho_in, rho_out, width):
    """rho(d) = (rho_in + rho_out)/2 - (rho_in - rho_out)/2 tanh(2 (d - R) / width)."""
    return 0.5 * (rho_in + rho_out) - 0.5 * (rho_in - rho_out) * np.tanh(2.0 * (d - R) / width)


def droplet(nz, nr, R, rho_l, rho_v, width=2.0, zc=None, eps=0.0):
    """Axisymmetric droplet centred on the axis at z = zc (default nz/2).

    eps != 0 perturbs the radius by the second Legendre mode,
    R(theta) = R (1 + eps P2(cos theta)), theta measured from +z."""
    Z, Rr = grid(nz, nr)
    zc = nz / 2.0 if zc is None else zc
    dz = Z - zc
    d = np.sqrt(dz * dz + Rr * Rr)
    Rt = R
    if eps:
        cos_t = np.where(d > 0, dz / np.maximum(d, 1e-300), 1.0)
        Rt = R * (1.0 + eps * 0.5 * (3.0 * cos_t * cos_t - 1.0))
    rho = tanh_profile(d, Rt, rho_l, rho_v, width)
    return rho, np.zeros_like(rho), np.zeros_like(rho)


def ellipsoid(nz, nr, Ra, Rz, rho_l, rho_v, width=2.0, zc=None):
    """Axisymmetric ellipsoidal drop (r/Ra)^2 + ((z - zc)/Rz)^2 = 1 on the
    axis (semi-axes Ra radially, Rz along z), with the tanh profile applied
    to the scaled distance sqrt(...) times the equal-volume radius."""
    Z, Rr = grid(nz, nr)
    zc = nz / 2.0 if zc is None else zc
    Rm = (Ra * Ra * Rz) ** (1.0 / 3.0)
    s = np.sqrt((Rr / Ra) ** 2 + ((Z - zc) / Rz) ** 2)
    rho = tanh_profile(s * Rm, Rm, rho_l, rho_v, width)
    return rho, np.zeros_like(rho), np.zeros_like(rho)


def droplet_2d(nz, nr, R, rho_l, rho_v, width=2.0):
    """Planar (2D) droplet centred in a fully periodic nz x nr box."""
    Z, Rr = grid(nz, nr)
    d = np.sqrt((Z - nz / 2.0) ** 2 + (Rr - nr / 2.0) ** 2)
    rho = tanh_profile(d, R, rho_l, rho_v, width)
    return rho, np.zeros_like(rho), np.zeros_like(rho)


def slab(nz, nr, rho_l, rho_v, frac=0.5, width=2.0):
    """Liquid slab normal to z, centred at nz/2, of thickness frac*nz."""
    Z, _ = grid(nz, nr)
    d = np.abs(Z - nz / 2.0)
    rho = tanh_profile(d, 0.5 * frac * nz, rho_l, rho_v, width)
    return rho, np.zeros_like(rho), np.zeros_like(rho)


def density_wave(nz, nr, rho0, amp=0.01, noise=1e-4, seed=20151201):
    """rho = rho0 (1 + amp sin(2 pi z / nz)) + U(-noise, noise), u = 0.

    The noise is drawn with numpy's PCG64 (default_rng(seed)) in index order
    j * nz + k, so every consumer sees the same field."""
    Z, _ = grid(nz, nr)
    rng = np.random.default_rng(seed)
    rho = rho0 * (1.0 + amp * np.sin(2.0 * np.pi * Z / nz))
    rho = rho + rng.uniform(-noise, noise, size=nz * nr).reshape(nr, nz)
    return rho, np.zeros_like(rho), np.zeros_like(rho)


def radial_bump(nz, nr, rho0, rho_p, w_d, r_c=None):
    """rho = rho0 + rho_p exp(-((r - r_c)/w_d)^2), u = 0: a ring-shaped density
    disturbance that launches one wave towards the axis and one away from it."""
    _, Rr = grid(nz, nr)
    r_c = nr / 2.0 if r_c is None else r_c
    rho = rho0 + rho_p * np.exp(-(((Rr - r_c) / w_d) ** 2))
    return rho, np.zeros_like(rho), np.zeros_like(rho)


def radial_mode(nz, nr, rho0, eps, k):
    """rho = rho0 (1 + eps J0(k r)), u = 0 (a standing radial acoustic mode)."""
    from scipy import special

    _, Rr = grid(nz, nr)
    rho = rho0 * (1.0 + eps * special.j0(k * Rr))
    return rho, np.zeros_like(rho), np.zeros_like(rho)


def shear_wave(nz, nr, rho0, U):
    """u_z = U sin(2 pi r / nr), rho = rho0 (periodic in r)."""
    _, Rr = grid(nz, nr)
    rho = np.full((nr, nz), rho0)
    return rho, U * np.sin(2.0 * np.pi * Rr / nr), np.zeros_like(rho)


def uniform(nz, nr, rho0):
    rho = np.full((nr, nz), float(rho0))
    return rho, np.zeros_like(rho), np.zeros_like(rho)


def random_state(nz, nr, rho0, drho, du, seed):
    """Smoothly random density and velocity (low Fourier modes), for parity
    tests that must exercise every term of the update."""
    rng = np.random.default_rng(seed)
    Z, Rr = grid(nz, nr)
    rho = np.full((nr, nz), float(rho0))
    uz = np.zeros((nr, nz))
    ur = np.zeros((nr, nz))
    for _ in range(4):
        kz = rng.integers(1, 3) * 2.0 * np.pi / nz
        kr = rng.uniform(0.5, 2.0) * np.pi / nr
        ph = rng.uniform(0, 2 * np.pi, size=3)
        rho += drho * rng.uniform(0.3, 1.0) * np.cos(kz * Z + ph[0]) * np.cos(kr * Rr)
        uz += du * rng.uniform(0.3, 1.0) * np.cos(kz * Z + ph[1]) * np.cos(kr * Rr)
        ur += du * rng.uniform(0.3, 1.0) * np.cos(kz * Z + ph[2]) * np.sin(kr * Rr)
    return rho, uz, ur


# ---------------------------------------------------------- workload mixes --

def batch_droplets(n=256, seed=4, lo=(64, 32), scale_max=8.0):
    """Batched-droplet workload: sizes log-uniform between lo and scale_max*lo
    (same scale on both axes), radius 0.25 of the shorter side, T/T_c uniform
    in [0.5, 0.85], tau uniform in [0.6, 1.0].  Returns a list of dicts."""
    rng = np.random.default_rng(seed)
    out = []
    for _ in range(n):
        s = math.exp(rng.uniform(0.0, math.log(scale_max)))
        nz, nr = int(round(lo[0] * s)), int(round(lo[1] * s))
        out.append(dict(nz=nz, nr=nr, R=0.25 * min(nz, nr), T_over_Tc=float(rng.uniform(0.5, 0.85)),
                        tau=float(rng.uniform(0.6, 1.0))))
    return out


def request_stream(rate, n, seed=5, nz_range=(32, 1024), nr_range=(32, 512), steps_range=(1000, 20000),
                   T_range=(0.5, 0.9)):
    """Poisson arrival stream of droplet-oscillation and density-wave solves.

    Each request: arrival time (s), kind ('droplet' or 'wave'), EOS kind
    ('cs' or 'vdw'), grid (log-uniform per axis), step count (uniform) and
    T/T_c (uniform)."""
    rng = np.random.default_rng(seed)
    t = 0.0
    out = []
    for i in range(n):
        t += rng.exponential(1.0 / rate)
        nz = int(round(math.exp(rng.uniform(math.log(nz_range[0]), math.log(nz_range[1])))))
        nr = int(round(math.exp(rng.uniform(math.log(nr_range[0]), math.log(nr_range[1])))))
        out.append(dict(id=i, t_arrive=t, kind="droplet" if rng.random() < 0.5 else "wave",
                        eos="cs" if rng.random() < 0.5 else "vdw", nz=nz, nr=nr,
                        steps=int(rng.integers(steps_range[0], steps_range[1] + 1)),
                        T_over_Tc=float(rng.uniform(*T_range))))
    return out
