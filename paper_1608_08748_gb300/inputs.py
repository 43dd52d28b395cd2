"""Seeded synthetic initial conditions shared by the tests, the smoke check and the benchmark.

This module only builds inputs: it holds none of the time-step arithmetic and imports neither
the CUDA binding nor the oracle.  Every generator returns a dict with the conserved cell-centred
fields the C-ABI takes (``rho``, ``mom`` (3, nz, ny, nx), ``E``, ``B`` (3, nz, ny, nx),
``rho_h2`` or None), the adiabatic index ``gamma``, the cell size ``dx`` and ``options``
(boundary conditions, chemistry switch).  Arrays are float64, C order [k][j][i] (x fastest).

Code units for the astrophysical set-ups: length 1 pc, density m_H cm^-3 (so rho is the number
density of hydrogen nuclei in cm^-3), velocity 1 km/s, B in units where the Alfven speed is
B / sqrt(rho) (no 4 pi, as in the paper's total pressure p* = p + B^2/2).
"""
from __future__ import annotations

import numpy as np

KB_CGS = 1.380649e-16
MH_CGS = 1.6735575e-24
KMS_CGS = 1.0e5
P_UNIT_CGS = MH_CGS * KMS_CGS * KMS_CGS  # erg cm^-3 per code pressure unit


def conserved(rho, v, p, B, gamma, rho_h2=None):
    """Conserved state from primitives: m = rho v, rho E = p/(gamma-1) + rho v^2/2 + B^2/2."""
    rho = np.asarray(rho, dtype=np.float64)
    v = np.asarray(v, dtype=np.float64)
    B = np.asarray(B, dtype=np.float64)
    mom = rho[None] * v
    E = p / (gamma - 1.0) + 0.5 * rho * (v ** 2).sum(0) + 0.5 * (B ** 2).sum(0)
    return {"rho": np.ascontiguousarray(rho), "mom": np.ascontiguousarray(mom),
            "E": np.ascontiguousarray(E), "B": np.ascontiguousarray(B),
            "rho_h2": None if rho_h2 is None else np.ascontiguousarray(rho_h2, dtype=np.float64)}


def _tube(nx, ny, nz, left, right, gamma, x0=0.5, axis=0):
    """1D Riemann problem along `axis` on [0, 1): left/right = (rho, p, v(3), B(3))."""
    n = [nx, ny, nz][axis]
    shape = (nz, ny, nx)
    xc = (np.arange(n) + 0.5) / n
    sel = xc < x0
    idx = [None, None, None]
    idx[2 - axis] = slice(None)
    mask = np.broadcast_to(sel[tuple(idx)], shape)

    def field(a, b):
        return np.where(mask, a, b).astype(np.float64)

    rho = field(left[0], right[0])
    p = field(left[1], right[1])
    v = np.stack([field(left[2][c], right[2][c]) for c in range(3)])
    B = np.stack([field(left[3][c], right[3][c]) for c in range(3)])
    ic = conserved(rho, v, p, B, gamma)
    bc = [0, 0, 0]
    bc[axis] = 1
    ic.update(gamma=gamma, dx=1.0 / n,
              options={"bc_x": bc[0], "bc_y": bc[1], "bc_z": bc[2], "chem": 0})
    return ic


def brio_wu(nx=128, ny=4, nz=4, axis=0):
    """MHD shock tube of Brio & Wu: gamma = 2, left (rho, p, Bx, By, Bz) = (1, 1, 0.75, 1, 0),
    right (0.125, 0.1, 0.75, -1, 0), v = 0, jump at x = 0.5; outflow along the tube axis."""
    def perm(vec):  # vec given in (normal, t1, t2) = (x, y, z) for axis 0
        out = [0.0, 0.0, 0.0]
        for c in range(3):
            out[(axis + c) % 3] = vec[c]
        return out
    left = (1.0, 1.0, perm([0.0, 0.0, 0.0]), perm([0.75, 1.0, 0.0]))
    right = (0.125, 0.1, perm([0.0, 0.0, 0.0]), perm([0.75, -1.0, 0.0]))
    sizes = [nx, ny, nz]
    return _tube(*sizes, left, right, 2.0, axis=axis)


def barmin(nx=100, ny=4, nz=4):
    """Shock tube of Sec. 3.1 (Barmin et al. 1996), gamma = 1.4, B_x = 4 (B/sqrt(4 pi) listed, which
    is the code unit here): left (rho, p, v, B_y, B_z) = (0.18405, 0.3541, (3.8964, 0.5361, 2.4866),
    2.394, 1.197); right (0.1, 0.1, (-5.5, 0, 0), 2, 1); run to t = 0.15."""
    left = (0.18405, 0.3541, [3.8964, 0.5361, 2.4866], [4.0, 2.394, 1.197])
    right = (0.1, 0.1, [-5.5, 0.0, 0.0], [4.0, 2.0, 1.0])
    return _tube(nx, ny, nz, left, right, 1.4)


def sod(nx=128, ny=4, nz=4, gamma=1.4):
    """Hydrodynamic Sod tube (B = 0): left (1, 1), right (0.125, 0.1), v = 0."""
    z = [0.0, 0.0, 0.0]
    return _tube(nx, ny, nz, (1.0, 1.0, z, z), (0.125, 0.1, z, z), gamma)


def uniform(nx, ny, nz, rho=1.0, p=1.0, v=(0.0, 0.0, 0.0), B=(0.0, 0.0, 0.0), gamma=5.0 / 3.0,
            dx=None, chem=0, rho_h2=None):
    shape = (nz, ny, nx)
    r = np.full(shape, rho)
    vv = np.stack([np.full(shape, c) for c in v])
    BB = np.stack([np.full(shape, c) for c in B])
    h2 = None if rho_h2 is None else np.full(shape, rho_h2)
    ic = conserved(r, vv, np.full(shape, p), BB, gamma, h2)
    ic.update(gamma=gamma, dx=dx if dx is not None else 1.0 / nx,
              options={"bc_x": 0, "bc_y": 0, "bc_z": 0, "chem": chem})
    return ic


def orszag_tang(n=64, nz=4):
    """Orszag-Tang vortex of Sec. 3.2 on [0, 1)^2 x nz cells: rho = 25/(36 pi), p = 5/(12 pi),
    v = (-sin 2 pi y, sin 2 pi x), B = B0 (-sin 2 pi y, sin 4 pi x), B0 = 1/sqrt(4 pi),
    gamma = 5/3.  `bface` carries the face values (exactly divergence free)."""
    gamma = 5.0 / 3.0
    shape = (nz, n, n)
    xc = (np.arange(n) + 0.5) / n
    X = np.broadcast_to(xc[None, None, :], shape)
    Y = np.broadcast_to(xc[None, :, None], shape)
    B0 = 1.0 / np.sqrt(4.0 * np.pi)
    rho = np.full(shape, 25.0 / (36.0 * np.pi))
    p = np.full(shape, 5.0 / (12.0 * np.pi))
    v = np.stack([-np.sin(2 * np.pi * Y), np.sin(2 * np.pi * X), np.zeros(shape)])
    B = np.stack([-B0 * np.sin(2 * np.pi * Y), B0 * np.sin(4 * np.pi * X), np.zeros(shape)])
    ic = conserved(rho, v, p, B, gamma)
    # b_x depends on y only and b_y on x only, so the face values are the cell-centre values
    ic["bface"] = np.ascontiguousarray(np.stack([B[0], B[1], np.zeros(shape)]))
    ic.update(gamma=gamma, dx=1.0 / n, options={"bc_x": 0, "bc_y": 0, "bc_z": 0, "chem": 0})
    return ic


def solenoidal_field(shape, seed, kmin=1, kmax=8, slope=-2.0):
    """Random-phase solenoidal vector field on a periodic grid: Gaussian white noise per component,
    filtered in Fourier space to integer |k| in [kmin, kmax] with mode amplitude |k|^(slope)
    (shell power ~ k^(2 slope + 2) = k^-2 for slope -2), projected onto k . v = 0, normalised to
    unit 3D rms."""
    rng = np.random.default_rng(seed)
    nz, ny, nx = shape
    noise = rng.standard_normal((3,) + shape)
    fk = np.fft.rfftn(noise, axes=(1, 2, 3))
    kz = np.fft.fftfreq(nz, 1.0 / nz)[:, None, None]
    ky = np.fft.fftfreq(ny, 1.0 / ny)[None, :, None]
    kx = np.fft.rfftfreq(nx, 1.0 / nx)[None, None, :]
    k2 = kx ** 2 + ky ** 2 + kz ** 2
    kk = np.sqrt(k2)
    amp = np.where((kk >= kmin) & (kk <= kmax), np.power(np.maximum(kk, 1e-30), slope), 0.0)
    fk = fk * amp[None]
    kvec = [np.broadcast_to(kx, k2.shape), np.broadcast_to(ky, k2.shape),
            np.broadcast_to(kz, k2.shape)]
    kdotv = sum(kvec[c] * fk[c] for c in range(3))
    inv = np.where(k2 > 0, 1.0 / np.maximum(k2, 1e-30), 0.0)
    for c in range(3):
        fk[c] = fk[c] - kvec[c] * kdotv * inv
    v = np.fft.irfftn(fk, s=shape, axes=(1, 2, 3))
    rms = np.sqrt((v ** 2).sum(0).mean())
    return v / rms


def turbulence(n=128, mach=5.0, beta=1.0, seed=1, n_cm3=100.0, T_K=100.0, box_pc=256.0,
               chem=1, shape=None):
    """Decaying supersonic MHD turbulence with hydrogen chemistry: uniform n (cm^-3) of atomic
    hydrogen at temperature T, random-phase solenoidal velocity with shell power ~ k^-2 for
    integer k = 1..8 scaled to 3D rms Mach `mach` (sound speed at gamma = 5/3), uniform B_z at
    plasma beta 2 p / B^2 = `beta`, rho_H2 = 0, periodic box of `box_pc` parsecs."""
    gamma = 5.0 / 3.0
    shape = tuple(shape) if shape is not None else (n, n, n)
    nz, ny, nx = shape
    rho = np.full(shape, float(n_cm3))
    p0 = n_cm3 * KB_CGS * T_K / P_UNIT_CGS
    cs = np.sqrt(gamma * p0 / n_cm3)
    v = solenoidal_field(shape, seed) * (mach * cs)
    Bz = np.sqrt(2.0 * p0 / beta)
    B = np.stack([np.zeros(shape), np.zeros(shape), np.full(shape, Bz)])
    ic = conserved(rho, v, np.full(shape, p0), B, gamma, np.zeros(shape))
    ic.update(gamma=gamma, dx=box_pc / nx,
              options={"bc_x": 0, "bc_y": 0, "bc_z": 0, "chem": chem})
    return ic


def turbulence_from_field(v_unit, mach=5.0, beta=1.0, shift=(0, 0, 0), n_cm3=100.0, T_K=100.0,
                          box_pc=256.0, chem=1):
    """Turbulence initial state from a precomputed unit-rms solenoidal field (as made by
    solenoidal_field), periodically shifted by `shift` cells (a cheap new realisation of the same
    statistics), with the set-up of `turbulence`."""
    gamma = 5.0 / 3.0
    shape = v_unit.shape[1:]
    rho = np.full(shape, float(n_cm3))
    p0 = n_cm3 * KB_CGS * T_K / P_UNIT_CGS
    cs = np.sqrt(gamma * p0 / n_cm3)
    v = np.roll(v_unit, shift=tuple(int(x) for x in shift), axis=(1, 2, 3)) * (mach * cs)
    Bz = np.sqrt(2.0 * p0 / beta)
    B = np.stack([np.zeros(shape), np.zeros(shape), np.full(shape, Bz)])
    ic = conserved(rho, v, np.full(shape, p0), B, gamma, np.zeros(shape))
    ic.update(gamma=gamma, dx=box_pc / shape[2],
              options={"bc_x": 0, "bc_y": 0, "bc_z": 0, "chem": chem})
    return ic


def ensemble_boxes(count=64, seed=4):
    """Box table of the batched ensemble: per box, each axis from {16, 24, ..., 96}, Mach from
    U[1, 10], beta log-uniform in [0.1, 10], turbulence seed = seed + box index."""
    rng = np.random.default_rng(seed)
    sizes = rng.choice(np.arange(16, 97, 8), size=(count, 3))
    mach = rng.uniform(1.0, 10.0, size=count)
    beta = 10.0 ** rng.uniform(-1.0, 1.0, size=count)
    return [{"shape": (int(s[2]), int(s[1]), int(s[0])), "mach": float(m), "beta": float(b),
             "seed": seed + i} for i, (s, m, b) in enumerate(zip(sizes, mach, beta))]


def serving_arrivals(rate=20.0, duration=60.0, seed=5, big_prob=0.005):
    """Poisson request stream: arrival times, cubic size n in {32, 40, ..., 192} (512 with
    probability big_prob), steps in {20..200}."""
    rng = np.random.default_rng(seed)
    t, out = 0.0, []
    while True:
        t += rng.exponential(1.0 / rate)
        if t > duration:
            break
        n = 512 if rng.random() < big_prob else int(rng.choice(np.arange(32, 193, 8)))
        out.append({"t": t, "n": n, "steps": int(rng.integers(20, 201)),
                    "mach": float(rng.uniform(1.0, 10.0)), "beta": float(10.0 ** rng.uniform(-1, 1)),
                    "seed": 1000 + len(out)})
    return out
