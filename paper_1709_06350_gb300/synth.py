"""Seeded synthetic inputs (the only module shared by the CUDA path's tests
and the oracle's).  It holds none of the reconstruction method's arithmetic:
no stencil, no determinant, no cubic, no density assignment.

Recipe (stand-in for the paper's N-body snapshots, which are not available):

1. white noise ``numpy.random.default_rng(seed).standard_normal((N, N, N))``;
2. Fourier filter by sqrt(P(k)), P(k) = k^-1.5 exp(-(k / 1 h/Mpc)^2),
   k = 2 pi m / L, the k = 0 mode zeroed;
3. scale so that the rms of the linear field on the grid is ``sigma_lin``;
4. Zel'dovich displacement psi = i k delta / k^2 (so that delta = -div psi);
   particles start on cell centres q = (i + 1/2) h and move to
   x = q + psi(q) (mod L).

The density assigned from these particles (a CIC deposit) is then
conditioned -- Gaussian window exp(-k^2 R^2 / 2), a floor 1 + delta >= 0.05
and a renormalisation to mean 1 -- by the code under test
(``recon_smooth_density``) or by the oracle (``oracle.smooth_and_floor``);
this module holds none of that arithmetic.

``backend="torch"`` runs the FFTs with torch (on a CUDA device when one is
given) for sizes where numpy's single-threaded FFT is slow; the white noise
always comes from numpy's generator so the field is the same either way up
to FFT rounding.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np


@dataclass(frozen=True)
class Workload:
    """One seeded synthetic workload: grid, box, field amplitude, smoothing."""
    name: str
    N: int
    L: float          # box side, Mpc/h
    sigma_lin: float  # rms of the linear field on the grid
    R: float          # Gaussian smoothing radius, Mpc/h
    tol: float        # solver stop rule ||r|| / ||b - 1||
    seed: int


# The five workload families of the benchmark plan.  seed = 1000 * family + r.
WORKLOADS = {
    "fp64-32": Workload("fp64-32", 32, 100.0, 0.5, 5.0, 1e-10, 1000),
    "zel-128": Workload("zel-128", 128, 256.0, 0.8, 4.0, 1e-10, 2000),
    "mixed-384": Workload("mixed-384", 384, 384.0, 1.0, 2.0, 1e-8, 3002),
    "mixed-512": Workload("mixed-512", 512, 512.0, 1.0, 2.0, 1e-8, 3000),
    "mixed-1024": Workload("mixed-1024", 1024, 1024.0, 1.0, 2.0, 1e-8, 3001),
    "adjoint-256": Workload("adjoint-256", 256, 512.0, 0.8, 4.0, 1e-10, 5000),
}


def batched_workloads(count: int = 64):
    """Family 4: ``count`` realisations, N cycling through 64..256, h = 2 Mpc/h."""
    sizes = (64, 96, 128, 192, 256)
    return [Workload(f"batch-{r}", sizes[r % len(sizes)], 2.0 * sizes[r % len(sizes)],
                     0.8, 4.0, 1e-8, 4000 + r) for r in range(count)]


def _kgrid(N: int, L: float):
    kf = 2.0 * np.pi / L
    k1 = np.fft.fftfreq(N, d=1.0 / N) * kf
    kz = np.fft.rfftfreq(N, d=1.0 / N) * kf
    return k1[:, None, None], k1[None, :, None], kz[None, None, :]


def _power(k):
    with np.errstate(divide="ignore"):
        P = np.where(k > 0, k ** -1.5 * np.exp(-(k / 1.0) ** 2), 0.0)
    return P


def linear_field(N: int, L: float, sigma_lin: float, seed: int,
                 backend: str = "numpy", device=None):
    """Gaussian random field with P(k) ~ k^-1.5 exp(-k^2), rms sigma_lin.

    Returns ``(delta_L, delta_hat)``: the real field [N,N,N] (float64) and
    its rFFT (numpy or torch complex, matching ``backend``).
    """
    white = np.random.default_rng(seed).standard_normal((N, N, N))
    kx, ky, kz = _kgrid(N, L)
    k = np.sqrt(kx * kx + ky * ky + kz * kz)
    amp = np.sqrt(_power(k))
    if backend == "numpy":
        dh = np.fft.rfftn(white) * amp
        d = np.fft.irfftn(dh, s=(N, N, N), axes=(0, 1, 2))
        s = sigma_lin / d.std()
        return d * s, dh * s
    import torch
    dev = torch.device(device) if device is not None else torch.device("cpu")
    w = torch.from_numpy(white).to(dev)
    dh = torch.fft.rfftn(w) * torch.from_numpy(amp).to(dev)
    d = torch.fft.irfftn(dh, s=(N, N, N))
    s = sigma_lin / float(d.std(unbiased=False))
    return d * s, dh * s


def zeldovich_positions(delta_hat, N: int, L: float):
    """Particle positions [N^3, 3] (float64) displaced by psi = i k delta / k^2."""
    kx, ky, kz = _kgrid(N, L)
    k2 = kx * kx + ky * ky + kz * kz
    k2[0, 0, 0] = 1.0
    h = L / N
    cell = (np.arange(N) + 0.5) * h
    if isinstance(delta_hat, np.ndarray):
        comps = []
        for kk in (kx, ky, kz):
            comps.append(np.fft.irfftn(1j * kk / k2 * delta_hat, s=(N, N, N), axes=(0, 1, 2)))
        q = np.meshgrid(cell, cell, cell, indexing="ij")
        pos = np.stack([np.mod(q[d] + comps[d], L) for d in range(3)], axis=-1)
        return np.ascontiguousarray(pos.reshape(-1, 3))
    import torch
    dev = delta_hat.device
    inv = torch.from_numpy(1.0 / k2).to(dev)
    qc = torch.from_numpy(cell).to(dev)
    out = torch.empty((N, N, N, 3), dtype=torch.float64, device=dev)
    for d, kk in enumerate((kx, ky, kz)):
        fac = torch.from_numpy(kk).to(dev) * inv
        psi = torch.fft.irfftn(1j * fac * delta_hat, s=(N, N, N))
        shape = [1, 1, 1]
        shape[d] = N
        out[..., d] = torch.remainder(qc.view(shape) + psi, L)
        del psi
    return out.reshape(-1, 3)


def lattice_positions(N: int, L: float) -> np.ndarray:
    """Unperturbed particles on cell centres, [N^3, 3]."""
    h = L / N
    cell = (np.arange(N) + 0.5) * h
    q = np.meshgrid(cell, cell, cell, indexing="ij")
    return np.ascontiguousarray(np.stack(q, axis=-1).reshape(-1, 3))


def cube_positions(n: int, L: float, l: float) -> np.ndarray:
    """The cubic test's particles: an n^3 lattice filling a cube of side l at
    the centre of the box of side L (cell-centred sub-lattice), [n^3, 3]."""
    s = (np.arange(n) + 0.5) * (l / n) + 0.5 * (L - l)
    q = np.meshgrid(s, s, s, indexing="ij")
    return np.ascontiguousarray(np.stack(q, axis=-1).reshape(-1, 3))


def smooth_field(N: int, seed: int, amplitude: float, kmax: int = 3) -> np.ndarray:
    """A smooth periodic test field: a few random low-order Fourier modes.

    Used to build manufactured potentials and small-grid densities.
    """
    rng = np.random.default_rng(seed)
    x = np.arange(N) / N
    X, Y, Z = np.meshgrid(x, x, x, indexing="ij")
    f = np.zeros((N, N, N))
    for _ in range(6):
        m = rng.integers(-kmax, kmax + 1, size=3)
        if not m.any():
            continue
        ph = rng.uniform(0, 2 * np.pi)
        f += rng.normal() * np.sin(2 * np.pi * (m[0] * X + m[1] * Y + m[2] * Z) + ph)
    f -= f.mean()
    s = np.abs(f).max()
    return f * (amplitude / s) if s > 0 else f
