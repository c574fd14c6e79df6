"""Seeded synthetic inputs for BU-MBAR problems.

This module only *draws* reduced-potential matrices u_kn and their sample
counts; it holds none of the estimator's arithmetic (no log-sum-exp, no
free energies). Both the CUDA path and the CPU oracle are fed from here.

Every generator is a pure function of its arguments and its seed: the
random stream is numpy's Philox counter-based generator, so a problem is
reproducible from (kind, sizes, seed) alone.

Workloads
---------
harmonic    K harmonic wells u_k(x) = 0.5*kappa_k*|x - mu_k|^2 in d dims,
            exact Gaussian samples (the plain-FP64 MBAR case).
umbrella    1-D double well U(x) = 5(x^2-1)^2 with K harmonic bias windows
            0.5*kappa*(x - x_k)^2 on [-1.5, 1.5]; samples drawn per window by
            inverse CDF of the tabulated window density.
alchemical  u_kn = u0_n + lambda_k * du_n, lambda_k = sin^2(pi k / (2(K-1)))
            (denser near both ends), du_n = 20 kT * student-t(nu=4),
            u0_n = -1e4 + 100 N(0,1) kT; all samples i.i.d. regardless of the
            state label (a numerical stress case with heavy tails and a large
            per-sample offset).
gaussian_overlap  energies of the paper's synthetic scaling study (Sec. IV):
            unit-variance normal energy histograms with a fixed overlap between
            neighbouring states, u_kn = beta_k * E_n.
parallel_tempering  a PT-shaped stand-in (Sec. III): K inverse temperatures
            exponentially spaced in T between 298 K and 600 K, u_kn = beta_k E_n,
            with a Gaussian density-of-states energy model.
"""
from __future__ import annotations

from dataclasses import dataclass, field
import math

import numpy as np


def _rng(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.Philox(seed))


@dataclass
class Problem:
    """A K-state, N-sample problem: row-major u_kn (float64) plus N_k.

    ``phi`` is the 1-D bin coordinate used by the binning step (None means the
    library default, row 0 of u_kn). ``meta`` carries the generator's
    parameters so a test can compute closed-form references itself.
    """
    kind: str
    u_kn: np.ndarray | None
    N_k: np.ndarray
    phi: np.ndarray | None = None
    meta: dict = field(default_factory=dict)

    @property
    def K(self) -> int:
        return int(self.N_k.shape[0])

    @property
    def N(self) -> int:
        return int(self.N_k.sum())


def harmonic(K: int = 8, d: int = 3, N_k: int = 1000, seed: int = 0) -> Problem:
    """K harmonic states, kappa_k ~ U[1,4], mu_k ~ U[0,2]^d, N_k exact samples each."""
    g = _rng(seed)
    kappa = g.uniform(1.0, 4.0, size=K)
    mu = g.uniform(0.0, 2.0, size=(K, d))
    xs = []
    for k in range(K):
        xs.append(mu[k] + g.standard_normal((N_k, d)) / np.sqrt(kappa[k]))
    x = np.concatenate(xs, axis=0)                       # N x d
    diff = x[None, :, :] - mu[:, None, :]                # K x N x d
    u = 0.5 * kappa[:, None] * np.sum(diff * diff, axis=2)
    Nk = np.full(K, N_k, dtype=np.int64)
    return Problem("harmonic", np.ascontiguousarray(u), Nk, phi=None,
                   meta=dict(kappa=kappa, mu=mu, d=d, x=x))


def double_well(x):
    return 5.0 * (x * x - 1.0) ** 2


def umbrella(K: int = 64, N_k: int = 5000, kappa: float = 50.0, seed: int = 0,
             grid_points: int = 1 << 18) -> Problem:
    """Umbrella windows on the double well; inverse-CDF sampling per window.

    The window density exp(-U(x) - kappa/2 (x-x_k)^2) is tabulated on a
    uniform grid over [x_k - 1.5, x_k + 1.5] (the density there is > 1e-20 of
    its peak only well inside the interval), its CDF is accumulated with the
    trapezoid rule, and uniforms are mapped through the piecewise-linear
    inverse CDF.
    """
    g = _rng(seed)
    centres = np.linspace(-1.5, 1.5, K)
    xs = []
    for k in range(K):
        grid = np.linspace(centres[k] - 1.5, centres[k] + 1.5, grid_points)
        e = double_well(grid) + 0.5 * kappa * (grid - centres[k]) ** 2
        dens = np.exp(-(e - e.min()))
        cdf = np.concatenate([[0.0], np.cumsum(0.5 * (dens[1:] + dens[:-1]))])
        cdf /= cdf[-1]
        uu = g.uniform(0.0, 1.0, size=N_k)
        xs.append(np.interp(uu, cdf, grid))
    x = np.concatenate(xs)
    u = double_well(x)[None, :] + 0.5 * kappa * (x[None, :] - centres[:, None]) ** 2
    Nk = np.full(K, N_k, dtype=np.int64)
    return Problem("umbrella", np.ascontiguousarray(u), Nk, phi=x.copy(),
                   meta=dict(centres=centres, kappa=kappa))


def alchemical_lambdas(K: int) -> np.ndarray:
    if K == 1:
        return np.zeros(1)
    k = np.arange(K)
    return np.sin(np.pi * k / (2.0 * (K - 1))) ** 2


def alchemical_factors(K: int = 500, N_k: int = 4000, nu: float = 4.0, scale: float = 20.0,
                       seed: int = 0):
    """(lambda_k, u0_n, du_n, N_k) for u_kn = u0_n + lambda_k du_n."""
    g = _rng(seed)
    N = K * N_k
    lam = alchemical_lambdas(K)
    du = scale * g.standard_t(nu, size=N)
    u0 = -1.0e4 + 100.0 * g.standard_normal(N)
    Nk = np.full(K, N_k, dtype=np.int64)
    return lam, u0, du, Nk


def alchemical_rows(lam, u0, du, k0: int, k1: int) -> np.ndarray:
    """Rows k0..k1-1 of u_kn = u0_n + lambda_k du_n, float64."""
    return u0[None, :] + lam[k0:k1, None] * du[None, :]


def alchemical(K: int = 500, N_k: int = 4000, nu: float = 4.0, scale: float = 20.0,
               seed: int = 0, materialize: bool = True) -> Problem:
    lam, u0, du, Nk = alchemical_factors(K, N_k, nu, scale, seed)
    u = alchemical_rows(lam, u0, du, 0, K) if materialize else None
    return Problem("alchemical", u, Nk, phi=du.copy(),
                   meta=dict(lam=lam, u0=u0, du=du))


def gaussian_overlap(M: int = 20, N_0: int = 1000, overlap: float = 0.8, seed: int = 0) -> Problem:
    """Sec. IV synthetic data: unit-variance normal energy histograms whose
    neighbours overlap by ``overlap`` (the overlapping coefficient of two
    unit normals at distance D is 2*Phi(-D/2)).

    With a Gaussian density of states, state beta has energies N(-beta, 1),
    so consecutive means differ by D = delta beta; u_kn = beta_k E_n.
    """
    g = _rng(seed)
    # 2*Phi(-D/2) = overlap  ->  D = -2 * Phi^{-1}(overlap / 2)
    from statistics import NormalDist
    D = -2.0 * NormalDist().inv_cdf(overlap / 2.0)
    beta = 1.0 + D * np.arange(M)
    E = np.concatenate([-beta[k] + g.standard_normal(N_0) for k in range(M)])
    u = beta[:, None] * E[None, :]
    Nk = np.full(M, N_0, dtype=np.int64)
    return Problem("gaussian_overlap", np.ascontiguousarray(u), Nk, phi=E.copy(),
                   meta=dict(beta=beta, spacing=D))


def overlap_spacing(overlap: float = 0.8) -> float:
    """Distance D between the means of two unit normals whose overlapping
    coefficient 2 Phi(-D/2) is ``overlap`` (the Sec. IV construction)."""
    from statistics import NormalDist
    return -2.0 * NormalDist().inv_cdf(overlap / 2.0)


def gaussian_overlap_device(M: int, N_i: int, seed: int, overlap: float = 0.8, device="cuda"):
    """(beta float64 [M] on `device`, E float64 [M N_i] on `device`, N_k):
    the Sec. IV energies of `gaussian_overlap` drawn with torch's Philox
    generator on the device (state k: E ~ N(-beta_k, 1), beta_k = 1 + D k);
    the reduced potentials are u_kn = beta_k E_n (the factorised form)."""
    import torch
    g = torch.Generator(device=device)
    g.manual_seed(int(seed))
    beta = 1.0 + overlap_spacing(overlap) * torch.arange(M, device=device, dtype=torch.float64)
    E = torch.randn(M, N_i, generator=g, device=device, dtype=torch.float64)
    E.sub_(beta[:, None])
    return beta, E.reshape(-1).contiguous(), np.full(M, N_i, dtype=np.int64)


def parallel_tempering(K: int = 50, N_k: int = 200_000, T_min: float = 298.0, T_max: float = 600.0,
                       sigma2: float = 2000.0, seed: int = 0, materialize: bool = True) -> Problem:
    """PT-shaped stand-in for the Sec. III workload (no MD data available).

    Temperatures T_k = T_min exp(t_k), t_k equidistant on [0, log(T_max/T_min)]
    (the OpenMM schedule quoted in Sec. III). Energies, in units of kT_min,
    come from a Gaussian density of states of variance sigma2: at reduced
    inverse temperature b_k = T_min/T_k the energy is N(-b_k sigma2, sigma2).
    Reduced potentials u_kn = b_k E_n.
    """
    g = _rng(seed)
    t = np.linspace(0.0, math.log(T_max / T_min), K)
    T = T_min * np.exp(t)
    b = T_min / T
    sd = math.sqrt(sigma2)
    E = np.concatenate([-b[k] * sigma2 + sd * g.standard_normal(N_k) for k in range(K)])
    u = (b[:, None] * E[None, :]) if materialize else None
    Nk = np.full(K, N_k, dtype=np.int64)
    return Problem("parallel_tempering", u, Nk, phi=E.copy(), meta=dict(T=T, b=b, sigma2=sigma2))


def batch_of_problems(count: int = 512, K_range=(4, 256), N_k_range=(100, 10000), seed: int = 0,
                      scale: float = 1.0):
    """Uneven problems for the batched form: alternating harmonic (d=3) and
    umbrella; K ~ U{K_range}, N_k ~ U{N_k_range} (both scaled by ``scale``)."""
    g = _rng(seed)
    out = []
    for i in range(count):
        K = int(g.integers(K_range[0], K_range[1] + 1))
        Nk = max(2, int(g.integers(N_k_range[0], N_k_range[1] + 1) * scale))
        s = int(g.integers(0, 2**31 - 1))
        if i % 2 == 0:
            out.append(harmonic(K=K, d=3, N_k=Nk, seed=s))
        else:
            out.append(umbrella(K=K, N_k=Nk, seed=s, grid_points=1 << 14))
    return out


# ---------------------------------------------------------------------------
# device-side generators (torch on the GPU): the batched and served workloads
# are too large to draw on the host. Same models as harmonic / umbrella above,
# drawn with torch's counter-based Philox generator from (kind, K, N_k, seed).
# ---------------------------------------------------------------------------

def harmonic_device(K: int, N_k: int, seed: int, d: int = 3, device="cuda"):
    """(u_kn float64 K x N on `device`, N_k array, phi=None): harmonic wells,
    kappa_k ~ U[1,4], mu_k ~ U[0,2]^d, N_k exact Gaussian samples per state.
    u_kn = 0.5 kappa_k (|x|^2 - 2 mu_k.x + |mu_k|^2), formed by one small
    matrix product (no K x N x d intermediate)."""
    import torch
    g = torch.Generator(device=device)
    g.manual_seed(int(seed))
    kappa = 1.0 + 3.0 * torch.rand(K, generator=g, device=device, dtype=torch.float64)
    mu = 2.0 * torch.rand(K, d, generator=g, device=device, dtype=torch.float64)
    x = torch.empty(K * N_k, d, device=device, dtype=torch.float64)
    step = max(1, (1 << 24) // max(1, N_k * d))        # states per chunk of draws
    for k0 in range(0, K, step):
        k1 = min(K, k0 + step)
        z = torch.randn(k1 - k0, N_k, d, generator=g, device=device, dtype=torch.float64)
        z.div_(torch.sqrt(kappa[k0:k1])[:, None, None]).add_(mu[k0:k1, None, :])
        x[k0 * N_k:k1 * N_k] = z.reshape(-1, d)
    x2 = (x * x).sum(dim=1)
    mu2 = (mu * mu).sum(dim=1)
    u = mu @ x.T                                        # K x N, formed in place from here on
    u.mul_(-2.0).add_(x2[None, :]).add_(mu2[:, None]).mul_(0.5 * kappa[:, None]).clamp_(min=0.0)
    return u.contiguous(), np.full(K, N_k, dtype=np.int64), None


def _umbrella_samples_device(K: int, N_k: int, seed: int, kappa: float, grid_points: int, device):
    """(window centres x_k, samples x in state-major order) of `umbrella_device`."""
    import torch
    g = torch.Generator(device=device)
    g.manual_seed(int(seed))
    xc = torch.linspace(-1.5, 1.5, K, device=device, dtype=torch.float64)
    t = torch.linspace(-1.5, 1.5, grid_points, device=device, dtype=torch.float64)
    grid = xc[:, None] + t[None, :]                                    # K x G
    logp = -5.0 * (grid * grid - 1.0) ** 2 - 0.5 * kappa * (grid - xc[:, None]) ** 2
    p = torch.exp(logp - logp.max(dim=1, keepdim=True).values)
    cdf = torch.zeros_like(p)
    cdf[:, 1:] = torch.cumsum(0.5 * (p[:, 1:] + p[:, :-1]), dim=1)
    cdf /= cdf[:, -1:].clone()
    r = torch.rand(K, N_k, generator=g, device=device, dtype=torch.float64)
    j = torch.searchsorted(cdf, r).clamp_(1, grid_points - 1)
    c0 = torch.gather(cdf, 1, j - 1)
    c1 = torch.gather(cdf, 1, j)
    x0 = torch.gather(grid, 1, j - 1)
    x1 = torch.gather(grid, 1, j)
    w = torch.where(c1 > c0, (r - c0) / (c1 - c0), torch.zeros_like(r))
    return xc, (x0 + w * (x1 - x0)).reshape(-1)


def umbrella_device(K: int, N_k: int, seed: int, kappa: float = 50.0, grid_points: int = 4096, device="cuda"):
    """(u_kn float64 K x N, N_k array, phi = x): the umbrella windows of
    `umbrella`, sampled by inverse CDF of each window's density tabulated on
    `grid_points` points over [x_k - 1.5, x_k + 1.5] (trapezoid CDF, linear
    interpolation)."""
    xc, x = _umbrella_samples_device(K, N_k, seed, kappa, grid_points, device)
    well = 5.0 * (x * x - 1.0) ** 2
    u = x[None, :].repeat(K, 1)                          # K x N, formed in place from here on
    u.sub_(xc[:, None]).square_().mul_(0.5 * kappa).add_(well[None, :])
    return u.contiguous(), np.full(K, N_k, dtype=np.int64), x.contiguous()


def umbrella_factorised_device(K: int, N_k: int, seed: int, kappa: float = 50.0, grid_points: int = 4096,
                               device="cuda"):
    """(a, b, phi, N_k): the samples of `umbrella_device` with u in the
    factorised form u_kn = a_k + b_k phi_n, a_k = kappa x_k^2 / 2,
    b_k = -kappa x_k, phi = x. This drops U(x_n) + kappa x_n^2 / 2 from every
    u_kn; a term that depends on the sample alone cancels between the
    numerator and the denominator of Eq. 1, so f is unchanged."""
    xc, x = _umbrella_samples_device(K, N_k, seed, kappa, grid_points, device)
    a = (0.5 * kappa) * xc * xc
    b = -kappa * xc
    return a.contiguous(), b.contiguous(), x.contiguous(), np.full(K, N_k, dtype=np.int64)

