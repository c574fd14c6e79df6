"""Store-free factorised contexts (MIXED): u_kn = a_k + b_k phi_n, the
paper's setting (Sec. II: u_ip = beta_i E_p), solved without any K x N
store. Binned levels are generated from a, b and the bin means of phi (a
binned level of factorised u is factorised at the bin means: the oracle's
pin of the bin-mean reading); the unbinned passes and the Hessian generate
u from phi. Results against the oracle's MBAR root at the mixed tolerance
(1e-4 kT); the Hessian at the tensor-core tolerance (2e-3 of max|H|)."""
import json
import os

import numpy as np
import pytest

import oracle as O
from paper_2609_03541_b300 import mbar as M
from paper_2609_03541_b300 import workloads as W

pytestmark = pytest.mark.gpu

HERE = os.path.dirname(os.path.abspath(__file__))


def _refs():
    with open(os.path.join(HERE, "golden", "solve_refs.json")) as fh:
        return {c["name"]: c for c in json.load(fh)["cases"]}


def _tempering(K, N_k, seed, s2=2000.0):
    p = W.parallel_tempering(K=K, N_k=N_k, sigma2=s2, seed=seed, materialize=False)
    return np.zeros(K), p.meta["b"], p.phi, p.N_k


def _gaussian(M_, N_0, seed):
    p = W.gaussian_overlap(M=M_, N_0=N_0, seed=seed)
    return np.zeros(M_), p.meta["beta"], p.phi, p.N_k


def _alchemical(K, N_k, seed):
    lam, u0, du, Nk = W.alchemical_factors(K=K, N_k=N_k, seed=seed)
    # the per-sample u0_n is a shift that leaves f unchanged
    return np.zeros(K), lam, du, Nk


CASES = {
    "tempering_K6": lambda: _tempering(6, 3000, 2, s2=40.0),
    "tempering_K20": lambda: _tempering(20, 2000, 5),
    "gaussian_M12": lambda: _gaussian(12, 2000, 4),
    "alchemical_K40": lambda: _alchemical(40, 300, 3),
    "alchemical_K130": lambda: _alchemical(130, 100, 8),
    # K > 512: the tensor-core Hessian in clusters of 6 CTAs, two launches
    "alchemical_K700": lambda: _alchemical(700, 12, 9),
}


@pytest.mark.parametrize("where", ["host", "device"])
@pytest.mark.parametrize("name", list(CASES))
def test_factorised_mixed_solve_matches_the_oracle(name, where):
    a, b, phi, Nk = CASES[name]()
    f_ref = O.solve_mbar(O.factorised_u(a, b, phi), Nk)
    if where == "device":
        import torch
        td = lambda x: torch.from_numpy(np.ascontiguousarray(x, dtype=np.float64)).cuda()
        ctx = M.Context.factorised(td(a), td(b), td(phi), Nk, M.MBAR_MIXED)
    else:
        ctx = M.Context.factorised(a, b, phi, Nk, M.MBAR_MIXED)
    with ctx:
        rep = ctx.solve().as_dict()
        f = ctx.free_energies()
    assert np.max(np.abs(f - f_ref)) < 1e-4, rep


@pytest.mark.parametrize("name", ["alchemical_K500", "tempering_K50"])
def test_factorised_bench_shapes_match_the_stored_roots(name):
    """The default benchmark's shapes in factorised form against the
    oracle's roots of the dense problems (tests/golden/solve_refs.json)."""
    case = _refs()[name]
    if name == "alchemical_K500":
        a, b, phi, Nk = _alchemical(**case["args"])
    else:
        p = W.parallel_tempering(materialize=False, **case["args"])
        a, b, phi, Nk = np.zeros(p.K), p.meta["b"], p.phi, p.N_k
    with M.Context.factorised(a, b, phi, Nk, M.MBAR_MIXED) as ctx:
        K, N = len(a), len(phi)
        assert ctx.device_bytes() < K * N * 4 // 2     # no K x N store
        rep = ctx.solve().as_dict()
        f = ctx.free_energies()
    assert np.max(np.abs(f - np.asarray(case["f"]))) < 1e-4, rep


# K = 600..1024 take clusters of 5..8 CTAs; above K = 640 the tile distances
# are split over two launches (at K = 700 half the CTAs form no tile in the
# second one, at K = 800 every CTA forms one, at K = 1024 two or one)
@pytest.mark.parametrize("K,N_k", [(20, 300), (150, 40), (300, 30), (500, 16), (600, 10), (700, 8), (800, 8),
                                   (1024, 6)])
def test_factorised_hessian_matches_the_oracle(K, N_k):
    a, b, phi, Nk = _alchemical(K, N_k, seed=K)
    u = O.factorised_u(a, b, phi)
    f = O.gauge(O.sci_step(u, np.zeros(K), Nk))
    with M.Context.factorised(a, b, phi, Nk, M.MBAR_MIXED) as ctx:
        Hs = ctx.hessian(f)
    H_ref = O.mbar_hessian(u, f, Nk)
    scale = np.max(np.abs(H_ref))
    assert np.max(np.abs(Hs - H_ref)) < 2e-3 * scale
    assert np.max(np.abs(Hs - Hs.T)) == 0.0


def test_factorised_unbinned_step_and_logden():
    """One unbinned Eq. 1 step on the factorised data (exact-split pass):
    f, gradient and logden (FP64, original sample order) against the
    oracle; the bound is a few FP32 ulps of the exponent's magnitude."""
    a, b, phi, Nk = _tempering(20, 2000, 7)
    u = O.factorised_u(a, b, phi)
    g0 = np.random.default_rng(1)
    f = O.gauge(-(b ** 2) * 2000.0 / 2 + g0.uniform(-1, 1, len(b)))
    with M.Context.factorised(a, b, phi, Nk, M.MBAR_MIXED) as ctx:
        fo, g, s, ld = ctx.sci_step(f, want_logden=True)
    ld_ref = O.log_denominator(u, f, Nk)
    X = float(np.max(np.abs(ld_ref)))
    tol = 1e-6 + 8.0 * X * 2.0 ** -24
    assert np.max(np.abs(ld - ld_ref)) < tol
    assert np.max(np.abs(fo - O.gauge(O.sci_step(u, f, Nk)))) < 10 * tol
    assert np.max(np.abs(g - O.mbar_gradient(u, f, Nk)) / Nk) < 10 * tol


def test_factorised_context_rejects_a_new_coordinate():
    a, b, phi, Nk = _tempering(6, 300, 3, s2=40.0)
    with M.Context.factorised(a, b, phi, Nk, M.MBAR_MIXED) as ctx:
        with pytest.raises(M.MbarError):
            ctx.set_coordinate(phi)


def _umbrella_factorised(K, N_k, seed):
    """The umbrella windows of workloads.umbrella in factorised form: the
    per-sample terms U(x) + kappa x^2 / 2 cancel in Eq. 1 and are dropped."""
    p = W.umbrella(K=K, N_k=N_k, seed=seed, grid_points=1 << 13)
    xc, kappa = p.meta["centres"], p.meta["kappa"]
    return 0.5 * kappa * xc * xc, -kappa * xc, p.phi, p.N_k


@pytest.mark.parametrize("N_k,seed", [(1546, 504), (10664, 850)])
def test_factorised_poorly_overlapping_windows_reach_the_oracle(N_k, seed):
    """Four windows 1.0 apart: the binned levels leave f several kT from
    the root and full Newton steps overshoot; backtracking along the Newton
    direction must still reach the MBAR root."""
    a, b, phi, Nk = _umbrella_factorised(4, N_k, seed)
    f_ref = O.solve_mbar(O.factorised_u(a, b, phi), Nk)
    with M.Context.factorised(a, b, phi, Nk, M.MBAR_MIXED) as ctx:
        rep = ctx.solve().as_dict()
        f = ctx.free_energies()
    assert np.max(np.abs(f - f_ref)) < 1e-4, rep


@pytest.mark.parametrize("M_,N_0,seed", [(12, 200, 4), (30, 100, 1)])
def test_factorised_covariance_matches_the_oracle(M_, N_0, seed):
    """mbar_covariance of a store-free context (its Hessian from FP16 P~
    formed from phi at every K) on Sec. IV ladders: the asymptotic
    covariance within 2e-3 of the oracle's weight-matrix form (scaled by
    sd_i sd_j), so the 5-sigma checks against the analytic f divide by the
    right standard deviations."""
    a, b, phi, Nk = _gaussian(M_, N_0, seed)
    with M.Context.factorised(a, b, phi, Nk, M.MBAR_MIXED) as ctx:
        ctx.solve()
        f = ctx.free_energies()
        C = ctx.covariance()
    u = O.factorised_u(a, b, phi)
    f_ref = O.solve_mbar(u, Nk)
    C_ref = O.mbar_covariance(u, f_ref, Nk)
    scale = np.sqrt(np.outer(np.diag(C_ref), np.diag(C_ref)))[1:, 1:]
    assert np.max(np.abs(f - f_ref)) < 1e-4
    assert np.max(np.abs(C[1:, 1:] - C_ref[1:, 1:]) / scale) < 2e-3


@pytest.mark.parametrize("M_,N_0", [(309, 396), (552, 760)])
def test_factorised_long_replica_ladder_matches_the_analytic_free_energies(M_, N_0):
    """Sec. IV replicas (80 % neighbour overlap) up to beta ~ 280: u reaches
    ~1e5 kT, the binned levels end thousands of kT from the root, and the
    root is checked against f_k = -beta_k^2 / 2 + c within 5 asymptotic
    standard deviations (the oracle's solve takes too long at these sizes)."""
    a, b, phi, Nk = _gaussian(M_, N_0, seed=M_)
    with M.Context.factorised(a, b, phi, Nk, M.MBAR_MIXED) as ctx:
        rep = ctx.solve().as_dict()
        f = ctx.free_energies()
        C = ctx.covariance()
    exact = -(b * b - b[0] * b[0]) / 2.0
    sd = np.sqrt(np.maximum(np.diag(C), 0.0))
    z = np.abs(f - exact)[1:] / sd[1:]
    assert np.max(z) < 5.0, (float(np.max(z)), rep)

