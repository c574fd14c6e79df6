"""Tensor-core (tcgen05) Hessian against the oracle and the CUDA-core path.

Tolerance: FP16 operands round each P~ to 2^-11 relative; the overlap sums
accumulate in FP32 and reduce in FP64, so entries agree to ~1e-3 relative;
the test allows 2e-3 of max|H|. The Laplacian structure (symmetry, zero row
sums) is exact by construction.
"""
import numpy as np
import pytest

import oracle as O
from paper_2609_03541_b300 import mbar as M
from paper_2609_03541_b300 import workloads as W

pytestmark = pytest.mark.gpu


def _problem(K, N, seed):
    g = np.random.default_rng(seed)
    Nk = np.full(K, N // K, dtype=np.int64)
    Nk[: N - Nk.sum()] += 1
    # neighbouring states overlap: state k prefers samples near k/K
    x = g.uniform(0, 1, size=N)
    centres = np.linspace(0, 1, K)
    u = 0.5 * (K * 0.8) ** 2 * (x[None, :] - centres[:, None]) ** 2
    return u, Nk


@pytest.fixture(autouse=True)
def _tensor_cores():
    M.set_hessian_path(2)
    yield
    M.set_hessian_path(0)


# path 2: tensor cores (thread-block-cluster kernel for FP32 data with
# K <= 512, one cluster CTA per 128-row tile); path 3: tensor cores with the
# per-item kernel only
@pytest.mark.parametrize("path", [2, 3])
@pytest.mark.parametrize("prec", ["mixed", "fp64"])
@pytest.mark.parametrize("K,N", [(64, 3000), (128, 4099), (200, 5001), (300, 70001), (500, 6000), (512, 20000),
                                 (1000, 9001)])
def test_tc_hessian_matches_oracle(prec, K, N, path):
    M.set_hessian_path(path)
    u, Nk = _problem(K, N, seed=K)
    f = O.gauge(O.sci_step(u, np.zeros(K), Nk))
    ctx = M.Context(u, Nk, M.MBAR_MIXED if prec == "mixed" else M.MBAR_FP64)
    Hs = ctx.hessian(f)
    ctx.close()
    H_ref = O.mbar_hessian(u, f, Nk)
    scale = np.max(np.abs(H_ref))
    assert np.max(np.abs(Hs - H_ref)) < 2e-3 * scale
    assert np.max(np.abs(Hs - Hs.T)) == 0.0
    assert np.max(np.abs(Hs.sum(axis=1))) < 1e-9 * scale


def test_tc_hessian_binned_counts():
    p = W.umbrella(K=80, N_k=400, seed=3, grid_points=1 << 12)
    f = O.gauge(O.sci_step(p.u_kn, np.zeros(80), p.N_k))
    ctx = M.Context(p.u_kn, p.N_k, M.MBAR_FP64)
    ctx.set_coordinate(p.phi)
    ctx.bin(0.01)
    Hs = ctx.hessian(f)
    ctx.close()
    hist = O.histogram(p.phi, 0.01)
    ub = O.binned_u(p.u_kn, hist)
    H_ref = O.mbar_hessian(ub, f, p.N_k, hist.H)
    assert np.max(np.abs(Hs - H_ref)) < 2e-3 * np.max(np.abs(H_ref))


def test_tc_and_cuda_core_paths_agree():
    u, Nk = _problem(150, 4000, seed=5)
    f = np.zeros(150)
    ctx = M.Context(u, Nk, M.MBAR_MIXED)
    H_tc = ctx.hessian(f)
    M.set_hessian_path(1)
    H_cc = ctx.hessian(f)
    ctx.close()
    assert np.max(np.abs(H_tc - H_cc)) < 2e-3 * np.max(np.abs(H_cc))


@pytest.mark.parametrize("K", [90, 260, 500])
def test_tc_cluster_hessian_binned_counts_mixed(K):
    """Binned counts H_p (sqrt(H_p) scaling of P~) on the cluster kernel."""
    p = W.umbrella(K=K, N_k=200, seed=K, grid_points=1 << 12)
    f = O.gauge(O.sci_step(p.u_kn, np.zeros(K), p.N_k))
    ctx = M.Context(p.u_kn, p.N_k, M.MBAR_MIXED)
    ctx.set_coordinate(p.phi)
    ctx.bin(0.003)
    Hs = ctx.hessian(f)
    ctx.close()
    hist = O.histogram(p.phi, 0.003)
    ub = O.binned_u(p.u_kn, hist)
    H_ref = O.mbar_hessian(ub, f, p.N_k, hist.H)
    assert np.max(np.abs(Hs - H_ref)) < 2e-3 * np.max(np.abs(H_ref))


@pytest.mark.parametrize("K,N", [(64, 64), (100, 100), (257, 300), (400, 450)])
def test_tc_cluster_and_item_kernels_agree_on_few_samples(K, N):
    """One to seven 64-sample chunks in all, the last one partial."""
    u, Nk = _problem(K, N, seed=N)
    f = np.zeros(K)
    ctx = M.Context(u, Nk, M.MBAR_MIXED)
    H2 = ctx.hessian(f)
    M.set_hessian_path(3)
    H3 = ctx.hessian(f)
    ctx.close()
    H_ref = O.mbar_hessian(u, f, Nk)
    scale = np.max(np.abs(H_ref))
    assert np.max(np.abs(H2 - H_ref)) < 2e-3 * scale
    assert np.max(np.abs(H2 - H3)) < 2e-3 * scale
