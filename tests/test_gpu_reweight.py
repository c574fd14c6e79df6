"""Reweighting to a target state (Eqs. 5-6) and the weighted 2-D histogram
of Fig. 1, against the oracle."""
import numpy as np
import pytest

import oracle as O
from paper_2609_03541_b300 import mbar as M
from paper_2609_03541_b300 import workloads as W

pytestmark = pytest.mark.gpu


def _solved(p, prec, phi=None):
    ctx = M.Context(p.u_kn, p.N_k, prec)
    if phi is not None:
        ctx.set_coordinate(phi)
    ctx.solve()
    return ctx, ctx.free_energies()


@pytest.mark.parametrize("prec,rtol", [(M.MBAR_FP64, 1e-10), (M.MBAR_MIXED, 2e-5)])
def test_reweight_matches_the_oracle(prec, rtol):
    p = W.harmonic(K=8, d=3, N_k=1000, seed=0)
    ctx, f = _solved(p, prec)
    g = np.random.default_rng(1)
    u0 = 0.5 * 2.5 * np.sum((p.meta["x"] - 1.0) ** 2, axis=1) + g.normal(0, 0.01, size=p.N)
    pw, logc = ctx.reweight(u0)
    ctx.close()
    ref = O.reweight(u0, p.u_kn, f, p.N_k)
    big = ref > 1e-3 * ref.max()
    assert np.max(np.abs(pw[big] - ref[big]) / ref[big]) < rtol
    assert np.max(np.abs(pw - ref)) < rtol * ref.max()
    assert abs(pw.sum() - 1.0) < 1e-10


def test_reweight_to_a_sampled_state_gives_its_free_energy():
    """At the MBAR solution sum_n exp(f_k - u_kn) / sum_m N_m exp(f_m - u_mn) = 1,
    so reweighting to state k has C = exp(-f_k)."""
    p = W.harmonic(K=6, d=2, N_k=800, seed=3)
    ctx, f = _solved(p, M.MBAR_FP64)
    for k in (0, 2, 5):
        _, logc = ctx.reweight(p.u_kn[k])
        assert abs(logc + f[k]) < 1e-8
    ctx.close()


def test_reweight_keeps_the_callers_sample_order_after_sorting():
    p = W.alchemical(K=20, N_k=200, seed=5)
    ctx, f = _solved(p, M.MBAR_MIXED, phi=p.phi)     # columns are stored in phi order
    u0 = p.u_kn[7]
    pw, _ = ctx.reweight(u0)
    ctx.close()
    ref = O.reweight(u0, p.u_kn, f, p.N_k)
    big = ref > 1e-3 * ref.max()
    assert np.max(np.abs(pw[big] - ref[big]) / ref[big]) < 2e-5


def test_weighted_histogram2d_matches_a_plain_accumulation():
    p = W.harmonic(K=5, d=2, N_k=2000, seed=8)
    ctx, f = _solved(p, M.MBAR_FP64)
    x, y = p.meta["x"][:, 0], p.meta["x"][:, 1]
    u0 = 0.5 * 3.0 * ((x - 1.0) ** 2 + (y - 1.0) ** 2)
    pw, _ = ctx.reweight(u0)
    x0, dx, nx, y0, dy, ny = -0.5, 0.05, 60, -0.25, 0.1, 30
    h = ctx.weighted_histogram2d(x, y, x0, dx, nx, y0, dy, ny)
    ctx.close()
    ix = np.floor((x - x0) / dx)
    iy = np.floor((y - y0) / dy)
    keep = (ix >= 0) & (ix < nx) & (iy >= 0) & (iy < ny)
    ref = np.zeros((nx, ny))
    np.add.at(ref, (ix[keep].astype(int), iy[keep].astype(int)), O.reweight(u0, p.u_kn, f, p.N_k)[keep])
    assert np.max(np.abs(h - ref)) < 1e-10 * ref.max()
    assert abs(h.sum() - pw[keep].sum()) < 1e-12


def test_histogram_before_any_reweight_is_a_state_error():
    p = W.harmonic(K=3, d=1, N_k=100, seed=0)
    ctx = M.Context(p.u_kn, p.N_k, M.MBAR_FP64)
    with pytest.raises(M.MbarError) as e:
        ctx.weighted_histogram2d(np.zeros(p.N), np.zeros(p.N), 0.0, 1.0, 2, 0.0, 1.0, 2)
    assert e.value.name == "MBAR_ESTATE"
    with pytest.raises(M.MbarError) as e:
        ctx.reweight(np.full(p.N, np.nan))
    assert e.value.name == "MBAR_EINVAL"
    ctx.close()
