"""Parity of the CUDA path (through the C ABI) with the CPU oracle.

Tolerances (from the arithmetic of each path):
  * bin keys / counts / width search: bit-exact (integer work, binary64
    bin index with the same rounding on both sides);
  * FP64 path: 1e-9 kT per step and 1e-8 kT for the solve (sums of a few
    thousand binary64 terms in another order differ by ~1e-14 relative);
  * MIXED path: 1e-4 kT (FP32 exp with row sums accumulated in FP64);
  * Hessian: 1e-4 of max|H| on the CUDA-core path (FP32 products, FP64
    reduction across slices), 2e-3 on the tensor-core path (FP16 operands).
"""
import numpy as np
import pytest

import oracle as O
from paper_2609_03541_b300 import mbar as M
from paper_2609_03541_b300 import workloads as W
from shapes import LANE_SHAPE_CASES

pytestmark = pytest.mark.gpu

PREC = {"fp64": M.MBAR_FP64, "mixed": M.MBAR_MIXED}
F_TOL = {"fp64": 1e-9, "mixed": 1e-4}
SOLVE_TOL = {"fp64": 1e-8, "mixed": 1e-4}


def rand_problem(K, N, seed=0, spread=3.0, offset=0.0):
    g = np.random.default_rng(seed)
    base = np.full(K, N // K, dtype=np.int64)
    base[: N - base.sum()] += 1
    u = spread * g.standard_normal((K, N)) + g.uniform(-2, 2, size=(K, 1)) + offset * g.standard_normal((1, N))
    return u, base


def rand_f(K, seed=1):
    g = np.random.default_rng(seed)
    f = g.uniform(-1.0, 1.0, size=K)
    f[0] = 0.0
    return f


# ---------------------------------------------------------------------------
# b1/b2: one SCI step, gradient and logden, unbinned
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("prec", ["fp64", "mixed"])
@pytest.mark.parametrize("K,N", [(1, 50), (2, 33), (3, 1000), (8, 8013), (64, 4099), (100, 3333), (200, 2111),
                                 (257, 3001), (500, 2053), (513, 1500), (1000, 1031)])
def test_sci_step_unbinned(prec, K, N):
    u, Nk = rand_problem(K, N, seed=K + N, offset=200.0)
    f = rand_f(K)
    ctx = M.Context(u, Nk, PREC[prec])
    fo, g, s, ld = ctx.sci_step(f, want_logden=True)
    ctx.close()
    fo_ref = O.gauge(O.sci_step(u, f, Nk))
    g_ref = O.mbar_gradient(u, f, Nk)
    ld_ref = O.log_denominator(u, f, Nk)
    s_ref = O.relative_step(fo_ref, f)
    tol = F_TOL[prec]
    assert np.max(np.abs(fo - fo_ref)) < tol
    assert np.max(np.abs(g - g_ref) / Nk) < tol
    assert np.max(np.abs(ld - ld_ref)) < tol * 10
    if K > 1:
        assert abs(s - s_ref) <= tol * max(1.0, abs(s_ref)) * 10


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_sci_step_first_step_from_zero(prec):
    p = W.harmonic(K=8, N_k=1000, seed=0)
    ctx = M.Context(p.u_kn, p.N_k, PREC[prec])
    fo, g, s = ctx.sci_step(np.zeros(8))
    ctx.close()
    assert s == np.inf
    assert np.max(np.abs(fo - O.gauge(O.sci_step(p.u_kn, np.zeros(8), p.N_k)))) < F_TOL[prec]


# ---------------------------------------------------------------------------
# a1-a4: binning
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("prec", ["fp64", "mixed"])
@pytest.mark.parametrize("h", [0.5, 0.1, 0.013, 1e-3, 1e-6])
def test_histogram_bit_exact(prec, h):
    p = W.umbrella(K=6, N_k=700, seed=3, grid_points=1 << 12)
    phi = p.phi.copy()
    phi[::97] = np.round(phi[::97], 1)        # ties and values on bin edges
    ctx = M.Context(p.u_kn, p.N_k, PREC[prec])
    ctx.set_coordinate(phi)
    nb = ctx.bin(h)
    keys, H, ub = ctx.get_bins(nb)
    hist = O.histogram(phi, h)
    assert nb == hist.H.shape[0]
    assert np.array_equal(keys, hist.keys)
    assert np.array_equal(H, hist.H)
    ub_ref = O.binned_u(p.u_kn, hist)
    if prec == "fp64":
        assert np.max(np.abs(ub - ub_ref)) < 1e-11
    else:  # stored with a per-bin shift; state differences are exact up to FP32
        d = (ub - ub[0]) - (ub_ref - ub_ref[0])
        assert np.max(np.abs(d)) < 1e-4 * max(1.0, np.max(np.abs(ub_ref - ub_ref[0])))
    ctx.close()


def test_histogram_golden_edges(golden_dir):
    import json, os
    spec = json.load(open(os.path.join(golden_dir, "binning_cases.json")))
    for case in spec["cases"]:
        phi = np.array(case["phi"])
        N = phi.shape[0]
        u = np.vstack([phi, 2 * phi])
        ctx = M.Context(u, np.array([N - N // 2, N // 2]) if N > 1 else np.array([1, 0]), M.MBAR_FP64) if N > 1 else None
        if ctx is None:
            continue
        ctx.set_coordinate(phi)
        nb = ctx.bin(case["w"])
        keys, H, _ = ctx.get_bins(nb)
        assert keys.tolist() == case["nonempty_keys"], case["name"]
        assert H.tolist() == case["H"], case["name"]
        ctx.close()


@pytest.mark.parametrize("n", [2, 10, 100, 1000, 5000])
def test_width_search_bit_exact(n):
    p = W.gaussian_overlap(M=6, N_0=1500, seed=2)
    ctx = M.Context(p.u_kn, p.N_k, M.MBAR_FP64)
    ctx.set_coordinate(p.phi)
    w, nb = ctx.bin_count(n)
    w_ref = O.width_for_bins(p.phi, n)
    assert w == w_ref
    assert nb == O.nonempty_bins(p.phi, w_ref)
    ctx.close()


def test_width_search_unreachable_gives_unbinned():
    p = W.harmonic(K=3, N_k=50, seed=1)
    ctx = M.Context(p.u_kn, p.N_k, M.MBAR_FP64)
    w, nb = ctx.bin_count(10**6)
    assert w == 0.0 and nb == p.N
    ctx.close()


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_binned_sci_step(prec):
    p = W.umbrella(K=10, N_k=900, seed=5, grid_points=1 << 12)
    f = rand_f(10, seed=4)
    ctx = M.Context(p.u_kn, p.N_k, PREC[prec])
    ctx.set_coordinate(p.phi)
    for h in (0.2, 0.02, 0.002):
        nb = ctx.bin(h)
        fo, g, s = ctx.sci_step(f)
        hist = O.histogram(p.phi, h)
        ub = O.binned_u(p.u_kn, hist)
        fo_ref = O.gauge(O.sci_step(ub, f, p.N_k, hist.H))
        g_ref = O.mbar_gradient(ub, f, p.N_k, hist.H)
        assert nb == hist.H.shape[0]
        assert np.max(np.abs(fo - fo_ref)) < F_TOL[prec]
        assert np.max(np.abs(g - g_ref) / p.N_k) < F_TOL[prec]
    ctx.close()


# ---------------------------------------------------------------------------
# c1/c2: Hessian and Newton step
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("path,tol", [(1, 1e-4), (2, 2e-3)])
@pytest.mark.parametrize("prec", ["fp64", "mixed"])
@pytest.mark.parametrize("K,N", [(2, 500), (8, 8000), (70, 3001), (200, 2500)])
def test_hessian(prec, K, N, path, tol):
    u, Nk = rand_problem(K, N, seed=3 * K, spread=1.5)
    f = O.solve_mbar(u, Nk, tol=1e-10) if K <= 8 else rand_f(K, seed=2) * 0.1
    M.set_hessian_path(path)   # 1: CUDA cores (FP32), 2: tensor cores (FP16 operands)
    try:
        ctx = M.Context(u, Nk, PREC[prec])
        Hs = ctx.hessian(f)
        ctx.close()
    finally:
        M.set_hessian_path(0)
    H_ref = O.mbar_hessian(u, f, Nk)
    scale = np.max(np.abs(H_ref))
    assert np.max(np.abs(Hs - H_ref)) < tol * scale
    assert np.max(np.abs(Hs - Hs.T)) < 1e-9 * scale
    assert np.max(np.abs(Hs.sum(axis=1))) < 1e-9 * scale


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_newton_step(prec):
    p = W.harmonic(K=8, N_k=1000, seed=0)
    f0 = O.gauge(O.sci_step(p.u_kn, np.zeros(8), p.N_k))
    ctx = M.Context(p.u_kn, p.N_k, PREC[prec])
    fo, step = ctx.newton_step(f0)
    ctx.close()
    d = O.newton_direction(O.mbar_hessian(p.u_kn, f0, p.N_k), O.mbar_gradient(p.u_kn, f0, p.N_k))
    assert np.max(np.abs(fo - (f0 + d))) < (1e-6 if prec == "fp64" else 1e-3) * max(1, np.max(np.abs(d)))
    assert abs(step - np.max(np.abs(d))) < 1e-3 * np.max(np.abs(d))


# ---------------------------------------------------------------------------
# full solves
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_solve_harmonic_plain_and_binned(prec):
    p = W.harmonic(K=8, d=3, N_k=1000, seed=0)
    f_ref = O.solve_mbar(p.u_kn, p.N_k)
    for use_binning in (0, 1):
        o = M.default_opts(PREC[prec], use_binning=use_binning)
        ctx = M.Context(p.u_kn, p.N_k, PREC[prec], opts=o)
        rep = ctx.solve()
        f = ctx.free_energies()
        ctx.close()
        assert np.max(np.abs(f - f_ref)) < SOLVE_TOL[prec], (use_binning, rep.as_dict())
        assert f[0] == 0.0


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_solve_umbrella_width_schedule(prec):
    p = W.umbrella(K=16, N_k=1000, seed=1, grid_points=1 << 13)
    opts = O.BUOptions(h0=0.1)
    tr = []
    f_ref = O.bu_mbar(p.u_kn, p.N_k, phi=p.phi, opts=opts, trace=tr)
    o = M.default_opts(PREC[prec], h0=0.1)
    ctx = M.Context(p.u_kn, p.N_k, PREC[prec], opts=o)
    ctx.set_coordinate(p.phi)
    rep = ctx.solve()
    f = ctx.free_energies()
    ctx.close()
    assert np.max(np.abs(f - f_ref)) < SOLVE_TOL[prec], rep.as_dict()
    n_first = sum(1 for t in tr if t[0] == "phase1")
    if prec == "fp64":
        assert rep.iters_first_loop == n_first


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_solve_gaussian_overlap_count_schedule(prec):
    p = W.gaussian_overlap(M=12, N_0=2000, seed=4)
    f_ref = O.solve_mbar(p.u_kn, p.N_k)
    ctx = M.Context(p.u_kn, p.N_k, PREC[prec])
    ctx.set_coordinate(p.phi)
    rep = ctx.solve()
    f = ctx.free_energies()
    ctx.close()
    assert np.max(np.abs(f - f_ref)) < SOLVE_TOL[prec], rep.as_dict()
    assert rep.n_rebins >= 2


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_solve_alchemical_small(prec):
    p = W.alchemical(K=20, N_k=300, seed=2)
    f_ref = O.bu_mbar(p.u_kn, p.N_k, phi=p.phi)
    ctx = M.Context(p.u_kn, p.N_k, PREC[prec])
    ctx.set_coordinate(p.phi)
    rep = ctx.solve()
    f = ctx.free_energies()
    ctx.close()
    assert np.max(np.abs(f - f_ref)) < SOLVE_TOL[prec], rep.as_dict()


def test_solve_invariances_on_device():
    p = W.harmonic(K=5, N_k=400, seed=7)
    g = np.random.default_rng(0)
    c_n = g.normal(size=p.N) * 100
    perm = g.permutation(p.N)
    out = []
    for u in (p.u_kn, p.u_kn + c_n[None, :], p.u_kn[:, perm]):
        ctx = M.Context(u, p.N_k, M.MBAR_FP64)
        ctx.solve()
        out.append(ctx.free_energies())
        ctx.close()
    assert np.max(np.abs(out[1] - out[0])) < 1e-9
    assert np.max(np.abs(out[2] - out[0])) < 1e-9


def test_single_state_and_two_sample_closed_form():
    ctx = M.Context(np.array([[0.3, -1.0, 2.0]]), np.array([3]), M.MBAR_FP64)
    ctx.solve()
    assert ctx.free_energies().tolist() == [0.0]
    ctx.close()
    u = np.array([[0.0, 0.0], [1.3, -0.4]])
    ctx = M.Context(u, np.array([1, 1]), M.MBAR_FP64, opts=M.default_opts(M.MBAR_FP64, use_binning=0))
    ctx.solve()
    f = ctx.free_energies()
    ctx.close()
    assert abs(f[1] - 0.5 * (1.3 - 0.4)) < 1e-10


@pytest.mark.parametrize("K,N,k,n,bad", [(500, 4133, 321, 2777, np.nan), (500, 4133, 499, 4132, -np.inf),
                                          (37, 100, 0, 0, np.inf), (700, 300, 650, 17, np.nan)])
def test_nonfinite_entry_anywhere_is_rejected(K, N, k, n, bad):
    """One non-finite u_kn anywhere (any row residue of the staging's
    per-sample minimum, the last entry, the row-major fallback above
    K = 512) makes a mixed-precision context fail with MBAR_EINVAL."""
    u, Nk = rand_problem(K, N, seed=3)
    u[k, n] = bad
    with pytest.raises(M.MbarError) as e:
        M.Context(u, Nk, M.MBAR_MIXED)
    assert e.value.name == "MBAR_EINVAL"


def test_bad_inputs_are_rejected():
    u = np.ones((2, 4))
    u[1, 2] = np.nan
    with pytest.raises(M.MbarError) as e:
        M.Context(u, np.array([2, 2]), M.MBAR_MIXED)
    assert e.value.name == "MBAR_EINVAL"
    ctx = M.Context(np.ones((2, 4)), np.array([2, 2]), M.MBAR_FP64)
    with pytest.raises(M.MbarError):
        ctx.bin(-1.0)
    with pytest.raises(M.MbarError):
        ctx.get_bins(1)          # unbinned level
    with pytest.raises(M.MbarError):
        ctx.set_coordinate(np.array([0.0, np.inf, 1.0, 2.0]))
    ctx.close()


# ---------------------------------------------------------------------------
# stateless device-level pass
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("dtype", ["float32", "float64"])
def test_lse_pass_stateless(dtype):
    import torch
    K, N = 37, 5001
    u, Nk = rand_problem(K, N, seed=9)
    f = rand_f(K, seed=3)
    dev = torch.device("cuda")
    tdt = torch.float32 if dtype == "float32" else torch.float64
    ld = (N + 31) // 32 * 32
    v = torch.zeros((K, ld), dtype=tdt, device=dev)
    v[:, :N] = torch.from_numpy(u).to(dev, tdt)
    vv = v[:, :N]
    ft = torch.from_numpy(f).to(dev)
    lN = torch.from_numpy(np.log(Nk.astype(np.float64))).to(dev)
    Q = torch.empty(K, dtype=torch.float64, device=dev)
    logden = torch.empty(N, dtype=tdt, device=dev)
    nbytes = M.lse_scratch_bytes(K, N, v.element_size())
    scratch = torch.zeros(nbytes, dtype=torch.uint8, device=dev)
    for _ in range(2):
        M.lse_pass(vv, ft, lN, Q, logden=logden, scratch=scratch)
    torch.cuda.synchronize()
    Wk = O.mbar_weights(u, f, Nk)
    Q_ref = Nk * Wk.sum(axis=1)
    tol = 1e-10 if dtype == "float64" else 1e-5
    assert np.max(np.abs(Q.cpu().numpy() - Q_ref) / Q_ref) < tol
    assert np.max(np.abs(logden.cpu().numpy().astype(np.float64) - O.log_denominator(u, f, Nk))) < tol * 100


@pytest.mark.parametrize("K,N", LANE_SHAPE_CASES)
@pytest.mark.parametrize("counts", [False, True])
def test_lse_pass_sample_major(K, N, counts):
    """The sample-major FP32 pass (the layout of MIXED's unbinned passes):
    every lane-group shape, ragged last stages, per-sample counts H, and
    padding entries that must get weight 0."""
    import torch
    u, Nk = rand_problem(K, N, seed=K + 7 * N)
    f = rand_f(K, seed=5)
    dev = torch.device("cuda")
    Kp = (K + 3) // 4 * 4
    v = torch.full((N, Kp), 7.0, dtype=torch.float32, device=dev)   # padding: finite, weight 0
    v[:, :K] = torch.from_numpy(np.ascontiguousarray(u.T)).to(dev, torch.float32)
    H = None
    Hn = np.ones(N)
    if counts:
        Hn = 1.0 + (np.arange(N) % 5)
        H = torch.from_numpy(Hn.astype(np.int32)).to(dev)
    ft = torch.from_numpy(f).to(dev)
    lN = torch.from_numpy(np.log(Nk.astype(np.float64))).to(dev)
    Q = torch.empty(K, dtype=torch.float64, device=dev)
    logden = torch.empty(N, dtype=torch.float32, device=dev)
    scratch = torch.zeros(M.lse_samples_scratch_bytes(K, N), dtype=torch.uint8, device=dev)
    for _ in range(2):
        M.lse_pass_samples(v, K, ft, lN, Q, H=H, logden=logden, scratch=scratch)
    torch.cuda.synchronize()
    u32 = u.astype(np.float32).astype(np.float64)        # the data as stored
    ld_ref = O.log_denominator(u32, f, Nk)
    Q_ref = Nk * (O.mbar_weights(u32, f, Nk) * Hn[None, :]).sum(axis=1)
    Qg = Q.cpu().numpy()
    occupied = Nk > 0                                  # N // K < 1 leaves states without samples
    assert np.max(np.abs(Qg[occupied] - Q_ref[occupied]) / Q_ref[occupied]) < 1e-5
    assert np.all(Qg[~occupied] == 0.0)
    assert np.max(np.abs(logden.cpu().numpy().astype(np.float64) - ld_ref)) < 1e-4


@pytest.mark.parametrize("K,N", LANE_SHAPE_CASES)
@pytest.mark.parametrize("regime", ["tempering", "small"])
@pytest.mark.parametrize("counts", [False, True])
def test_lse_pass_factorised(K, N, regime, counts):
    """u_kp = a_k + b_k phi_p generated on the device (mbar_lse_pass_factorised)
    against the oracle on the materialised u: every lane-group shape, ragged
    chunks and counts. "tempering": b over 298..600 K, energies of a Gaussian
    density of states (variance 2000 kT^2), so u and logden are ~1e3 kT;
    "small": O(1) potentials. The exponent is FP32 at its own magnitude
    X = max |logden|: the bound is a few FP32 ulps of X."""
    import torch
    g = np.random.default_rng(K * 31 + N)
    state = np.arange(N) % K
    Nk = np.bincount(state, minlength=K).astype(np.int64)
    if regime == "tempering":
        s2 = 2000.0
        b = 1.0 / np.exp(np.linspace(0.0, np.log(600.0 / 298.0), K))
        phi = -b[state] * s2 + np.sqrt(s2) * g.standard_normal(N)
        a = 5.0 * g.standard_normal(K)
        f = -(b**2) * s2 / 2 + a
    else:
        b = g.uniform(0.5, 1.5, size=K)
        phi = 3.0 * g.standard_normal(N)
        a = g.standard_normal(K)
        f = 0.3 * g.standard_normal(K)
    Hn = np.ones(N)
    dev = torch.device("cuda")
    H = None
    if counts:
        Hn = 1.0 + (np.arange(N) % 5)
        H = torch.from_numpy(Hn.astype(np.int32)).to(dev)
    u = O.factorised_u(a, b, phi)
    ld_ref = O.log_denominator(u, f, Nk)
    Q_ref = Nk * (O.mbar_weights(u, f, Nk) * Hn[None, :]).sum(axis=1)
    td = lambda x: torch.from_numpy(np.ascontiguousarray(x, dtype=np.float64)).to(dev)
    lN = np.log(np.maximum(Nk, 0).astype(np.float64))
    Q = torch.empty(K, dtype=torch.float64, device=dev)
    logden = torch.empty(N, dtype=torch.float64, device=dev)
    scratch = torch.zeros(M.lse_factorised_scratch_bytes(K, N), dtype=torch.uint8, device=dev)
    for _ in range(2):   # the scratch is left zero for the next call
        M.lse_pass_factorised(td(a), td(b), td(phi), td(f), td(lN), Q, H=H, logden=logden, scratch=scratch)
    torch.cuda.synchronize()
    X = float(np.max(np.abs(ld_ref)))
    tol = 1e-6 + 8.0 * X * 2.0**-24
    Qg = Q.cpu().numpy()
    occupied = Nk > 0
    assert np.max(np.abs(Qg[occupied] - Q_ref[occupied]) / Q_ref[occupied]) < tol
    assert np.all(Qg[~occupied] == 0.0)
    assert np.max(np.abs(logden.cpu().numpy() - ld_ref)) < tol


def test_lse_pass_factorised_rejects_bad_arguments():
    import torch
    dev = torch.device("cuda")
    K, N = 4, 10
    z = lambda n: torch.zeros(n, dtype=torch.float64, device=dev)
    Q = z(K)
    small = torch.zeros(16, dtype=torch.uint8, device=dev)
    with pytest.raises(M.MbarError):
        M.lse_pass_factorised(z(K), z(K), z(N), z(K), z(K), Q, scratch=small)
    big = torch.zeros(M.lse_factorised_scratch_bytes(K, N), dtype=torch.uint8, device=dev)
    with pytest.raises(M.MbarError):
        M.lse_pass_factorised(z(1025), z(1025), z(N), z(1025), z(1025), z(1025), scratch=big)


def _pt_factorised(K=6, N_k=3000, s2=40.0, seed=2):
    p = W.parallel_tempering(K=K, N_k=N_k, sigma2=s2, seed=seed, materialize=False)
    b = p.meta["b"]
    a = np.linspace(-2.0, 3.0, K)
    return a, b, p.phi, p.N_k


@pytest.mark.parametrize("prec", [M.MBAR_FP64])
@pytest.mark.parametrize("where", ["host", "device"])
def test_create_factorised_is_create_on_the_generated_u(prec, where):
    """FP64: mbar_create_factorised generates u_kn = a_k + b_k phi_n with
    the host's binary64 rounding and bins by phi: the solve is bit for bit
    the one of mbar_create on the oracle's materialised u with phi set as the
    coordinate, and both match the oracle's MBAR solution. (MIXED contexts
    keep no K x N store: tests/test_gpu_factorised.py.)"""
    import torch
    a, b, phi, Nk = _pt_factorised()
    if where == "device":
        td = lambda x: torch.from_numpy(np.ascontiguousarray(x, dtype=np.float64)).cuda()
        c1 = M.Context.factorised(td(a), td(b), td(phi), Nk, prec)
    else:
        c1 = M.Context.factorised(a, b, phi, Nk, prec)
    c1.solve()
    f1 = c1.free_energies()
    c1.close()
    u = O.factorised_u(a, b, phi)
    c2 = M.Context(u, Nk, prec)
    c2.set_coordinate(phi)
    c2.solve()
    f2 = c2.free_energies()
    c2.close()
    assert np.array_equal(f1, f2)
    f_ref = O.solve_mbar(u, Nk)
    assert np.max(np.abs(f1 - f_ref)) < (1e-8 if prec == M.MBAR_FP64 else 1e-4)


def test_create_factorised_rejects_bad_input():
    a, b, phi, Nk = _pt_factorised(K=3, N_k=50)
    with pytest.raises(M.MbarError):
        M.Context.factorised(a, b, np.where(np.arange(len(phi)) == 7, np.nan, phi), Nk, M.MBAR_MIXED)
    with pytest.raises(M.MbarError):
        M.Context.factorised(a, b, phi, Nk + 1, M.MBAR_MIXED)
    with pytest.raises(ValueError):
        M.Context.factorised(a[:2], b, phi, Nk, M.MBAR_MIXED)


@pytest.mark.parametrize("case", ["gaussian", "umbrella_h0", "harmonic_wide"])
def test_algorithm1_trajectory_matches_oracle_fp64(case):
    """Every Eq. 3 check of the second loop (level size, s_n, s_next) and the
    end of the first loop agree with the oracle's run: the binned levels,
    built up front from one read of the data, carry the same bin means as the
    oracle's level-by-level histograms."""
    if case == "gaussian":
        p = W.gaussian_overlap(M=12, N_0=2000, seed=4)
        opts = O.BUOptions()
        o = M.default_opts(M.MBAR_FP64)
    elif case == "umbrella_h0":
        p = W.umbrella(K=16, N_k=1000, seed=1, grid_points=1 << 13)
        opts = O.BUOptions(h0=0.1)
        o = M.default_opts(M.MBAR_FP64, h0=0.1)
    else:   # 80 000 samples: single-bin tiles at 100 bins, boundaries at 1000, small bins at 10 000
        p = W.harmonic(K=4, d=1, N_k=20000, seed=9)
        p.phi = p.u_kn[0].copy()
        opts = O.BUOptions()
        o = M.default_opts(M.MBAR_FP64)
    tr = []
    O.bu_mbar(p.u_kn, p.N_k, phi=p.phi, opts=opts, trace=tr)
    ctx = M.Context(p.u_kn, p.N_k, M.MBAR_FP64, opts=o)
    ctx.set_coordinate(p.phi)
    ctx.solve()
    gt = ctx.trace()
    ctx.close()
    ph1 = [t for t in tr if t[0] == "phase1"]
    ph2 = [t for t in tr if t[0] == "phase2"]
    g1 = [r for r in gt if r[0] == 1]
    g2 = [r for r in gt if r[0] == 2]
    assert len(g1) == 1 and int(g1[0][3]) == len(ph1)
    assert g1[0][2] == pytest.approx(ph1[-1][2], rel=1e-6)
    assert len(g2) == len(ph2) and len(g2) >= 1
    for r, t in zip(g2, ph2):
        assert int(r[1]) == t[1]
        for a, b in ((r[2], t[2]), (r[3], t[3])):
            if b > 1e-9:
                assert a == pytest.approx(b, rel=1e-6)
            else:   # a converged level: both at the FP64 rounding floor
                assert a < 1e-9


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_solve_parallel_tempering_spread_needs_log_domain_steps(prec):
    """Sec. III-shaped energies spread over ~1000 kT between the coldest and
    hottest state: from f = 0 some states' linear-domain row sums underflow
    (even in FP64); those steps are redone exactly in the log domain."""
    p = W.parallel_tempering(K=16, N_k=800, seed=2)
    f_ref = O.solve_mbar(p.u_kn, p.N_k)
    ctx = M.Context(p.u_kn, p.N_k, PREC[prec])
    ctx.set_coordinate(p.phi)
    rep = ctx.solve()
    f = ctx.free_energies()
    ctx.close()
    assert np.max(np.abs(f - f_ref)) < SOLVE_TOL[prec], rep.as_dict()


def test_parallel_tempering_trajectory_matches_oracle_fp64():
    """The log-domain redo of an underflowed step is the oracle's step: the
    first loop's length and every Eq. 3 check agree."""
    p = W.parallel_tempering(K=12, N_k=1000, seed=4)
    tr = []
    O.bu_mbar(p.u_kn, p.N_k, phi=p.phi, trace=tr)
    ctx = M.Context(p.u_kn, p.N_k, M.MBAR_FP64)
    ctx.set_coordinate(p.phi)
    ctx.solve()
    gt = ctx.trace()
    ctx.close()
    ph1 = [t for t in tr if t[0] == "phase1"]
    g1 = [r for r in gt if r[0] == 1]
    assert int(g1[0][3]) == len(ph1)
    ph2 = [t for t in tr if t[0] == "phase2"]
    g2 = [r for r in gt if r[0] == 2]
    assert len(g2) == len(ph2)
    for r, t in zip(g2, ph2):
        for a, b in ((r[2], t[2]), (r[3], t[3])):
            if b > 1e-9:
                assert a == pytest.approx(b, rel=1e-6)
            else:
                assert a < 1e-9


def test_mixed_tempering_offsets_are_not_quantised():
    """States whose offsets a_k = f_k + ln N_k reach hundreds of kT (the
    tempering spread) keep their full precision in the FP32 passes: MIXED's
    loops stop about where FP64's do, instead of cycling at the FP32 spacing
    of a_k (4e-5 kT at |a_k| ~ 760) until max_sci, and it ends within
    3 f_tol of the oracle (the FP32 log2(e) alone biased it by 1e-5 kT)."""
    p = W.parallel_tempering(K=16, N_k=1500, seed=6)
    f_ref = O.solve_mbar(p.u_kn, p.N_k)
    out = {}
    for prec in (M.MBAR_FP64, M.MBAR_MIXED):
        ctx = M.Context(p.u_kn, p.N_k, prec)
        ctx.set_coordinate(p.phi)
        rep = ctx.solve().as_dict()
        out[prec] = (ctx.free_energies(), rep)
        ctx.close()
    assert np.max(np.abs(f_ref[1:] - f_ref[:-1])) > 10.0     # the spread is really there
    f, rep = out[M.MBAR_MIXED]
    _, rep64 = out[M.MBAR_FP64]
    assert np.max(np.abs(f - f_ref)) < 3e-5, rep
    sci = rep["iters_first_loop"] + rep["iters_second_loop"]
    sci64 = rep64["iters_first_loop"] + rep64["iters_second_loop"]
    assert sci <= 2 * sci64 + 500, (rep, rep64)


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
@pytest.mark.parametrize("K,N", [(3, 37), (100, 2001), (500, 4133), (1000, 1031)])
def test_store_formed_late_or_early_is_the_same(prec, K, N):
    """The data is staged sample-major at creation and stored row-major by
    the first call that needs it: in the coordinate's order when that call is
    the coordinate (one gather of whole samples), in the original order
    otherwise (a later coordinate then reorders the stored columns). Both
    routes end in the same store: identical SCI steps and solves."""
    u, Nk = rand_problem(K, N, seed=K, offset=50.0)
    phi = u[0] + 0.01 * np.arange(N) % 7
    f = rand_f(K)
    a = M.Context(u, Nk, PREC[prec])            # coordinate first
    a.set_coordinate(phi)
    b = M.Context(u, Nk, PREC[prec])            # unbinned step first, coordinate later
    fb0, _, _, ldb0 = b.sci_step(f, want_logden=True)
    b.set_coordinate(phi)
    fa, ga, sa, lda = a.sci_step(f, want_logden=True)
    fb, gb, sb, ldb = b.sci_step(f, want_logden=True)
    tol = F_TOL[prec]
    assert np.max(np.abs(fb0 - O.gauge(O.sci_step(u, f, Nk)))) < tol
    assert np.array_equal(fa, fb) and np.array_equal(lda, ldb) and sa == sb and np.array_equal(ga, gb)
    assert np.max(np.abs(ldb0 - ldb)) < tol
    if K <= 500:
        a.solve()
        b.solve()
        assert np.array_equal(a.free_energies(), b.free_energies())
    a.close()
    b.close()


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
@pytest.mark.parametrize("K,N_k", [(3, 400), (12, 150), (80, 30)])
def test_covariance_matches_oracle(prec, K, N_k):
    """mbar_covariance (Cholesky of the reduced Hessian, column-by-column
    inverse, sample terms) against the oracle's weight-matrix formula at the
    same f; the tensor-core Hessian (K >= 64) carries FP16 products."""
    p = W.harmonic(K=K, d=2, N_k=N_k, seed=K)
    ctx = M.Context(p.u_kn, p.N_k, PREC[prec])
    ctx.solve()
    f = ctx.free_energies()
    C = ctx.covariance()
    ctx.close()
    C_ref = O.mbar_covariance(p.u_kn, f, p.N_k)
    scale = np.sqrt(np.outer(np.diag(C_ref), np.diag(C_ref)))[1:, 1:]
    tol = 3e-2 if K >= 64 else 1e-3       # the Hessian kernels' FP16 / FP32 products
    assert np.all(C[0] == 0.0) and np.all(C[:, 0] == 0.0)
    assert np.max(np.abs(C[1:, 1:] - C_ref[1:, 1:]) / scale) < tol


@pytest.mark.parametrize("case", ["gaussian", "umbrella_h0", "alchemical"])
def test_mixed_first_loop_follows_the_oracle(case):
    """MIXED runs the first loop on its small FP32 level in single launches
    (the whole loop on chip): it stops within one step of where the oracle's
    FP64 first loop stops, with the same last relative step to 2 % (Eq. 2
    divides FP32 rounding by the small f_k next to the gauge state), and the
    solve still ends at the oracle's free energies."""
    if case == "gaussian":
        p = W.gaussian_overlap(M=12, N_0=2000, seed=4)
        opts, o = O.BUOptions(), M.default_opts(M.MBAR_MIXED)
    elif case == "umbrella_h0":
        p = W.umbrella(K=16, N_k=1000, seed=1, grid_points=1 << 13)
        opts, o = O.BUOptions(h0=0.1), M.default_opts(M.MBAR_MIXED, h0=0.1)
    else:
        p = W.alchemical(K=40, N_k=300, seed=3)
        opts, o = O.BUOptions(), M.default_opts(M.MBAR_MIXED)
    tr = []
    f_ref = O.bu_mbar(p.u_kn, p.N_k, phi=p.phi, opts=opts, trace=tr)
    ctx = M.Context(p.u_kn, p.N_k, M.MBAR_MIXED, opts=o)
    ctx.set_coordinate(p.phi)
    ctx.solve()
    gt = ctx.trace()
    f = ctx.free_energies()
    ctx.close()
    ph1 = [t for t in tr if t[0] == "phase1"]
    g1 = [r for r in gt if r[0] == 1]
    assert len(g1) == 1 and abs(int(g1[0][3]) - len(ph1)) <= 1
    if int(g1[0][3]) == len(ph1):
        assert g1[0][2] == pytest.approx(ph1[-1][2], rel=2e-2)
    assert np.max(np.abs(f - f_ref)) < SOLVE_TOL["mixed"]


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_mixed_second_loop_stall_then_newton_reaches_the_oracle(seed):
    """Four umbrella windows 1.0 apart barely overlap (the reduced Hessian's
    smallest eigenvalue is 0.02-0.2): SCI contracts so slowly that the FP64
    second loop runs 1e5-2e5 steps. MIXED raises n once its steps stop
    shrinking (they sit on the FP32 rounding of the evaluation) instead of
    running to max_sci; the unbinned Newton phase, whose gradient keeps each
    sample's largest weight as an exact count plus its small remainder, then
    ends within the mixed tolerance of the oracle."""
    p = W.umbrella(K=4, N_k=4299, seed=seed, grid_points=1 << 13)
    f_ref = O.solve_mbar(p.u_kn, p.N_k)
    ctx = M.Context(p.u_kn, p.N_k, M.MBAR_MIXED)
    ctx.set_coordinate(p.phi)
    rep = ctx.solve().as_dict()
    f = ctx.free_energies()
    ctx.close()
    assert rep["iters_second_loop"] < 20000, rep
    assert np.max(np.abs(f - f_ref)) < SOLVE_TOL["mixed"], rep
