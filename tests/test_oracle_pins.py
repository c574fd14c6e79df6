"""Pins for the CPU oracle: each check ties an oracle function to something
other than itself (a closed form, an independent equation, a high-precision
brute force, finite differences, an exact invariance or a hand-derived
fixture). CPU only."""
import json
import math
import os

import mpmath as mp
import numpy as np
import pytest

import oracle as O
from paper_2609_03541_b300 import workloads as W


def _rand_problem(K=4, Nk=(3, 5, 2, 4), seed=0, scale=2.0):
    g = np.random.default_rng(seed)
    N_k = np.asarray(Nk[:K], dtype=np.int64)
    u = scale * g.standard_normal((K, int(N_k.sum()))) + g.uniform(-3, 3, size=(K, 1))
    return u, N_k


# ---------------------------------------------------------------------------
# closed forms
# ---------------------------------------------------------------------------

def test_two_samples_two_states_closed_form():
    """K = 2, one sample per state. With f_0 = 0 the state-0 equation reads
    1/(1+A) + 1/(1+B) = 1 with A = e^{f-da}, B = e^{f-db} (da, db the energy
    differences u_1n - u_0n), i.e. AB = 1, so f_1 = (da + db) / 2."""
    g = np.random.default_rng(3)
    for _ in range(5):
        u = g.normal(size=(2, 2)) * 3
        f = O.solve_mbar(u, np.array([1, 1]))
        da, db = u[1] - u[0]
        assert abs(f[1] - 0.5 * (da + db)) < 1e-12


def test_constant_offset_states_closed_form():
    """If u_k = u_0 + c_k for every sample, then f_k = c_k - c_0 for any data."""
    g = np.random.default_rng(4)
    u0 = g.normal(size=50) * 2
    c = g.uniform(-5, 5, size=6)
    u = u0[None, :] + c[:, None]
    N_k = np.array([10, 5, 5, 10, 15, 5])
    f = O.solve_mbar(u, N_k)
    assert np.max(np.abs(f - (c - c[0]))) < 1e-12
    # one Eq. 1 step from f = 0 already lands there
    f1 = O.gauge(O.sci_step(u, np.zeros(6), N_k))
    assert np.max(np.abs(f1 - (c - c[0]))) < 1e-12


def test_bar_equivalence_for_two_states():
    """MBAR with K = 2 is Bennett's acceptance ratio. Solve Bennett's
    implicit equation (which uses the sample labels, unlike MBAR) by
    bisection and compare. N_0 != N_1 catches a transposed N_k."""
    g = np.random.default_rng(5)
    N0, N1 = 300, 170
    x0 = g.normal(0.0, 1.0, N0)
    x1 = g.normal(0.7, 1.2, N1)
    x = np.concatenate([x0, x1])
    u = np.stack([0.5 * x**2, 0.5 * ((x - 0.7) / 1.2) ** 2 + math.log(1.2)])
    du = u[1] - u[0]

    def bennett(df):
        lhs = np.sum(1.0 / (1.0 + (N0 / N1) * np.exp(du[:N0] - df)))
        rhs = np.sum(1.0 / (1.0 + (N1 / N0) * np.exp(-du[N0:] + df)))
        return lhs - rhs          # increasing in df

    lo, hi = -50.0, 50.0
    for _ in range(200):
        mid = 0.5 * (lo + hi)
        if bennett(mid) > 0:
            hi = mid
        else:
            lo = mid
    f = O.solve_mbar(u, np.array([N0, N1]))
    assert abs(f[1] - 0.5 * (lo + hi)) < 1e-10


def _mp_solve(u, N_k, dps=40):
    mp.mp.dps = dps
    K, N = u.shape
    U = [[mp.mpf(float(u[k, n])) for n in range(N)] for k in range(K)]
    Nk = [mp.mpf(int(v)) for v in N_k]

    def eqs(*fs):
        f = [mp.mpf(0)] + list(fs)
        out = []
        for i in range(1, K):
            tot = mp.mpf(0)
            for n in range(N):
                den = mp.fsum(Nk[j] * mp.exp(f[j] - U[j][n]) for j in range(K))
                tot += mp.exp(f[i] - U[i][n]) / den
            out.append(tot - 1)
        return out

    sol = mp.findroot(eqs, [mp.mpf(0)] * (K - 1))
    sol = [sol] if K == 2 else list(sol)
    return np.array([0.0] + [float(s) for s in sol])


@pytest.mark.parametrize("seed", [0, 1])
def test_bruteforce_40_digits(seed):
    """Root of sum_n W_kn = 1 found by mpmath at 40 digits, directly from the
    definition (plain sums, no log-sum-exp), K = 3, N = 6."""
    u, N_k = _rand_problem(K=3, Nk=(2, 3, 1), seed=seed, scale=1.5)
    f_mp = _mp_solve(u, N_k)
    f = O.solve_mbar(u, N_k)
    assert np.max(np.abs(f - f_mp)) < 1e-12


def test_sci_step_against_direct_eq1_in_high_precision():
    """Eq. 1 evaluated literally with 40-digit sums, binned (H_p > 1)."""
    u, N_k = _rand_problem(K=3, Nk=(2, 3, 2), seed=7, scale=3.0)
    H = np.array([1, 3, 2, 1, 4, 1, 2])
    f = np.array([0.0, 0.4, -1.3])
    mp.mp.dps = 40
    K, n = u.shape
    expect = []
    for i in range(K):
        tot = mp.mpf(0)
        for p in range(n):
            den = mp.fsum(int(N_k[j]) * mp.exp(mp.mpf(f[j]) - mp.mpf(float(u[j, p]))) for j in range(K))
            tot += int(H[p]) * mp.exp(-mp.mpf(float(u[i, p]))) / den
        expect.append(float(-mp.log(tot)))
    got = O.sci_step(u, f, N_k, H)
    assert np.max(np.abs(got - np.array(expect))) < 1e-13


# ---------------------------------------------------------------------------
# derivatives
# ---------------------------------------------------------------------------

def test_gradient_is_derivative_of_objective():
    u, N_k = _rand_problem(K=4, seed=11)
    H = np.array([1, 2, 1, 3, 1, 1, 2, 1, 1, 1, 2, 1, 1, 1])
    f = np.array([0.0, 0.3, -0.2, 1.1])
    g = O.mbar_gradient(u, f, N_k, H)
    h = 1e-5
    fd = np.array([(O.mbar_objective(u, f + h * e, N_k, H) - O.mbar_objective(u, f - h * e, N_k, H)) / (2 * h)
                   for e in np.eye(4)])
    assert np.max(np.abs(g - fd)) < 1e-7 * max(1.0, np.max(np.abs(g)))


def test_hessian_is_derivative_of_gradient_and_has_gauge_null_vector():
    u, N_k = _rand_problem(K=4, seed=12)
    f = np.array([0.0, -0.4, 0.2, 0.9])
    Hs = O.mbar_hessian(u, f, N_k)
    h = 1e-5
    fd = np.stack([(O.mbar_gradient(u, f + h * e, N_k) - O.mbar_gradient(u, f - h * e, N_k)) / (2 * h)
                   for e in np.eye(4)], axis=1)
    assert np.max(np.abs(Hs - fd)) < 1e-7
    assert np.max(np.abs(Hs - Hs.T)) < 1e-14
    assert np.max(np.abs(Hs @ np.ones(4))) < 1e-12
    assert np.min(np.linalg.eigvalsh(Hs)) > -1e-12
    # binned form, counts H_n as weights
    Hn = np.array([1, 2, 1, 3, 1, 1, 2, 1, 1, 1, 2, 1, 1, 1])
    Hb = O.mbar_hessian(u, f, N_k, Hn)
    fd = np.stack([(O.mbar_gradient(u, f + h * e, N_k, Hn) - O.mbar_gradient(u, f - h * e, N_k, Hn)) / (2 * h)
                   for e in np.eye(4)], axis=1)
    assert np.max(np.abs(Hb - fd)) < 1e-7


# ---------------------------------------------------------------------------
# solution properties and invariances
# ---------------------------------------------------------------------------

def test_fixed_point_and_weight_sums():
    p = W.harmonic(K=5, N_k=200, seed=2)
    f = O.solve_mbar(p.u_kn, p.N_k)
    Wkn = O.mbar_weights(p.u_kn, f, p.N_k)
    assert np.max(np.abs(Wkn.sum(axis=1) - 1.0)) < 1e-12          # each state's weights sum to 1
    assert np.max(np.abs((p.N_k[:, None] * Wkn).sum(axis=0) - 1.0)) < 1e-12   # each sample's
    assert f[0] == 0.0                                             # gauge
    f_sci = O.gauge(O.sci_step(p.u_kn, f, p.N_k))                   # Eq. 1 fixed point
    assert np.max(np.abs(f_sci - f)) < 1e-11


def test_exact_invariances():
    p = W.harmonic(K=4, N_k=100, seed=9)
    f = O.solve_mbar(p.u_kn, p.N_k)
    g = np.random.default_rng(0)
    c_k = g.normal(size=4) * 3
    c_n = g.normal(size=p.N) * 50
    f_state = O.solve_mbar(p.u_kn + c_k[:, None], p.N_k)
    assert np.max(np.abs(f_state - (f + c_k - c_k[0]))) < 1e-10
    f_sample = O.solve_mbar(p.u_kn + c_n[None, :], p.N_k)
    assert np.max(np.abs(f_sample - f)) < 1e-10
    perm = g.permutation(p.N)
    f_perm = O.solve_mbar(p.u_kn[:, perm], p.N_k)
    assert np.max(np.abs(f_perm - f)) < 1e-10


def test_duplicate_sample_equals_count_two():
    u, N_k = _rand_problem(K=3, Nk=(2, 2, 2), seed=21)
    f = np.array([0.0, 0.5, -0.5])
    H = np.array([1, 2, 1, 1, 1, 1])
    dup = np.concatenate([u, u[:, 1:2]], axis=1)
    a = O.sci_step(u, f, N_k, H)
    b = O.sci_step(dup, f, N_k)
    assert np.max(np.abs(a - b)) < 1e-14
    ga = O.mbar_gradient(u, f, N_k, H)
    gb = O.mbar_gradient(dup, f, N_k)
    assert np.max(np.abs(ga - gb)) < 1e-13


def test_one_sample_per_bin_is_the_unbinned_step():
    p = W.umbrella(K=6, N_k=40, seed=1, grid_points=1 << 12)
    phi = p.phi
    w = np.min(np.diff(np.unique(phi))) / 4
    hist = O.histogram(phi, w)
    assert np.all(hist.H == 1) and hist.H.shape[0] == p.N
    ub = O.binned_u(p.u_kn, hist)
    f = np.linspace(0, 1, 6)
    a = O.sci_step(ub, f, p.N_k, hist.H)
    b = O.sci_step(p.u_kn, f, p.N_k)
    assert np.max(np.abs(a - b)) < 1e-13


# ---------------------------------------------------------------------------
# binning fixtures (hand-derived) and the width rule
# ---------------------------------------------------------------------------

def test_binning_golden(golden_dir):
    spec = json.load(open(os.path.join(golden_dir, "binning_cases.json")))
    for case in spec["cases"]:
        phi = np.array(case["phi"])
        keys = O.bin_keys(phi, phi.min(), case["w"])
        assert keys.tolist() == case["keys"], case["name"]
        h = O.histogram(phi, case["w"])
        assert h.keys.tolist() == case["nonempty_keys"], case["name"]
        assert h.H.tolist() == case["H"], case["name"]
        assert O.nonempty_bins(phi, case["w"]) == len(case["H"])
    for case in spec["width_cases"]:
        phi = np.arange(float(case["phi_range"]))
        assert O.width_for_bins(phi, case["n"]) == case["w_star"], case["name"]


def test_width_rule_properties():
    """w* has g(w*) >= n and the next binary64 number above it has fewer."""
    g = np.random.default_rng(8)
    phi = np.concatenate([g.normal(size=3000), 5 + 0.1 * g.standard_t(3, size=500)])
    for n in (10, 100, 1000):
        w = O.width_for_bins(phi, n)
        assert O.nonempty_bins(phi, w) >= n
        assert O.nonempty_bins(phi, np.nextafter(w, np.inf)) < n
    assert O.width_for_bins(phi, 10**6) is None          # more bins than distinct values


def test_binned_u_is_member_mean():
    g = np.random.default_rng(2)
    phi = np.round(g.normal(size=200), 1)
    u = g.normal(size=(3, 200))
    hist = O.histogram(phi, 0.25)
    ub = O.binned_u(u, hist)
    for p, m in enumerate(hist.members):
        assert np.allclose(ub[:, p], u[:, m].mean(axis=1), rtol=0, atol=1e-14)
    assert hist.H.sum() == 200


# ---------------------------------------------------------------------------
# Algorithm 1
# ---------------------------------------------------------------------------

def test_algorithm1_defaults(golden_dir):
    spec = json.load(open(os.path.join(golden_dir, "algorithm1_hyperparameters.json")))
    o = O.BUOptions()
    assert (o.n0, o.eps, o.inc, o.n_intermediate) == (spec["n0"], spec["eps"], spec["inc"], spec["n_intermediate"])


def test_algorithm1_reaches_the_mbar_solution():
    p = W.gaussian_overlap(M=8, N_0=3000, seed=3)
    tr = []
    f_bu = O.bu_mbar(p.u_kn, p.N_k, phi=p.phi, trace=tr)
    f = O.solve_mbar(p.u_kn, p.N_k)
    assert np.max(np.abs(f_bu - f)) < 1e-10
    ns = [t[1] for t in tr if t[0] in ("phase1", "phase2")]
    assert ns[0] == 100
    assert all(b >= a for a, b in zip(ns, ns[1:]))              # bins only ever refine
    assert set(ns) <= {100, 1000, 10000}


def _trace_fixture(golden_dir):
    with open(os.path.join(golden_dir, "algorithm1_trace.json")) as fh:
        return json.load(fh)


@pytest.mark.parametrize("which", ["trace", "trace_noise_floor"])
def test_algorithm1_trace_matches_the_derivation(golden_dir, which):
    """The oracle's Algorithm 1 takes every decision of the 50-digit
    derivation (tests/golden/derive_algorithm1_trace.py: Eqs. 1-3 in their
    printed form): the same first-loop length under s < eps, the same Eq. 3
    outcome in every round (the next round's n), the same end by the break
    rule 2 inc n > sum N_i, and the same step widths s, s_n, s_next. The
    second case adds the noise-floor rule of the finite-precision reading."""
    spec = _trace_fixture(golden_dir)
    P = spec["params"]
    floor = spec["noise_floor"] if which == "trace_noise_floor" else 0.0
    opts = O.BUOptions(n0=P["n0"], eps=P["eps"], inc=P["inc"], n_intermediate=P["n_intermediate"],
                       noise_floor=floor)
    tr = []
    O.bu_mbar(np.asarray(spec["u"]), np.asarray(spec["N_k"]), phi=np.asarray(spec["phi"]), opts=opts, trace=tr)
    rows = [t for t in tr if t[0] in ("phase1", "phase2")]
    exp = spec[which]
    assert [(r[0], r[1]) for r in rows] == [(f"phase{e['phase']}", e["n"]) for e in exp]
    for r, e in zip(rows, exp):
        if e["phase"] == 1:
            assert (r[2] == math.inf) if e["s"] == "inf" else r[2] == pytest.approx(e["s"], rel=1e-7)
        else:
            assert r[2] == pytest.approx(e["s_n"], rel=1e-7)
            assert r[3] == pytest.approx(e["s_next"], rel=1e-7)


def test_algorithm1_trace_fixture_tells_the_rules_apart(golden_dir):
    """The derived trace would change under the plausible slips in Eq. 3 and
    the break rule: it has rounds that raise n and rounds that do not (a
    flipped inequality), a round that raises n only with the factor 2
    (inc s_n < 2 s_next but not inc s_n < s_next), a last raise where
    2 inc n exceeds sum N_i but inc n does not, a first loop that stops on
    s < eps, and, with the noise floor, a first-loop stop and a raise that
    come from the floor alone."""
    spec = _trace_fixture(golden_dir)
    inc, N = spec["params"]["inc"], sum(spec["N_k"])
    p2 = [e for e in spec["trace"] if e["phase"] == 2]
    assert any(e["raise_n"] for e in p2) and any(not e["raise_n"] for e in p2)
    assert all(e["raise_n"] == (inc * e["s_n"] < 2 * e["s_next"]) for e in p2)
    assert any(inc * e["s_n"] < 2 * e["s_next"] and not inc * e["s_n"] < e["s_next"] for e in p2)
    n_last = p2[-1]["n"] * inc
    assert p2[-1]["raise_n"] and 2 * inc * n_last > N and not inc * n_last > N
    assert spec["trace"][[e["phase"] for e in spec["trace"]].index(2) - 1]["stop"]
    nf = spec["trace_noise_floor"]
    assert any(e["phase"] == 1 and e["by_noise_floor"] for e in nf)
    assert any(e["phase"] == 2 and e["by_noise_floor"] for e in nf)
    assert min(e["eq3_margin"] for e in p2) > 1e-3      # no decision within rounding of its threshold


def test_algorithm1_width_schedule():
    p = W.umbrella(K=8, N_k=400, seed=4, grid_points=1 << 12)
    o = O.BUOptions(h0=0.1)
    f_bu = O.bu_mbar(p.u_kn, p.N_k, phi=p.phi, opts=o)
    f = O.solve_mbar(p.u_kn, p.N_k)
    assert np.max(np.abs(f_bu - f)) < 1e-10


def test_relative_step_reading():
    assert O.relative_step(np.array([0.0, 1.0]), np.zeros(2)) == math.inf
    assert O.relative_step(np.array([0.0, 1.5, -2.0]), np.array([0.0, 1.0, -1.0])) == 1.0


# ---------------------------------------------------------------------------
# statistical pins against analytic free energies
# ---------------------------------------------------------------------------

def _sigma(u, f, N_k):
    Hs = O.mbar_hessian(u, f, N_k)
    cov = np.linalg.inv(Hs[1:, 1:])
    return np.concatenate([[0.0], np.sqrt(np.diag(cov))])


def test_harmonic_analytic():
    """f_k - f_0 = (d/2) ln(kappa_k/kappa_0) for u_k = kappa_k |x - mu_k|^2 / 2."""
    p = W.harmonic(K=8, d=3, N_k=1000, seed=0)
    f = O.solve_mbar(p.u_kn, p.N_k)
    kap = p.meta["kappa"]
    exact = 1.5 * np.log(kap / kap[0])
    sig = _sigma(p.u_kn, f, p.N_k)
    assert np.all(np.abs(f - exact)[1:] < 5 * sig[1:] + 1e-3)
    assert np.max(sig) < 0.2


def test_gaussian_overlap_analytic():
    """Unit-variance Gaussian density of states: f(beta) = -beta^2/2 + const."""
    p = W.gaussian_overlap(M=10, N_0=2000, seed=1)
    f = O.solve_mbar(p.u_kn, p.N_k)
    b = p.meta["beta"]
    exact = -(b**2 - b[0] ** 2) / 2
    sig = _sigma(p.u_kn, f, p.N_k)
    assert np.all(np.abs(f - exact)[1:] < 5 * sig[1:] + 1e-3)


def test_factorised_u_without_phi_dependence_is_closed_form():
    """b = 0: every sample sees the same potentials a_k, so logden_p =
    log sum_j N_j exp(f_j - a_j) for every p, and Q_i = N_i sum_p W_ip =
    n N_i exp(f_i - a_i) / sum_j N_j exp(f_j - a_j)."""
    g = np.random.default_rng(3)
    K, n = 5, 11
    a = 3.0 * g.normal(size=K)
    f = g.normal(size=K)
    Nk = g.integers(1, 9, size=K)
    phi = 100.0 * g.normal(size=n)
    u = O.factorised_u(a, np.zeros(K), phi)
    ld = O.log_denominator(u, f, Nk)
    exact = math.log(sum(int(Nk[j]) * math.exp(f[j] - a[j]) for j in range(K)))
    assert np.max(np.abs(ld - exact)) < 1e-13
    Q = Nk * O.mbar_weights(u, f, Nk).sum(axis=1)
    Q_exact = n * Nk * np.exp(f - a) / math.exp(exact)
    assert np.max(np.abs(Q / Q_exact - 1.0)) < 1e-13


def test_factorised_u_gaussian_density_of_states():
    """u_kp = b_k E_p with E from a Gaussian density of states of variance s2
    (state b draws N(-b s2, s2)): f(b) = -b^2 s2 / 2 + const, the paper's
    tempering setting. The MBAR solution on factorised_u(0, b, E) lies
    within statistical error of it, and a per-state offset a_k moves f_k by
    a_k exactly (u_kp + a_k has Boltzmann factor e^{-a_k} times the old)."""
    s2 = 40.0
    p = W.parallel_tempering(K=6, N_k=3000, sigma2=s2, seed=2, materialize=False)
    b = p.meta["b"]
    u = O.factorised_u(np.zeros_like(b), b, p.phi)
    f = O.solve_mbar(u, p.N_k)
    exact = -(b**2 - b[0] ** 2) * s2 / 2
    sig = _sigma(u, f, p.N_k)
    assert np.all(np.abs(f - exact)[1:] < 5 * sig[1:] + 1e-3)
    assert np.max(sig) < 0.2
    a = np.linspace(-3.0, 5.0, len(b))
    f2 = O.solve_mbar(O.factorised_u(a, b, p.phi), p.N_k)
    assert np.max(np.abs((f2 - f) - (a - a[0]))) < 1e-8


def test_binned_factorised_u_is_factorised_u_at_the_bin_means():
    """Reading c4 (bin representative = mean of the members) on factorised
    potentials: the mean of a_k + b_k phi_n over a bin is a_k + b_k times the
    mean phi of the bin, so a binned level of factorised u is itself
    factorised, (mean phi_b, H_b), up to FP64 rounding."""
    p = W.parallel_tempering(K=5, N_k=400, sigma2=40.0, seed=4, materialize=False)
    b = p.meta["b"]
    a = np.linspace(-1.0, 2.0, len(b))
    u = O.factorised_u(a, b, p.phi)
    for n_bins in (7, 60, 500):
        w = O.width_for_bins(p.phi, n_bins)
        hist = O.histogram(p.phi, w)
        ub = O.binned_u(u, hist)
        phib = np.array([p.phi[m].mean() for m in hist.members])
        assert np.max(np.abs(ub - O.factorised_u(a, b, phib))) < 1e-12 * np.max(np.abs(u))
        assert int(hist.H.sum()) == len(p.phi)


def test_umbrella_quadrature():
    from scipy.integrate import quad
    p = W.umbrella(K=12, N_k=800, seed=2, grid_points=1 << 14)
    f = O.solve_mbar(p.u_kn, p.N_k)
    c = p.meta["centres"]
    kap = p.meta["kappa"]
    Z = [quad(lambda x: math.exp(-W.double_well(x) - 0.5 * kap * (x - ck) ** 2), ck - 2, ck + 2,
              epsabs=0, epsrel=1e-12, limit=200)[0] for ck in c]
    exact = -np.log(Z)
    exact -= exact[0]
    sig = _sigma(p.u_kn, f, p.N_k)
    assert np.all(np.abs(f - exact)[1:] < 5 * sig[1:] + 1e-3)


# ---------------------------------------------------------------------------
# Eqs. 5-7
# ---------------------------------------------------------------------------

def test_reweight_to_a_sampled_state_gives_its_mbar_weights():
    p = W.harmonic(K=4, N_k=150, seed=6)
    f = O.solve_mbar(p.u_kn, p.N_k)
    pw = O.reweight(p.u_kn[2], p.u_kn, f, p.N_k)
    assert abs(pw.sum() - 1.0) < 1e-13
    Wkn = O.mbar_weights(p.u_kn, f, p.N_k)
    assert np.max(np.abs(pw - Wkn[2])) < 1e-14


def test_reweight_high_precision():
    u, N_k = _rand_problem(K=3, Nk=(2, 2, 1), seed=31)
    f = np.array([0.0, 0.2, -0.7])
    u0 = np.array([0.1, -0.3, 1.2, 0.0, 0.5])
    mp.mp.dps = 40
    raw = []
    for n in range(5):
        den = mp.fsum(int(N_k[m]) * mp.exp(mp.mpf(f[m]) - mp.mpf(float(u[m, n]))) for m in range(3))
        raw.append(mp.exp(-mp.mpf(float(u0[n]))) / den)
    C = mp.fsum(raw)
    expect = np.array([float(r / C) for r in raw])
    assert np.max(np.abs(O.reweight(u0, u, f, N_k) - expect)) < 1e-15


def test_mae():
    assert O.mae(np.array([0.0, 1.0, 2.0]), np.array([0.0, 1.5, 1.0])) == pytest.approx(0.5)


# ---------------------------------------------------------------------------
# uncertainty: asymptotic covariance of f
# ---------------------------------------------------------------------------

def test_covariance_of_identical_states_is_zero():
    """Two states with the same reduced potential: the estimate of
    f_1 - f_0 is exactly 0 for every sample, so its variance is 0."""
    g = np.random.default_rng(3)
    x = g.standard_normal(400)
    u = np.vstack([0.5 * x * x, 0.5 * x * x])
    Nk = np.array([150, 250])
    f = O.solve_mbar(u, Nk)
    C = O.mbar_covariance(u, f, Nk)
    assert C.shape == (2, 2) and abs(C[1, 1]) < 1e-12 and np.all(C[0] == 0.0)


def test_covariance_equals_reduced_inverse_hessian_minus_sample_terms():
    """The weight-matrix form equals the Hessian form
    inv(H_red) - diag(1/N_i) - 1/N_0 (H_red: the Hessian of the MBAR
    objective without state 0); symmetric and positive semi-definite."""
    p = W.harmonic(K=4, d=1, N_k=150, seed=2)
    f = O.solve_mbar(p.u_kn, p.N_k)
    C = O.mbar_covariance(p.u_kn, f, p.N_k)
    H = O.mbar_hessian(p.u_kn, f, p.N_k)
    Nk = p.N_k.astype(np.float64)
    ref = np.linalg.inv(H[1:, 1:]) - np.diag(1.0 / Nk[1:]) - 1.0 / Nk[0]
    assert np.allclose(C[1:, 1:], ref, rtol=1e-8, atol=1e-12)
    assert np.allclose(C, C.T, atol=1e-14)
    assert np.min(np.linalg.eigvalsh(C)) > -1e-12


def test_covariance_matches_repeated_sampling():
    """Large-sample theory against experiment: the covariance of f over 400
    independent samplings of three 1-D harmonic states agrees with the
    predicted one (the sampling error of a variance from 400 draws is ~7 %)."""
    kap = np.array([1.0, 1.5, 2.2])
    mu = np.array([0.0, 0.5, 1.0])
    Nk = np.array([200, 200, 200])
    g = np.random.default_rng(11)
    fs, pred = [], []
    for r in range(400):
        x = np.concatenate([mu[k] + g.standard_normal(Nk[k]) / np.sqrt(kap[k]) for k in range(3)])
        u = 0.5 * kap[:, None] * (x[None, :] - mu[:, None]) ** 2
        f = O.solve_mbar(u, Nk)
        fs.append(f[1:])
        if r < 8:
            pred.append(O.mbar_covariance(u, f, Nk)[1:, 1:])
    emp = np.cov(np.array(fs).T)
    th = np.mean(pred, axis=0)
    sd = np.sqrt(np.outer(np.diag(th), np.diag(th)))
    assert np.all(np.abs(np.diag(emp) / np.diag(th) - 1.0) < 0.3)
    assert np.all(np.abs(emp - th) < 0.3 * sd)
