"""Plain CPU FP64 oracle for the BU-MBAR hot path.

TEST INFRASTRUCTURE ONLY. Nothing in the product path may import this module:
only the tests, the smoke check and the benchmark's CPU-baseline / reference
leg use it. It shares no code with the CUDA library (no headers, helpers or
tables); both sides are fed the same seeded inputs and nothing else.

Everything here is a slow, direct transcription of the paper's definitions in
float64 numpy, in the paper's order and (generalised) notation:

  * u_kn   reduced potential of sample n in state k (the paper's beta_i E_p);
  * N_k    number of samples drawn in state k, N = sum_k N_k;
  * f_k    dimensionless free energies, gauge f_0 = 0;
  * H_p    bin counts (multiplicities), p over nonempty bins only.

Section map (BU-MBAR: Mueller, Alesiani, Christiansen):
  Eq. 1        sci_step            self-consistent (WHAM) update over n bins
  Sec. II      factorised_u        u_kp = a_k + b_k phi_p (the paper's beta_i E_p)
  Sec. II      bin_keys, histogram, nonempty_bins, width_for_bins, binned_u
  Eq. 2        relative_step
  Eq. 3 / Alg. 1  bu_mbar          binned-to-unbinned driver
  Sec. II      mbar_objective, mbar_gradient, mbar_hessian, newton_finish,
               solve_mbar          the unbinned MBAR/UWHAM limit and its
                                   derivative-based final phase (the paper names
                                   the switch; the derivatives are the standard
                                   ones of the convex MBAR objective)
  Eqs. 5-6     reweight            per-sample weights at a target state
  Eq. 7        mae
  (none)       mbar_covariance     asymptotic covariance of f (standard MBAR
                                   large-sample theory; the paper reports
                                   no error bars)

Pins (tests/test_oracle_pins.py) tie each function to something other than
itself: closed forms, Bennett's acceptance ratio for K = 2, a 40-digit
brute-force root of the MBAR equations, finite differences of the objective,
exact invariances and hand-derived binning fixtures. Functions without such a
pin would say "parity unpinned" here; at present none is unpinned.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

__all__ = [
    "logsumexp", "log_denominator", "factorised_u", "sci_step", "gauge", "relative_step",
    "mbar_weights", "mbar_objective", "mbar_gradient", "mbar_hessian",
    "newton_direction", "newton_finish", "solve_mbar",
    "bin_keys", "nonempty_bins", "histogram", "binned_u", "width_for_bins",
    "BUOptions", "bu_mbar", "reweight", "mbar_covariance", "mae",
]


# ---------------------------------------------------------------------------
# Eq. 1 and its pieces
# ---------------------------------------------------------------------------

def logsumexp(x: np.ndarray, axis: int) -> np.ndarray:
    """log(sum(exp(x))) along ``axis``, shifted by the maximum for range safety."""
    x = np.asarray(x, dtype=np.float64)
    m = np.max(x, axis=axis, keepdims=True)
    m = np.where(np.isfinite(m), m, 0.0)
    return np.squeeze(m, axis=axis) + np.log(np.sum(np.exp(x - m), axis=axis))


def log_denominator(u_kp: np.ndarray, f_k: np.ndarray, N_k: np.ndarray) -> np.ndarray:
    """Denominator of Eq. 1 in log form, one value per bin (or sample) p:

        logden_p = log sum_j N_j exp(f_j - u_jp).
    """
    u_kp = np.asarray(u_kp, dtype=np.float64)
    a = np.asarray(f_k, dtype=np.float64)[:, None] + np.log(np.asarray(N_k, dtype=np.float64))[:, None]
    return logsumexp(a - u_kp, axis=0)


def factorised_u(a_k: np.ndarray, b_k: np.ndarray, phi_p: np.ndarray) -> np.ndarray:
    """Reduced potentials of the factorised form the paper starts from
    (Sec. II: u_ip = beta_i E_p for samples with energy E_p at inverse
    temperatures beta_i), generalised by a per-state offset:

        u_kp = a_k + b_k phi_p.

    Every other function here takes the K x n matrix this returns.
    """
    a = np.asarray(a_k, dtype=np.float64)
    b = np.asarray(b_k, dtype=np.float64)
    phi = np.asarray(phi_p, dtype=np.float64)
    return a[:, None] + b[:, None] * phi[None, :]


def sci_step(u_kp: np.ndarray, f_k: np.ndarray, N_k: np.ndarray,
             H_p: np.ndarray | None = None) -> np.ndarray:
    """One self-consistent iteration, Eq. 1:

        f_i^{new} = -log sum_p  H_p exp(-u_ip) / sum_j N_j exp(f_j - u_jp)

    over the n columns p of u_kp (bins with counts H_p; H_p = 1 when the
    columns are individual samples, the UWHAM/MBAR limit of Sec. II).
    Returned without gauge fixing (see ``gauge``).
    """
    u_kp = np.asarray(u_kp, dtype=np.float64)
    n = u_kp.shape[1]
    logH = np.zeros(n) if H_p is None else np.log(np.asarray(H_p, dtype=np.float64))
    logden = log_denominator(u_kp, f_k, N_k)
    return -logsumexp(logH[None, :] - u_kp - logden[None, :], axis=1)


def gauge(f_k: np.ndarray) -> np.ndarray:
    """Fix the additive freedom of the equations by f_0 = 0."""
    f_k = np.asarray(f_k, dtype=np.float64)
    return f_k - f_k[0]


def relative_step(f_new: np.ndarray, f_old: np.ndarray) -> float:
    """Relative step width of Eq. 2, s = max_i |f_new_i / f_old_i - 1|.

    Reading for the division by zero the formula leaves open: entries with
    f_old_i == 0 (the gauge state, and every state on the first step from
    f = 0) are skipped; if no entry is left, s = +inf.
    """
    f_new = np.asarray(f_new, dtype=np.float64)
    f_old = np.asarray(f_old, dtype=np.float64)
    mask = f_old != 0.0
    if not np.any(mask):
        return math.inf
    return float(np.max(np.abs(f_new[mask] / f_old[mask] - 1.0)))


# ---------------------------------------------------------------------------
# The unbinned limit (UWHAM = MBAR) and its derivatives
# ---------------------------------------------------------------------------

def mbar_weights(u_kn: np.ndarray, f_k: np.ndarray, N_k: np.ndarray) -> np.ndarray:
    """W_kn = exp(f_k - u_kn) / sum_j N_j exp(f_j - u_jn) (K x N).

    At the solution sum_n W_kn = 1 for every k; for any f,
    sum_k N_k W_kn = 1 for every n.
    """
    u_kn = np.asarray(u_kn, dtype=np.float64)
    logden = log_denominator(u_kn, f_k, N_k)
    return np.exp(np.asarray(f_k, dtype=np.float64)[:, None] - u_kn - logden[None, :])


def mbar_objective(u_kn, f_k, N_k, H_n=None) -> float:
    """Convex function whose stationary points are the MBAR solutions:

        F(f) = sum_n H_n log sum_k N_k exp(f_k - u_kn) - sum_k N_k f_k.

    Its gradient vanishes exactly when Eq. 1 is at its fixed point.
    """
    logden = log_denominator(u_kn, f_k, N_k)
    H = np.ones_like(logden) if H_n is None else np.asarray(H_n, dtype=np.float64)
    return float(np.sum(H * logden) - np.dot(np.asarray(N_k, dtype=np.float64), f_k))


def mbar_gradient(u_kn, f_k, N_k, H_n=None) -> np.ndarray:
    """dF/df_k = sum_n H_n N_k W_kn - N_k."""
    W = mbar_weights(u_kn, f_k, N_k)
    Nk = np.asarray(N_k, dtype=np.float64)
    H = np.ones(W.shape[1]) if H_n is None else np.asarray(H_n, dtype=np.float64)
    return Nk * (W @ H) - Nk


def mbar_hessian(u_kn, f_k, N_k, H_n=None) -> np.ndarray:
    """d2F/df_k df_j = delta_kj sum_n H_n p_kn - sum_n H_n p_kn p_jn,
    with p_kn = N_k W_kn. Symmetric, positive semi-definite, and
    annihilates the all-ones vector (the gauge direction)."""
    W = mbar_weights(u_kn, f_k, N_k)
    Nk = np.asarray(N_k, dtype=np.float64)
    P = Nk[:, None] * W
    H = np.ones(W.shape[1]) if H_n is None else np.asarray(H_n, dtype=np.float64)
    return np.diag(P @ H) - (P * H[None, :]) @ P.T


def newton_direction(hess: np.ndarray, grad: np.ndarray) -> np.ndarray:
    """Gauge-fixed Newton step: drop state 0 and solve H_red d = -g_red by
    Cholesky (least squares if the reduced Hessian is not numerically
    positive definite). d_0 = 0."""
    K = grad.shape[0]
    d = np.zeros(K)
    if K == 1:
        return d
    Hr = hess[1:, 1:]
    gr = grad[1:]
    try:
        L = np.linalg.cholesky(Hr)
        y = np.linalg.solve(L, -gr)
        d[1:] = np.linalg.solve(L.T, y)
    except np.linalg.LinAlgError:
        d[1:] = np.linalg.lstsq(Hr, -gr, rcond=None)[0]
    return d


def newton_finish(u_kn, N_k, f_k, tol: float = 1e-12, max_iter: int = 100, trace=None):
    """Derivative-based final phase on unbinned data (Sec. II; Sec. III notes
    the method ends with quasi-Newton iterations on the unbinned equations).

    Each iteration takes the full Newton step when it lowers max|g|, otherwise
    one Eq. 1 step instead. Stops when the accepted Newton step is below
    ``tol`` in max norm (or the gradient is exactly zero).
    """
    f = gauge(f_k)
    g = mbar_gradient(u_kn, f, N_k)
    for it in range(max_iter):
        if not np.any(g):
            break
        H = mbar_hessian(u_kn, f, N_k)
        d = newton_direction(H, g)
        f_try = gauge(f + d)
        g_try = mbar_gradient(u_kn, f_try, N_k)
        if np.max(np.abs(g_try)) <= np.max(np.abs(g)):
            f, g = f_try, g_try
            if trace is not None:
                trace.append(("newton", it, float(np.max(np.abs(d)))))
            if np.max(np.abs(d)) < tol:
                break
        else:
            f = gauge(sci_step(u_kn, f, N_k))
            g = mbar_gradient(u_kn, f, N_k)
            if trace is not None:
                trace.append(("newton-fallback-sci", it, float("nan")))
    return f


def solve_mbar(u_kn, N_k, f_init=None, warm_tol: float = 1e-3, max_sci: int = 20000,
               tol: float = 1e-12) -> np.ndarray:
    """The MBAR solution by its plain definition: SCI (Eq. 1, unbinned) until
    max_k |sum_n W_kn - 1| < warm_tol, then Newton to ``tol``."""
    u_kn = np.asarray(u_kn, dtype=np.float64)
    K = u_kn.shape[0]
    f = np.zeros(K) if f_init is None else gauge(f_init)
    Nk = np.asarray(N_k, dtype=np.float64)
    for _ in range(max_sci):
        g = mbar_gradient(u_kn, f, N_k)
        if np.max(np.abs(g / Nk)) < warm_tol:
            break
        f = gauge(sci_step(u_kn, f, N_k))
    return newton_finish(u_kn, N_k, f, tol=tol)


# ---------------------------------------------------------------------------
# Binning (Sec. II): uniform width, nonempty bins only
# ---------------------------------------------------------------------------

def bin_keys(phi: np.ndarray, phi_lo: float, w: float) -> np.ndarray:
    """Bin index of each sample, b_n = floor((phi_n - phi_lo) / w), with the
    subtraction and the division each rounded to nearest in IEEE binary64
    (numpy evaluates them as two separate correctly rounded operations)."""
    phi = np.asarray(phi, dtype=np.float64)
    q = (phi - np.float64(phi_lo)) / np.float64(w)
    return np.floor(q).astype(np.int64)


def nonempty_bins(phi: np.ndarray, w: float) -> int:
    """g(w): the number of nonempty bins of uniform width w anchored at min(phi)."""
    phi = np.asarray(phi, dtype=np.float64)
    return int(np.unique(bin_keys(phi, phi.min(), w)).shape[0])


@dataclass
class Histogram:
    w: float
    keys: np.ndarray        # sorted distinct bin indices, one per nonempty bin
    H: np.ndarray           # int64 counts, H_p >= 1
    members: list = field(default_factory=list)   # sample indices of each bin


def histogram(phi: np.ndarray, w: float) -> Histogram:
    """Nonempty bins of width w: distinct keys in increasing order, their
    counts H_p, and the samples in each bin."""
    phi = np.asarray(phi, dtype=np.float64)
    keys = bin_keys(phi, phi.min(), w)
    uniq, inverse, counts = np.unique(keys, return_inverse=True, return_counts=True)
    members = [[] for _ in range(uniq.shape[0])]
    for n, b in enumerate(inverse):
        members[b].append(n)
    return Histogram(w=float(w), keys=uniq, H=counts.astype(np.int64),
                     members=[np.asarray(m, dtype=np.int64) for m in members])


def binned_u(u_kn: np.ndarray, hist: Histogram) -> np.ndarray:
    """Reduced potential of each nonempty bin p in every state: the mean of
    u_kn over the bin's members (the bin's representative point)."""
    u_kn = np.asarray(u_kn, dtype=np.float64)
    out = np.empty((u_kn.shape[0], len(hist.members)))
    for p, m in enumerate(hist.members):
        out[:, p] = np.sum(u_kn[:, m], axis=1) / np.float64(m.shape[0])
    return out


WIDTH_SEARCH_MAX_INDEX = 2.0 ** 52
WIDTH_SEARCH_BISECTIONS = 64


def width_for_bins(phi: np.ndarray, n: int) -> float | None:
    """w*(n) = max{w : n <= g(w)} (Sec. II) by a deterministic search.

    g is not monotone, so the maximum is taken along this fixed procedure:
      R = max(phi) - min(phi); if n <= 1 or R == 0 the answer is 2R (one bin);
      w_hi = 2R (g = 1), w_lo = R / n;
      while g(w_lo) < n: w_hi = w_lo, w_lo = w_lo / 2, giving up (None =
                         unbinned) once R / w_lo > 2^52, where bin indices
                         stop being exact integers in binary64;
      up to 64 times: mid = sqrt(w_lo * w_hi) (each op rounded to nearest);
                      stop if mid is not strictly between them;
                      if g(mid) >= n: w_lo = mid else w_hi = mid;
      answer w_lo.
    Returns None when n exceeds the number of distinct bins reachable (the
    caller then uses the unbinned data).
    """
    phi = np.asarray(phi, dtype=np.float64)
    R = float(phi.max() - phi.min())
    if n <= 1 or R == 0.0:
        return 2.0 * R if R > 0.0 else 1.0
    w_hi = 2.0 * R
    w_lo = R / float(n)
    while True:
        if R / w_lo > WIDTH_SEARCH_MAX_INDEX:
            return None
        if nonempty_bins(phi, w_lo) >= n:
            break
        w_hi = w_lo
        w_lo = w_lo * 0.5
    for _ in range(WIDTH_SEARCH_BISECTIONS):
        mid = math.sqrt(w_lo * w_hi)
        if not (w_lo < mid < w_hi):
            break
        if nonempty_bins(phi, mid) >= n:
            w_lo = mid
        else:
            w_hi = mid
    return w_lo


# ---------------------------------------------------------------------------
# Algorithm 1: binned-to-unbinned driver
# ---------------------------------------------------------------------------

@dataclass
class BUOptions:
    """Hyperparameters of Algorithm 1, defaults from Sec. II (n0 = 100,
    eps = 1e-3, inc = 10, N_intermediate = 20). ``h0`` > 0 switches to an
    explicit width schedule h0, h0/inc, h0/inc^2, ... instead of w*(n).
    ``noise_floor`` > 0 treats an SCI step with max|delta f| below it as
    converged at its level (first loop stops, second loop raises n); 0 runs
    Eqs. 2-3 exactly as printed."""
    n0: int = 100
    eps: float = 1e-3
    inc: int = 10
    n_intermediate: int = 20
    h0: float = 0.0
    newton_tol: float = 1e-12
    max_phase1: int = 100000
    max_rounds: int = 100000
    noise_floor: float = 0.0


@dataclass
class Level:
    n: int                  # target number of nonempty bins (n-schedule) or g(h) (h-schedule)
    w: float | None         # width; None = unbinned
    u: np.ndarray
    H: np.ndarray | None


def _level(u_kn, phi, n_target, w):
    if w is None:
        return Level(n=u_kn.shape[1], w=None, u=u_kn, H=None)
    hist = histogram(phi, w)
    return Level(n=n_target if n_target is not None else hist.H.shape[0], w=w,
                 u=binned_u(u_kn, hist), H=hist.H)


def bu_mbar(u_kn, N_k, phi=None, opts: BUOptions | None = None, trace: list | None = None):
    """Algorithm 1 (BU-MBAR) followed by the unbinned derivative-based finish.

    Readings where the paper leaves a choice:
      * SCI(f, n) is one Eq. 1 step on the n-bin histogram;
      * every step is gauge fixed (f_0 = 0) and s follows ``relative_step``;
      * after the probes of the second loop, f takes f_next when n is raised
        and f_new otherwise (the listing computes both but assigns neither);
      * the bin coordinate defaults to row 0 of u_kn;
      * a level whose width search fails (more bins requested than distinct
        values allow) is the unbinned data.
    Returns the gauge-fixed f; ``trace`` (if given) receives (phase, n, s, s_next).
    """
    opts = opts or BUOptions()
    u_kn = np.asarray(u_kn, dtype=np.float64)
    K, Ntot = u_kn.shape
    Nk = np.asarray(N_k, dtype=np.int64)
    phi = u_kn[0] if phi is None else np.asarray(phi, dtype=np.float64)
    N = int(Nk.sum())
    inc = opts.inc
    R = float(phi.max() - phi.min())

    def level(idx):
        # idx-th level of the schedule
        if opts.h0 > 0.0:
            w = opts.h0 / float(inc) ** idx
            if R / w > WIDTH_SEARCH_MAX_INDEX:
                w = None
            return _level(u_kn, phi, None, w)
        n_target = opts.n0 * inc ** idx
        return _level(u_kn, phi, n_target, width_for_bins(phi, n_target))

    f = np.zeros(K)
    lvl_idx = 0
    cur = level(lvl_idx)
    # first loop: SCI at n0 until s < eps
    for _ in range(opts.max_phase1):
        f_new = gauge(sci_step(cur.u, f, Nk, cur.H))
        s = relative_step(f_new, f)
        f_prev, f = f, f_new
        if trace is not None:
            trace.append(("phase1", cur.n, s, None))
        if s < opts.eps or (opts.noise_floor > 0 and np.max(np.abs(f - f_prev)) < opts.noise_floor):
            break
    lvl_idx += 1
    cur = level(lvl_idx)
    if cur.w is not None:            # second loop (an unbinned level has nothing left to refine)
        nxt = level(lvl_idx + 1)
        for _ in range(opts.max_rounds):
            for _ in range(opts.n_intermediate):
                f = gauge(sci_step(cur.u, f, Nk, cur.H))
            f_new = gauge(sci_step(cur.u, f, Nk, cur.H))
            s_n = relative_step(f_new, f)
            f_next = gauge(sci_step(nxt.u, f, Nk, nxt.H))
            s_next = relative_step(f_next, f)
            if trace is not None:
                trace.append(("phase2", cur.n, s_n, s_next))
            floor_hit = opts.noise_floor > 0 and np.max(np.abs(f_new - f)) < opts.noise_floor
            if 2.0 * s_next > inc * s_n or floor_hit:
                f = f_next
                lvl_idx += 1
                cur = nxt
                if cur.w is None or 2 * inc * cur.n > N:
                    break
                nxt = level(lvl_idx + 1)
            else:
                f = f_new
    return newton_finish(u_kn, Nk, f, tol=opts.newton_tol, trace=trace)


# ---------------------------------------------------------------------------
# Eqs. 5-7: reweighting and the error measure of Fig. 2
# ---------------------------------------------------------------------------

def reweight(u0_n: np.ndarray, u_kn: np.ndarray, f_k: np.ndarray, N_k: np.ndarray) -> np.ndarray:
    """Statistical weight of every sample at a target state with reduced
    potential u0_n (beta_0 E_n in the paper), Eqs. 5-6:

        p_n = (1/C) exp(-u0_n) / sum_m N_m exp(f_m - u_mn),  C = sum_n (unnormalised p_n).
    """
    logden = log_denominator(u_kn, f_k, N_k)
    logp = -np.asarray(u0_n, dtype=np.float64) - logden
    return np.exp(logp - logsumexp(logp, axis=0))


# ---------------------------------------------------------------------------
# Uncertainty: asymptotic covariance of the free energies (not in the paper;
# the standard output of an MBAR solve)
# ---------------------------------------------------------------------------

def mbar_covariance(u_kn: np.ndarray, f_k: np.ndarray, N_k: np.ndarray) -> np.ndarray:
    """Asymptotic covariance of the estimated free energies at the solution
    f_k, in the gauge f_0 = 0: entry (i, j) is cov(f_i - f_0, f_j - f_0).

    Written as the weight-matrix form of the MBAR large-sample theory: with
    the N x K matrix W (W_nk = exp(f_k - u_kn) / sum_j N_j exp(f_j - u_jn))
    and N = diag(N_k),

        Theta = W^T (I_N - W N W^T)^+ W,

    and cov(f_i - f_0, f_j - f_0) = Theta_ij - Theta_i0 - Theta_0j + Theta_00.
    The N x N pseudo-inverse is formed explicitly (numpy.linalg.pinv), so this
    is for small N only.
    """
    Wt = mbar_weights(u_kn, f_k, N_k).T                     # N x K
    Nd = np.diag(np.asarray(N_k, dtype=np.float64))
    A = np.eye(Wt.shape[0]) - Wt @ Nd @ Wt.T
    theta = Wt.T @ np.linalg.pinv(A, rcond=1e-10, hermitian=True) @ Wt
    d = theta - theta[:, :1] - theta[:1, :] + theta[0, 0]
    d[0, :] = 0.0
    d[:, 0] = 0.0
    return d


def mae(f_ref: np.ndarray, f: np.ndarray) -> float:
    """Mean absolute error of Eq. 7."""
    return float(np.mean(np.abs(np.asarray(f_ref) - np.asarray(f))))
