"""Derives tests/golden/algorithm1_trace.json: the control-flow trace of
Algorithm 1 on a tiny problem, computed at 50 significant digits with
mpmath from the paper's printed formulas, independently of oracle/.

What it fixes (Sec. II, Eqs. 1-3, Algorithm 1, with n0 and inc scaled down
so that a K = 2, N = 300 problem passes through five refinements):
  * Eq. 1, one SCI step over the nonempty bins of the current width,
        f_i <- -log sum_p H_p e^{-u_ip} / sum_j N_j e^{f_j - u_jp},
    followed by the gauge f_0 = 0;
  * Eq. 2, s = max_i |f_new_i / f_old_i - 1| over states with f_old_i != 0
    (+inf if there are none: the first step from f = 0);
  * the first loop: SCI at n0 bins until s < eps;
  * the second loop: N_intermediate SCI steps, then one probe step at n
    (s_n) and one at n' = n inc (s_next) from the same f; Eq. 3 in the
    printed form s_n / n < 2 s_next / n' decides whether n <- n'
    (f <- f_next) or not (f <- f_new); after a raise the loop ends once
    2 inc n > sum_i N_i;
  * optionally the noise-floor rule of the reading for finite precision:
    a step whose max |f_new - f_old| is below the floor counts as converged
    at its level (the first loop stops; the second loop raises n).

Binning of a level with n bins uses the width procedure of the reading for
the width rule (largest w with g(w) >= n, by halving from R / n and then
geometric bisection, every operation rounded to nearest in binary64) and
the bin index floor((phi - min phi) / w) with the subtraction and the
division each rounded to nearest in binary64 (the reading for bin edges;
Python's float operations are exactly those). The bin representative is the
mean of the members' u.

Every recorded decision carries its margin: the relative gap between the
two sides of Eq. 3 (and between s and eps), so a check in binary64 cannot
fall on the other side by rounding.

Run from the repository root:  python tests/golden/derive_algorithm1_trace.py
"""
from __future__ import annotations

import json
import math
import os

import mpmath as mp
import numpy as np

mp.mp.dps = 50
HERE = os.path.dirname(os.path.abspath(__file__))

# tiny two-state problem: harmonic states of equal stiffness 1 centred at 0
# and 2.0, 150 exact Gaussian samples each, bin coordinate x
K, N_K, MU = 2, 150, (0.0, 2.0)
PARAMS = dict(n0=4, eps=1e-3, inc=2, n_intermediate=1)


def draw():
    g = np.random.Generator(np.random.Philox(2600))
    x = np.concatenate([MU[k] + g.standard_normal(N_K) for k in range(K)])
    u = np.stack([0.5 * (x - MU[k]) ** 2 for k in range(K)])
    return x, u


# --- Sec. II binning, as binary64 operations --------------------------------

def keys(phi, w):
    lo = min(phi)
    return [math.floor((p - lo) / w) for p in phi]


def g_of(phi, w):
    return len(set(keys(phi, w)))


def width(phi, n):
    R = max(phi) - min(phi)
    w_hi, w_lo = 2.0 * R, R / float(n)
    while g_of(phi, w_lo) < n:
        w_hi, w_lo = w_lo, w_lo * 0.5
    for _ in range(64):
        mid = math.sqrt(w_lo * w_hi)
        if not (w_lo < mid < w_hi):
            break
        if g_of(phi, mid) >= n:
            w_lo = mid
        else:
            w_hi = mid
    return w_lo


def level(phi, u, n):
    w = width(phi, n)
    ks = keys(phi, w)
    bins = sorted(set(ks))
    members = {b: [i for i, k in enumerate(ks) if k == b] for b in bins}
    H = [len(members[b]) for b in bins]
    ub = [[mp.fsum(mp.mpf(u[k][i]) for i in members[b]) / len(members[b]) for b in bins] for k in range(K)]
    return dict(n=n, w=w, H=H, u=ub, g=len(bins))


# --- Eqs. 1-2 at 50 digits ---------------------------------------------------

def sci(f, L, Nk):
    nb = len(L["H"])
    den = [mp.fsum(Nk[j] * mp.exp(f[j] - L["u"][j][p]) for j in range(K)) for p in range(nb)]
    fn = [-mp.log(mp.fsum(L["H"][p] * mp.exp(-L["u"][i][p]) / den[p] for p in range(nb))) for i in range(K)]
    return [x - fn[0] for x in fn]


def rel_step(fn, fo):
    r = [abs(a / b - 1) for a, b in zip(fn, fo) if b != 0]
    return max(r) if r else mp.inf


def run(phi, u, noise_floor=None):
    Nk = [N_K] * K
    N = sum(Nk)
    n0, eps, inc, nint = PARAMS["n0"], PARAMS["eps"], PARAMS["inc"], PARAMS["n_intermediate"]
    floor = mp.mpf(noise_floor) if noise_floor else None
    rows = []
    f = [mp.mpf(0)] * K
    cur = level(phi, u, n0)
    while True:
        fn = sci(f, cur, Nk)
        s = rel_step(fn, f)
        d = max(abs(a - b) for a, b in zip(fn, f))
        f = fn
        by_floor = floor is not None and d < floor
        stop = s < eps or by_floor
        margin = None if s == mp.inf else float(abs(s - eps) / eps)
        rows.append(dict(phase=1, n=cur["n"], s=float(s) if s != mp.inf else "inf", stop=stop,
                         eps_margin=margin, by_noise_floor=bool(by_floor and not s < eps)))
        if stop:
            break
    cur = level(phi, u, n0 * inc)
    nxt = level(phi, u, n0 * inc * inc)
    while True:
        for _ in range(nint):
            f = sci(f, cur, Nk)
        f_new = sci(f, cur, Nk)
        s_n = rel_step(f_new, f)
        f_next = sci(f, nxt, Nk)
        s_next = rel_step(f_next, f)
        lhs, rhs = s_n / cur["n"], 2 * s_next / nxt["n"]        # Eq. 3 as printed
        d = max(abs(a - b) for a, b in zip(f_new, f))
        by_floor = floor is not None and d < floor
        raise_n = lhs < rhs or by_floor
        rows.append(dict(phase=2, n=cur["n"], s_n=float(s_n), s_next=float(s_next), raise_n=bool(raise_n),
                         eq3_margin=float(abs(lhs - rhs) / max(lhs, rhs)),
                         by_noise_floor=bool(by_floor and not lhs < rhs)))
        if raise_n:
            f = f_next
            cur = nxt
            if 2 * inc * cur["n"] > N:                          # break rule of Algorithm 1
                break
            nxt = level(phi, u, cur["n"] * inc)
        else:
            f = f_new
    return rows, [float(x) for x in f]


def main():
    x, u = draw()
    phi = [float(v) for v in x]
    uu = [[float(v) for v in row] for row in u]
    rows, f = run(phi, uu)
    rows_nf, f_nf = run(phi, uu, noise_floor=2e-3)
    out = dict(
        citation="Algorithm 1 with Eqs. 1-3 (Sec. II), n0 and inc scaled down from 100 and 10; derived at 50 digits "
                 "by tests/golden/derive_algorithm1_trace.py (mpmath), independently of the oracle. Eq. 3 is applied "
                 "in its printed form s(f,n)/n < 2 s(f,n')/n'.",
        params=PARAMS, K=K, N_k=[N_K] * K, phi=phi, u=uu,
        trace=rows, f_end_of_loops=f,
        noise_floor=2e-3, trace_noise_floor=rows_nf, f_end_of_loops_noise_floor=f_nf,
    )
    with open(os.path.join(HERE, "algorithm1_trace.json"), "w") as fh:
        json.dump(out, fh, indent=1)
    for r in rows:
        print(r)
    print("noise floor:")
    for r in rows_nf:
        print(r)


if __name__ == "__main__":
    main()
