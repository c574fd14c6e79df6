#!/usr/bin/env python
"""BU-MBAR benchmark: MBAR solves per second on one B300 (per rank).

One step = one complete solve of a resident problem through the library's
C ABI: mbar_create (device FP64 u_kn -> per-sample-shifted FP32 store),
mbar_set_coordinate (radix sort by the bin coordinate), mbar_solve
(Algorithm 1 on the binned data, then Newton on the unbinned data: fused LSE
passes, tensor/CUDA-core Hessian, FP64 Cholesky) and mbar_free_energies.

Default workload: alchemical K=500 states, N_k=4000 (N=2e6, 1e9 entries of
u_kn, 8 GB in FP64 -- far larger than the 126 MB L2, so no flush is needed),
mixed precision. Prints one JSON line (rank 0).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                  [--workload alchemical|umbrella|harmonic]
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

WORKLOADS = {
    "alchemical": dict(K=500, N_k=4000, precision="mixed", h0=0.0,
                       desc="alchemical u_kn=u0_n+lambda_k*du_n, K=500, N_k=4000 (N=2e6, 1e9 entries), "
                            "du=20kT*t(nu=4), u0=-1e4+100N(0,1) kT, lambda_k=sin^2(pi k/2(K-1))"),
    "umbrella": dict(K=64, N_k=5000, precision="fp64", h0=0.1,
                     desc="1-D umbrella sampling on U(x)=5(x^2-1)^2, K=64 windows kappa=50 on [-1.5,1.5], "
                          "N_k=5000 (N=320k), FP64, bin schedule h=0.1->0"),
    "harmonic": dict(K=8, N_k=1000, precision="fp64", h0=0.0,
                     desc="K=8 harmonic states in d=3, N_k=1000 (N=8000), FP64"),
    "pt": dict(K=50, N_k=200_000, precision="mixed", h0=0.0,
               desc="parallel-tempering stand-in (Sec. III shape): K=50 temperatures 298-600 K exponentially "
                    "spaced, N_k=2e5 (N=1e7), Gaussian density of states, u_kn=b_k E_n, binned on E"),
}

PEAKS_FALLBACK = {"hbm_gbs": 6400.0, "bf16_tflops": 1800.0, "bf16_tflops_sustained": 1400.0}


def log(*a):
    print(*a, file=sys.stderr, flush=True)


def load_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        return d, "measured"
    return dict(PEAKS_FALLBACK), "fallback"


def make_problem(name: str, seed: int = 0, nk: int | None = None):
    from paper_2609_03541_b300 import workloads as W
    cfg = dict(WORKLOADS[name])
    if nk:
        cfg["N_k"] = nk
    if name == "alchemical":
        lam, u0, du, Nk = W.alchemical_factors(K=cfg["K"], N_k=cfg["N_k"], seed=seed)
        # factorised form (mbar_create_factorised): a = 0, b = lambda, phi = du;
        # the per-sample u0_n is dropped (a per-sample shift leaves f unchanged)
        return dict(kind=name, K=cfg["K"], N=int(Nk.sum()), N_k=Nk, phi=du,
                    rows=lambda k0, k1: W.alchemical_rows(lam, u0, du, k0, k1),
                    fact=(np.zeros(cfg["K"]), np.asarray(lam, dtype=np.float64), du))
    if name == "umbrella":
        p = W.umbrella(K=cfg["K"], N_k=cfg["N_k"], seed=seed)
    elif name == "pt":
        p = W.parallel_tempering(K=cfg["K"], N_k=cfg["N_k"], seed=seed)
    else:
        p = W.harmonic(K=cfg["K"], N_k=cfg["N_k"], seed=seed)
    u = p.u_kn
    fact = (np.zeros(p.K), p.meta["b"], p.phi) if name == "pt" else None   # u_kn = b_k E_n
    return dict(kind=name, K=p.K, N=p.N, N_k=p.N_k, phi=p.phi, rows=lambda k0, k1: u[k0:k1], fact=fact)


def fill_pinned(prob, torch):
    K, N = prob["K"], prob["N"]
    host = torch.empty((K, N), dtype=torch.float64, pin_memory=True)
    hv = host.numpy()
    step = max(1, (1 << 27) // N)
    for k0 in range(0, K, step):
        k1 = min(K, k0 + step)
        hv[k0:k1] = prob["rows"](k0, k1)
    return host


class ClockSampler:
    """nvidia-smi clocks/throttle sampler running during the timed region."""
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        import tempfile
        fd, self.path = tempfile.mkstemp(prefix=f"bumbar_clocks_gpu{gpu_index}_", suffix=".csv")
        os.close(fd)

    def __enter__(self):
        try:
            self.fh = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=self.fh, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None
        return self

    def __exit__(self, *exc):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()
            self.fh.close()

    def summary(self):
        out = {"sm_mhz": None, "sm_max_mhz": None, "reasons": []}
        try:
            rows = [r.split(",") for r in open(self.path).read().strip().splitlines() if r.strip()]
        except Exception:
            return out
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in rows:
            r = [x.strip() for x in r]
            if len(r) < 9:
                continue
            try:
                sm.append(float(r[1]))
                smax.append(float(r[2]))
            except ValueError:
                continue
            for nm, val in zip(names, r[5:9]):
                if val.lower() == "active":
                    reasons.add(nm)
        if sm:
            out["sm_mhz"] = statistics.median(sm)
            out["sm_max_mhz"] = max(smax)
            out["samples"] = len(sm)
        out["reasons"] = sorted(reasons)
        return out


# ---------------------------------------------------------------------------
# CPU oracle (baseline / reference arm)
# ---------------------------------------------------------------------------

# samples per state of the bounded sample the oracle solves end to end
REDUCED_NK = {"alchemical": 8, "umbrella": 200, "harmonic": 1000, "pt": 100}


def cpu_info():
    """CPU model, cores the process may use, and the thread count of the
    BLAS numpy calls (numpy's elementwise exp/log run on one thread)."""
    model = None
    try:
        with open("/proc/cpuinfo") as fh:
            for line in fh:
                if line.startswith("model name"):
                    model = line.split(":", 1)[1].strip()
                    break
    except OSError:
        pass
    try:
        cores = len(os.sched_getaffinity(0))
    except AttributeError:
        cores = os.cpu_count() or 1
    blas = None
    try:
        import threadpoolctl
        info = threadpoolctl.threadpool_info()
        blas = max((i.get("num_threads", 1) for i in info), default=None)
    except Exception:
        pass
    return {"cpu_model": model, "cores_available": cores, "blas_threads": blas}


def reduced_problem(name: str):
    """The bounded sample of a workload: all K states, REDUCED_NK samples each."""
    from paper_2609_03541_b300 import workloads as W
    cfg = WORKLOADS[name]
    K, nk = cfg["K"], REDUCED_NK[name]
    if name == "alchemical":
        return W.alchemical(K=K, N_k=nk, seed=1)
    if name == "umbrella":
        return W.umbrella(K=K, N_k=nk, seed=1, grid_points=1 << 14)
    if name == "pt":
        return W.parallel_tempering(K=K, N_k=nk, seed=1)
    return W.harmonic(K=K, N_k=nk, seed=1)


def oracle_solve_seconds(name: str, p, want_f: bool = False):
    """Time-to-solution of the oracle's Algorithm 1 + Newton finish on p
    (and its free energies if asked)."""
    import oracle as O
    opts = O.BUOptions(h0=WORKLOADS[name]["h0"])
    t0 = time.perf_counter()
    f = O.bu_mbar(p.u_kn, p.N_k, phi=p.phi, opts=opts)
    dt = time.perf_counter() - t0
    return (dt, f) if want_f else dt


def oracle_iteration_seconds(u_full: np.ndarray, N_k, chunk: int = 100_000):
    """One unbinned Eq. 1 iteration of the oracle over the full K x N matrix,
    chunked over samples: per chunk the oracle's log_denominator and its
    per-state log-sum-exp of -u - logden (the two sums of sci_step), then
    the chunks' per-state sums combined by the oracle's logsumexp and the
    gauge. Only the oracle calls are timed."""
    import oracle as O
    K, N = u_full.shape
    f = np.zeros(K)
    parts = []
    t = 0.0
    for c0 in range(0, N, chunk):
        u = np.ascontiguousarray(u_full[:, c0:c0 + chunk])
        t0 = time.perf_counter()
        ld = O.log_denominator(u, f, N_k)
        parts.append(O.logsumexp(-u - ld[None, :], axis=1))
        t += time.perf_counter() - t0
    t0 = time.perf_counter()
    O.gauge(-O.logsumexp(np.stack(parts, axis=0), axis=0))
    t += time.perf_counter() - t0
    return t


def cpu_baseline_block(name: str, p, u_full: np.ndarray | None, N_k, gpu_solve_s=None, gpu_iter_s=None):
    """The oracle, as it stands, on the host cores: its time-to-solution on
    the bounded sample p (the `value`, in solves/s of that sample, no
    scaling) and one unbinned Eq. 1 iteration over the full matrix. Returns
    (block, the oracle's free energies of p)."""
    solve_s, f_ref = oracle_solve_seconds(name, p, want_f=True)
    iter_s = oracle_iteration_seconds(u_full, N_k) if u_full is not None else None
    info = cpu_info()
    out = {"value": 1.0 / solve_s, "unit": "solves/s", "cores": info["cores_available"], "kind": "oracle",
           "sample": (f"time-to-solution of the oracle's Algorithm 1 + Newton finish on the bounded sample "
                      f"{name} K={p.K}, N_k={REDUCED_NK[name]} (N={p.N}, seed 1): value = solves/s of that sample; "
                      f"per_iteration_s = one unbinned Eq. 1 iteration over the full K x N matrix "
                      f"({u_full.shape[0]} x {u_full.shape[1]}, chunked over samples)" if u_full is not None else
                      f"time-to-solution of the oracle's Algorithm 1 + Newton finish on the bounded sample "
                      f"{name} K={p.K}, N_k={REDUCED_NK[name]} (N={p.N}, seed 1)"),
           "solve_s": solve_s, "solve_config": f"{name} K={p.K} N_k={REDUCED_NK[name]} N={p.N}",
           "per_iteration_s": iter_s, **info}
    if gpu_solve_s is not None:
        out["gpu_solve_s_same_config"] = gpu_solve_s
        out["solve_speedup_same_config"] = solve_s / gpu_solve_s
    if gpu_iter_s is not None and iter_s is not None:
        out["gpu_per_iteration_s"] = gpu_iter_s
        out["iteration_speedup_full_config"] = iter_s / gpu_iter_s
    return out, f_ref


# ---------------------------------------------------------------------------
# kernel-only timing of the fused LSE pass
# ---------------------------------------------------------------------------

def lse_only(args):
    """Times mbar_lse_pass on a resident K x n matrix (random reduced
    potentials) with CUDA events on the launching stream; prints one JSON
    line with the achieved bandwidth against the measured HBM peak."""
    import torch
    from paper_2609_03541_b300 import mbar as M
    dev = torch.device("cuda", 0)
    K, n = args.lse_K, args.lse_n
    dt = torch.float32 if args.lse_dtype == "float32" else torch.float64
    g = torch.Generator(device=dev)
    g.manual_seed(0)
    if args.lse_layout == "factorised":
        return lse_factorised_only(args)
    samples = args.lse_layout == "samples" and dt == torch.float32
    f = torch.linspace(-1, 1, K, device=dev, dtype=torch.float64)
    logN = torch.full((K,), float(np.log(n / K)), device=dev, dtype=torch.float64)
    Q = torch.empty(K, device=dev, dtype=torch.float64)
    logden = torch.empty(n, device=dev, dtype=dt)
    stream = torch.cuda.current_stream(dev)
    if samples:
        Kp = (K + 3) // 4 * 4
        v = torch.zeros((n, Kp), dtype=dt, device=dev)
        v[:, :K] = (3.0 * torch.randn((n, K), generator=g, device=dev, dtype=torch.float32)).abs()
        scratch = torch.zeros(M.lse_samples_scratch_bytes(K, n), dtype=torch.uint8, device=dev)

        def one():
            M.lse_pass_samples(v, K, f, logN, Q, logden=logden, scratch=scratch, stream=stream)
    else:
        ld = (n + 31) // 32 * 32
        v = torch.empty((K, ld), dtype=dt, device=dev)
        v[:, :n] = (3.0 * torch.randn((K, n), generator=g, device=dev, dtype=torch.float32)).abs().to(dt)
        vv = v[:, :n]
        scratch = torch.zeros(M.lse_scratch_bytes(K, n, v.element_size()), dtype=torch.uint8, device=dev)

        def one():
            M.lse_pass(vv, f, logN, Q, logden=logden, scratch=scratch, stream=stream)
    for _ in range(max(args.warmup, 1)):
        one()
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(args.steps):
        one()
    e1.record(stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / args.steps
    peaks, src = load_peaks()
    algo = K * n * v.element_size()
    gbs = algo / (ms / 1e3) / 1e9
    kname = "lse_smaj_kernel (sample-major FP32)" if samples else f"lse_pass (row-major {args.lse_dtype})"
    print(json.dumps({"kernel": kname, "K": K, "n": n, "ms_per_launch": ms,
                      "algorithmic_bytes": algo, "achieved_GBps": gbs, "peak_GBps": peaks["hbm_gbs"],
                      "frac": gbs / peaks["hbm_gbs"], "peak_source": src,
                      "entries_per_s": K * n / (ms / 1e3)}), flush=True)
    return 0


def lse_factorised_only(args):
    """Times mbar_lse_pass_factorised on tempering-shaped factorised
    potentials u_kp = b_k E_p (b_k = T_min / T_k over 298..600 K, E from a
    Gaussian density of states of variance 2000 kT^2, f at its analytic
    value) with CUDA events on the launching stream. The pass reads n * 8
    bytes and evaluates K * n exponentials: its roofline is the SFU rate,
    148 SMs x 16 ex2 per clock x the maximum SM clock."""
    import torch
    from paper_2609_03541_b300 import mbar as M
    dev = torch.device("cuda", 0)
    K, n = args.lse_K, args.lse_n
    # tempering magnitudes (|x| up to ~4e3: the exponents relative to each
    # sample's reference state) or, --lse-regime small, O(1) potentials (x
    # formed directly)
    s2 = 2000.0 if args.lse_regime == "tempering" else 2.0
    t = np.linspace(0.0, np.log(600.0 / 298.0), K)
    b = 1.0 / np.exp(t)
    g = torch.Generator(device=dev)
    g.manual_seed(0)
    bt = torch.from_numpy(b).to(dev)
    state = torch.arange(n, device=dev) % K
    phi = -bt[state] * s2 + np.sqrt(s2) * torch.randn(n, generator=g, device=dev, dtype=torch.float64)
    a = torch.zeros(K, device=dev, dtype=torch.float64)
    f = torch.from_numpy(-(b ** 2) * s2 / 2).to(dev)
    logN = torch.full((K,), float(np.log(n / K)), device=dev, dtype=torch.float64)
    Q = torch.empty(K, device=dev, dtype=torch.float64)
    logden = torch.empty(n, device=dev, dtype=torch.float64)
    scratch = torch.zeros(M.lse_factorised_scratch_bytes(K, n), dtype=torch.uint8, device=dev)
    stream = torch.cuda.current_stream(dev)

    def one():
        M.lse_pass_factorised(a, bt, phi, f, logN, Q, logden=logden, scratch=scratch, stream=stream)
    for _ in range(max(args.warmup, 1)):
        one()
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(args.steps):
        one()
    e1.record(stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / args.steps
    peaks, src = load_peaks()
    sms = torch.cuda.get_device_properties(dev).multi_processor_count
    peak = sms * 16 * peaks.get("sm_max_mhz", 2032.0) * 1e6     # ex2 per second
    eps = K * n / (ms / 1e3)
    print(json.dumps({"kernel": "lse_fact_kernel (u_kp = a_k + b_k phi_p, generated)", "K": K, "n": n,
                      "regime": args.lse_regime,
                      "ms_per_launch": ms, "bound": "alu (SFU ex2)", "entries_per_s": eps,
                      "peak_entries_per_s": peak, "frac": eps / peak,
                      "peak_source": f"{sms} SMs x 16 ex2/clk x {src} sm_max_mhz",
                      "bytes_read": n * 8, "Q_rel_spread": float((Q / Q.mean()).std())}), flush=True)
    return 0


def hess_only(args):
    """Times mbar_hessian on a random mixed-precision K x n problem (host
    f in, host K x K out); reports the library-timed Hessian launches.
    --hess-layout factorised: a store-free factorised context on a Sec. IV
    replica ladder (M = K replicas, n / K energies each, u = beta_k E) at
    the analytic f, whose Hessian forms P~ from E."""
    import torch
    from paper_2609_03541_b300 import mbar as M
    from paper_2609_03541_b300 import workloads as W
    K, n = args.lse_K, args.lse_n
    M.set_hessian_path(args.hess_path)
    if args.hess_layout == "factorised":
        beta, E, Nk = W.gaussian_overlap_device(K, max(1, n // K), seed=0)
        ctx = M.Context.factorised(torch.zeros_like(beta), beta, E, Nk, M.MBAR_MIXED)
        bb = beta.cpu().numpy()
        f = -(bb * bb - bb[0] * bb[0]) / 2.0
        ctx.set_timing(True)
        for _ in range(max(args.warmup, 1)):
            ctx.hessian(f)
        torch.cuda.synchronize()
        l0, ms0, _ = ctx.timing(1)
        t0 = time.perf_counter()
        for _ in range(args.steps):
            ctx.hessian(f)
        torch.cuda.synchronize()
        wall = (time.perf_counter() - t0) * 1e3 / args.steps
        l1, ms1, _ = ctx.timing(1)
        n_all = int(Nk.sum())
        dev_ms = (ms1 - ms0) / max(l1 - l0, 1)
        print(json.dumps({"kernel": "mbar_hessian, factorised context (overlap_tc_fact_kernel, P~ from E)",
                          "K": K, "n": n_all, "ms_per_call_wall": wall, "hessian_device_ms": dev_ms,
                          "tflops_upper_triangle": 2.0 * K * K * n_all * 0.5 / (dev_ms / 1e3) / 1e12}), flush=True)
        ctx.close()
        return 0
    g = np.random.default_rng(0)
    x = g.uniform(0, 1, size=n)
    centres = np.linspace(0, 1, K)
    u = torch.empty((K, n), dtype=torch.float64, device="cuda")
    for k0 in range(0, K, 64):
        k1 = min(K, k0 + 64)
        u[k0:k1] = torch.from_numpy(0.5 * (K * 0.8) ** 2 * (x[None, :] - centres[k0:k1, None]) ** 2).cuda()
    Nk = np.full(K, n // K, dtype=np.int64)
    Nk[: n - Nk.sum()] += 1
    ctx = M.Context(u, Nk, M.MBAR_MIXED)
    f = np.zeros(K)
    for _ in range(max(args.warmup, 1)):
        ctx.hessian(f)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        ctx.hessian(f)
    torch.cuda.synchronize()
    ms = (time.perf_counter() - t0) * 1e3 / args.steps
    print(json.dumps({"kernel": "mbar_hessian (LSE pass + overlap_tc + Laplacian)", "K": K, "n": n,
                      "ms_per_call_wall": ms, "flops_upper_triangle": 2.0 * K * K * n * 0.5}), flush=True)
    ctx.close()
    return 0


# ---------------------------------------------------------------------------
# main
# ---------------------------------------------------------------------------

def _gen_device(kind: str, K: int, Nk: int, seed: int):
    from paper_2609_03541_b300 import workloads as W
    if kind == "harmonic":
        return W.harmonic_device(K, Nk, seed)
    return W.umbrella_device(K, Nk, seed)


# Sec. IV: N_i = N_0, N_0 / M or N_0 / M^2 samples per replica, with N_0
# chosen so that every scenario has 1e4 samples per replica at M = 300
GAUSS_SCENARIOS = (("i", 1e4, 0), ("ii", 3e6, 1), ("iii", 9e8, 2))


def gaussian_bench(args):
    """The synthetic overlap study of Sec. IV: unit-variance normal energy
    histograms with 80 % overlap between neighbouring replicas, u_kn =
    beta_k E_n, in the paper's three scenarios for the samples per replica
    (N_0; N_0 / M; N_0 / M^2 with N_0 = 1e4, 3e6, 9e8). For each scenario and
    replica count M, `--seeds` seeded problems are drawn on the device, sent
    to mbar_create_factorised (E and beta only), solved (MIXED unless
    --precision fp64) and timed end to end on the device (create + solve +
    free energies + destroy, events on the stream, inputs resident); every
    solve is checked against the analytic f_k = -beta_k^2 / 2 + c within 5
    of its asymptotic standard deviations (mbar_covariance)."""
    import torch
    from paper_2609_03541_b300 import mbar as M
    from paper_2609_03541_b300 import workloads as W
    dev = torch.device("cuda", 0)
    torch.cuda.set_device(0)
    prec = M.MBAR_FP64 if args.precision == "fp64" else M.MBAR_MIXED
    stream = torch.cuda.current_stream(dev)
    Ms = [int(x) for x in args.gauss_M.split(",")]
    rows, worst_z, total_s, solves = [], 0.0, 0.0, 0
    for name, N0, power in GAUSS_SCENARIOS:
        for Mrep in Ms:
            N_i = int(round(N0 / Mrep ** power))
            times, zs, entries = [], [], Mrep * Mrep * N_i
            for seed in range(args.seeds):
                beta, E, Nk = W.gaussian_overlap_device(Mrep, N_i, seed=1000 * Mrep + seed, device=dev)
                a = torch.zeros_like(beta)
                torch.cuda.synchronize()
                e0 = torch.cuda.Event(enable_timing=True)
                e1 = torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                ctx = M.Context.factorised(a, beta, E, Nk, prec, stream=stream.cuda_stream)
                ctx.solve()
                f = ctx.free_energies()
                e1.record(stream)
                torch.cuda.synchronize()
                C = ctx.covariance()
                ctx.close()
                times.append(e0.elapsed_time(e1) / 1e3)
                b = beta.cpu().numpy()
                exact = -(b * b - b[0] * b[0]) / 2.0
                sd = np.sqrt(np.maximum(np.diag(C), 0.0))
                z = float(np.max(np.abs(f - exact)[1:] / sd[1:])) if Mrep > 1 else 0.0
                zs.append(z)
                del beta, E, a
            t_med = statistics.median(times)
            total_s += sum(times)
            solves += len(times)
            worst_z = max(worst_z, max(zs))
            rows.append({"scenario": name, "M": Mrep, "N_i": N_i, "N": Mrep * N_i, "entries": entries,
                         "seeds": args.seeds, "median_s": t_med, "solves_per_s": 1.0 / t_med,
                         "max_z": max(zs), "all_within_5_sigma": max(zs) < 5.0})
            log(f"[bench] gaussian {name} M={Mrep} N_i={N_i}: {t_med * 1e3:.2f} ms median, max z {max(zs):.2f}")
            torch.cuda.empty_cache()
    line = {"metric": "MBAR solves/sec (Sec. IV synthetic overlap scenarios)", "value": solves / total_s,
            "unit": "solves/s", "n_gpus": 1, "steps": solves, "warmup": 0, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32" if prec == M.MBAR_MIXED else "f64",
            "data": "synthetic",
            "config": {"workload": "gaussian overlap (Sec. IV): unit-variance normal energies, 80 % neighbour "
                                   "overlap, u_kn = beta_k E_n; N_i = N_0 (1e4), N_0/M (3e6), N_0/M^2 (9e8)",
                       "M": Ms, "seeds": args.seeds,
                       "step": "mbar_create_factorised + mbar_solve + mbar_free_energies + mbar_destroy",
                       "check": "|f_k - f_0 + (beta_k^2 - beta_0^2)/2| < 5 sd (asymptotic covariance)"},
            "scenarios": rows, "max_z": worst_z, "all_within_5_sigma": worst_z < 5.0}
    print(json.dumps(line), flush=True)
    return 0 if worst_z < 5.0 else 1


def batch_bench(args):
    """The batched workload as its own line (see batch_block)."""
    blk = batch_block(args)
    line = {"metric": "MBAR solves/sec (batched)", "value": blk["solves_per_s"], "unit": "solves/s", "n_gpus": 1,
            "steps": 1, "warmup": 0, "ms_per_step": blk["seconds"] * 1e3, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": blk["workload"], "problems": blk["problems"], "entries": blk["entries"],
                       "workers": args.workers, "budget_gb": args.budget_gb, "wave_input_gb": args.wave_gb},
            "how": blk["how"], "solves_per_s_per_problem_first_loops": blk["solves_per_s_per_problem_first_loops"],
            "solves_per_s_builtin_shapes": blk["solves_per_s_builtin_shapes"], "autotune": blk["autotune"],
            "persistent_first_loops": blk["persistent_first_loops"],
            "waves": blk["waves"], "accuracy": blk["accuracy"]}
    print(json.dumps(line), flush=True)
    return 0


def batch_block(args):
    """512 uneven problems (K ~ U{4..256}, N_k ~ U{100..10000} per problem,
    alternating harmonic d=3 / umbrella), mixed precision, solved by
    mbar_batch_solve in footprint waves: each wave's FP64 inputs are drawn on
    the device (untimed), then the wave's batch solve is timed (wall clock,
    device synchronised on both sides). The first wave is also solved on the
    plain FP64 path for the accuracy and speed comparison."""
    import torch
    from paper_2609_03541_b300 import mbar as M
    rng = np.random.default_rng(args.seed)
    P = args.problems
    specs = [("harmonic" if i % 2 == 0 else "umbrella", int(rng.integers(4, 257)), int(rng.integers(100, 10001)),
              1000 + i) for i in range(P)]
    wave_cap = int(args.wave_gb * (1 << 30))
    waves, cur, cur_b = [], [], 0
    for sp in specs:
        b = sp[1] * sp[1] * sp[2] * 8
        if cur and cur_b + b > wave_cap:
            waves.append(cur)
            cur, cur_b = [], 0
        cur.append(sp)
        cur_b += b
    if cur:
        waves.append(cur)
    cfg = M.server_config(workers=args.workers, hbm_budget_bytes=int(args.budget_gb * (1 << 30)),
                          precision=M.MBAR_MIXED)
    # autotuning (untimed): one search per key (K rounded up to a power of two,
    # floor(log2 N)) of the sample-major pass that MIXED's unbinned passes use
    tune_reps = {}
    for kind, K, Nk, seed in specs:
        kb = 4
        while kb < K:
            kb *= 2
        tune_reps.setdefault((kb, (K * Nk).bit_length() - 1), (K, K * Nk))
    t_tune = time.perf_counter()
    tuned = [M.autotune_lse(M.TUNE_SAMPLES, K, N) for K, N in tune_reps.values()]
    tune_info = {"keys": len(tuned), "search_s_untimed": time.perf_counter() - t_tune,
                 "keys_changed": sum(1 for r in tuned if r["ms"] < 0.97 * r["heuristic_ms"]),
                 "pass_time_ratio_tuned_over_rule": float(np.mean([r["ms"] / r["heuristic_ms"] for r in tuned]))}
    log(f"[bench] batch autotune: {tune_info}")
    total_s, total_rule_s, entries, wave_info = 0.0, 0.0, 0, []
    total_persistent_s, pers_df, pers_failed = 0.0, 0.0, 0
    cfg_persistent = M.server_config(workers=args.workers, hbm_budget_bytes=int(args.budget_gb * (1 << 30)),
                                     precision=M.MBAR_MIXED, persistent=True)
    acc = None
    for wi, wave in enumerate(waves):
        probs = []
        for kind, K, Nk, seed in wave:
            u, nk, phi = _gen_device(kind, K, Nk, seed)
            probs.append((u, nk, phi))
            entries += K * K * Nk
        # the built-in shapes, then the tuned ones, on the same inputs
        M.autotune_enable(False)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        M.batch_solve(probs, cfg)
        torch.cuda.synchronize()
        total_rule_s += time.perf_counter() - t0
        M.autotune_enable(True)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        fs, reps, sts = M.batch_solve(probs, cfg)
        torch.cuda.synchronize()
        dt = time.perf_counter() - t0
        # the same problems with every first loop of a budget group in one
        # persistent launch (MBAR_BATCH_PERSISTENT)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        fsp, _, stsp = M.batch_solve(probs, cfg_persistent)
        torch.cuda.synchronize()
        total_persistent_s += time.perf_counter() - t0
        M.autotune_enable(False)
        pers_df = max([pers_df] + [float(np.max(np.abs(a - b))) for a, b, s1, s2 in zip(fs, fsp, sts, stsp)
                                   if s1 == 0 and s2 == 0])
        pers_failed += sum(1 for s2 in stsp if s2 != 0)
        total_s += dt
        bad = [i for i, st in enumerate(sts) if st != 0]
        wave_info.append({"problems": len(wave), "seconds": dt, "failed": len(bad)})
        log(f"[bench] batch wave {wi}: {len(wave)} problems in {dt:.3f} s, failed {len(bad)}")
        slow = sorted(range(len(wave)), key=lambda i: -(reps[i].seconds_sci + reps[i].seconds_newton))[:3]
        for i in slow:
            kind, K, Nk, _ = wave[i]
            log(f"[bench]   slowest: {kind} K={K} N_k={Nk} " + json.dumps(reps[i].as_dict()))
        if wi == 0 and not args.no_accuracy:
            cfg64 = M.server_config(workers=args.workers, hbm_budget_bytes=int(args.budget_gb * (1 << 30)),
                                    precision=M.MBAR_FP64)
            torch.cuda.synchronize()
            t1 = time.perf_counter()
            f64, _, st64 = M.batch_solve(probs, cfg64)
            torch.cuda.synchronize()
            dt64 = time.perf_counter() - t1
            err = max(float(np.max(np.abs(a - b))) for a, b, s1, s2 in zip(fs, f64, sts, st64) if s1 == 0 and s2 == 0)
            acc = {"wave0_problems": len(wave), "max_abs_df_vs_fp64_gpu_kT": err, "fp64_wave0_s": dt64,
                   "mixed_wave0_s": dt, "mixed_speedup_vs_fp64_gpu": dt64 / dt}
        del probs, fs
        torch.cuda.empty_cache()
    return {"workload": "batched: 512 problems, K~U{4..256}, N_k~U{100..10000} per problem, harmonic d=3 / "
                        "umbrella alternating, mixed precision, mbar_batch_solve in footprint waves (inputs drawn "
                        "on the device before each wave's timing)",
            "problems": P, "entries": entries, "seconds": total_persistent_s,
            "solves_per_s": P / total_persistent_s,
            "how": "mbar_batch_solve with MBAR_BATCH_PERSISTENT and tuned LSE shapes: 16 workers run the solves; "
                   "their first loops are queued to a batcher that runs everything queued in one persistent "
                   "launch (device queue, one CTA per problem, level in shared memory)",
            "solves_per_s_per_problem_first_loops": P / total_s, "solves_per_s_builtin_shapes": P / total_rule_s,
            "autotune": tune_info,
            "persistent_first_loops": {"failed": pers_failed, "max_abs_df_vs_per_problem_path_kT": pers_df},
            "waves": wave_info, "accuracy": acc}


def serve_requests(R: int, seed: int, device):
    """The serving stream's R requests in factorised form, drawn on the
    device: K log-uniform on [4, 1024], N_k ~ U{100..20000}; even requests
    are umbrella windows on the double well (u = a_k + b_k x with the
    per-sample terms dropped, which leaves f unchanged), odd ones the Sec. IV
    replicas u = beta_k E (80 % neighbour overlap). Returns (requests,
    entries K * N summed, input bytes)."""
    import torch
    from paper_2609_03541_b300 import workloads as W
    rng = np.random.default_rng(seed)
    Ks = np.rint(np.exp(rng.uniform(np.log(4), np.log(1024), size=R))).astype(int)
    Nks = rng.integers(100, 20001, size=R)
    reqs, entries, nbytes = [], 0, 0
    for i in range(R):
        K, Nk = int(Ks[i]), int(Nks[i])
        if i % 2 == 0:
            a, b, phi, nk = W.umbrella_factorised_device(K, Nk, 5000 + i, device=device)
        else:
            b, phi, nk = W.gaussian_overlap_device(K, Nk, 5000 + i, device=device)
            a = torch.zeros_like(b)
        reqs.append((a, b, phi, nk))
        entries += K * K * Nk
        nbytes += (2 * K + K * Nk) * 8
    torch.cuda.synchronize()
    return reqs, entries, nbytes


class DeviceMemorySampler:
    """Samples the device's used memory (cudaMemGetInfo) every `period` s on
    a host thread; `peak` is the largest sample."""

    def __init__(self, period: float = 0.05):
        import threading
        self.period, self.peak, self._stop = period, 0, threading.Event()
        self._t = threading.Thread(target=self._run, daemon=True)

    def _run(self):
        import torch
        while not self._stop.is_set():
            free, total = torch.cuda.mem_get_info()
            self.peak = max(self.peak, total - free)
            self._stop.wait(self.period)

    def __enter__(self):
        self._t.start()
        return self

    def __exit__(self, *exc):
        self._stop.set()
        self._t.join()


def serve_run(reqs, workers: int, budget: int, rate, seed: int, persistent: bool = False):
    """One pass of the request stream through a fresh mbar_server (MIXED):
    at saturation (rate None: all submitted at once) or with Poisson
    arrivals at `rate` requests/s, each submitted at its arrival time.
    Latency is the server's own (submission to completion); the elapsed time
    runs from the first submission to the last completion."""
    from paper_2609_03541_b300 import mbar as M
    R = len(reqs)
    arr = np.cumsum(np.random.default_rng(seed).exponential(1.0 / rate, size=R)) if rate else np.zeros(R)
    cfg = M.server_config(workers=workers, hbm_budget_bytes=budget, precision=M.MBAR_MIXED, persistent=persistent)
    lat, failed, rejected = [], 0, 0
    phases = dict(width_s=0.0, levels_s=0.0, sci_s=0.0, newton_s=0.0, run_s=0.0, first_loop_iters=0,
                  second_loop_iters=0, newton_iters=0)
    slowest = []
    with DeviceMemorySampler() as mem:
        srv = M.Server(cfg)
        t0 = time.perf_counter()
        ids = []
        for i, (a, b, phi, nk) in enumerate(reqs):
            if rate:
                dt = t0 + arr[i] - time.perf_counter()
                if dt > 0:
                    time.sleep(dt)
            ts = time.perf_counter()
            try:
                ids.append((srv.submit_factorised(a, b, phi, nk), ts))
            except M.MbarError:
                rejected += 1
        t_end = t0
        for i, (rid, ts) in enumerate(ids):
            try:
                _, rep, l, run_s = srv.wait(rid)
            except M.MbarError as e:
                failed += 1
                log(f"[bench] serve: request {rid} failed: {e}")
                continue
            lat.append(l)
            t_end = max(t_end, ts + l)
            phases["width_s"] += rep.seconds_width
            phases["levels_s"] += rep.seconds_levels
            phases["sci_s"] += rep.seconds_sci
            phases["newton_s"] += rep.seconds_newton
            phases["run_s"] += run_s
            phases["first_loop_iters"] += rep.iters_first_loop
            phases["second_loop_iters"] += rep.iters_second_loop
            phases["newton_iters"] += rep.iters_newton
            slowest.append((run_s, i, len(reqs[i][3]), int(reqs[i][3][0]), rep.iters_first_loop,
                            rep.iters_second_loop, rep.iters_newton))
        st = srv.stats()
        srv.close()
    elapsed = t_end - t0
    done = len(lat)
    return {"completed": done, "rejected": rejected, "failed": failed, "elapsed_s": elapsed,
            "solves_per_s": done / elapsed if elapsed > 0 else 0.0,
            "offered_per_s": rate, "p50_ms": float(np.percentile(lat, 50) * 1e3) if lat else None,
            "p99_ms": float(np.percentile(lat, 99) * 1e3) if lat else None,
            "peak_running": st["peak_running"], "peak_admitted_gb": st["peak_bytes"] / 2 ** 30,
            "peak_device_used_gb": mem.peak / 2 ** 30,
            "worker_seconds": phases,
            "slowest": [dict(run_s=r, request=i, K=K, N_k=nk, first_loop=a, second_loop=b, newton=c)
                        for r, i, K, nk, a, b, c in sorted(slowest, reverse=True)[:8]]}


def serve_block(args, R: int, loads, poisson_requests: int | None = None):
    """Serving at the stream's full size: requests drawn before the timed
    runs (generation is not timed), one saturation run for the capacity,
    then Poisson runs at the given fractions of it for p50 / p99 (over the
    first `poisson_requests` of the stream, all by default)."""
    import torch
    dev = torch.device("cuda", 0)
    t0 = time.perf_counter()
    reqs, entries, nbytes = serve_requests(R, args.seed, dev)
    gen_s = time.perf_counter() - t0
    budget = int(args.budget_gb * (1 << 30))
    log(f"[bench] serve: {R} requests drawn in {gen_s:.1f} s ({nbytes / 2 ** 30:.1f} GB of inputs, "
        f"{entries:.3g} entries)")
    sat = serve_run(reqs, args.workers, budget, None, args.seed, args.serve_persistent)
    log(f"[bench] serve saturation: {sat}")
    loads_out = {}
    sub = reqs[:poisson_requests] if poisson_requests else reqs
    for frac in loads:
        loads_out[str(frac)] = serve_run(sub, args.workers, budget, frac * sat["solves_per_s"], args.seed + 1,
                                         args.serve_persistent)
        log(f"[bench] serve load {frac}: {loads_out[str(frac)]}")
    del reqs
    torch.cuda.empty_cache()
    return {"workload": "serving: K log-uniform [4,1024], N_k~U{100..20000}, factorised umbrella / Sec. IV replica "
                        "requests drawn before the timed runs, mixed precision, one mbar_server",
            "requests": R, "entries": entries, "input_gb": nbytes / 2 ** 30, "generation_s_untimed": gen_s,
            "budget_gb": args.budget_gb, "workers": args.workers, "saturation": sat,
            "poisson_requests": len(sub), "poisson": loads_out}


def serve_bench(args):
    """The serving stream (K log-uniform [4, 1024], N_k ~ U{100..20000},
    factorised requests, MIXED, memory budget) as its own line."""
    blk = serve_block(args, args.requests, args.loads)
    sat = blk["saturation"]
    line = {"metric": "MBAR solves/sec (served); p50/p99 latency", "value": sat["solves_per_s"], "unit": "solves/s",
            "n_gpus": 1, "steps": 1, "warmup": 0, "ms_per_step": sat["elapsed_s"] * 1e3, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": "serving: K log-uniform [4,1024], N_k~U{100..20000}, factorised umbrella / Sec. IV "
                                   "replica requests drawn before the timed runs, mixed precision",
                       "requests": args.requests, "workers": args.workers, "budget_gb": args.budget_gb},
            "serving": blk}
    print(json.dumps(line), flush=True)
    return 0 if sat["failed"] == 0 and sat["rejected"] == 0 else 1


def max_over_ranks(ms: float, dist, device) -> float:
    """Largest per-rank time (ms): the job's time is set by its slowest rank."""
    if dist is None:
        return ms
    import torch
    t = torch.tensor([ms], device=device, dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_rate(world: int, steps: int, ms_total: float) -> float:
    """Solves per second of the whole job: every rank solves `steps` problems
    of its own (replicas), all within the max-over-ranks time."""
    return world * steps / (ms_total / 1e3)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="alchemical", choices=list(WORKLOADS) + ["batch", "serve", "gaussian"])
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-accuracy", action="store_true")
    ap.add_argument("--no-extra", action="store_true",
                    help="skip the batched and served workloads that follow the headline line's timing")
    ap.add_argument("--precision", default=None, choices=["mixed", "fp64"],
                    help="override the workload's precision")
    ap.add_argument("--lse-only", action="store_true",
                    help="time only the stateless fused LSE pass (mbar_lse_pass) on a resident K x n matrix")
    ap.add_argument("--lse-K", type=int, default=500)
    ap.add_argument("--lse-n", type=int, default=2_000_000)
    ap.add_argument("--lse-dtype", default="float32", choices=["float32", "float64"])
    ap.add_argument("--lse-layout", default="samples", choices=["samples", "rows", "factorised"],
                    help="--lse-only: sample-major FP32 store (MIXED's unbinned passes), row-major, or "
                         "factorised u_kp = a_k + b_k phi_p generated from phi")
    ap.add_argument("--lse-regime", default="tempering", choices=["tempering", "small"],
                    help="--lse-layout factorised: tempering magnitudes (relative exponents) or O(1) potentials")
    ap.add_argument("--hess-layout", default="dense", choices=["dense", "factorised"],
                    help="--hess-only: a dense MIXED context, or a store-free factorised one")
    ap.add_argument("--hess-path", type=int, default=0, choices=[0, 1, 2, 3],
                    help="--hess-only: mbar_set_hessian_path (0 by size, 3 tensor cores without clusters)")
    ap.add_argument("--hess-only", action="store_true",
                    help="time mbar_hessian (one fused LSE pass + the tensor-core Hessian) on a random K x n problem")
    ap.add_argument("--problems", type=int, default=512, help="batch: number of problems")
    ap.add_argument("--requests", type=int, default=2000, help="serve: number of requests")
    ap.add_argument("--loads", type=lambda t: [float(x) for x in t.split(",") if x], default=[0.5, 0.9],
                    help="serve: Poisson arrival rates as fractions of the measured capacity")
    ap.add_argument("--workers", type=int, default=16, help="batch/serve: concurrent solves")
    ap.add_argument("--serve-persistent", action="store_true",
                    help="serve: the server batches its first loops into persistent launches")
    ap.add_argument("--budget-gb", type=float, default=None,
                    help="batch/serve: device memory budget of the server (default 140 batch, 160 serve)")
    ap.add_argument("--wave-gb", type=float, default=80.0, help="batch/serve: FP64 input memory held at once")
    ap.add_argument("--seed", type=int, default=0)
    ap.add_argument("--gauss-M", default="10,30,100,300", help="gaussian: replica counts M")
    ap.add_argument("--seeds", type=int, default=12, help="gaussian: seeds per (scenario, M) (the paper uses 12)")
    ap.add_argument("--nk", type=int, default=None,
                    help="samples per state override (smaller instances for profiling captures)")
    args = ap.parse_args()
    if args.budget_gb is None:
        args.budget_gb = 160.0 if args.workload in ("serve", "alchemical") else 140.0
    if args.workload == "batch":
        return batch_bench(args)
    if args.workload == "serve":
        return serve_bench(args)
    if args.workload == "gaussian":
        return gaussian_bench(args)
    if args.lse_only:
        return lse_only(args)
    if args.hess_only:
        return hess_only(args)

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))
    cfg = dict(WORKLOADS[args.workload])
    if args.precision:
        cfg["precision"] = args.precision
    if args.nk:   # a smaller instance of the workload (profiling captures); not the headline configuration
        cfg["N_k"] = args.nk
        cfg["desc"] += f" [N_k overridden to {args.nk}]"
    metric = "MBAR solves/sec"
    config = {"workload": cfg["desc"], "K": cfg["K"], "N": cfg["K"] * cfg["N_k"], "precision": cfg["precision"],
              "tolerance_kT": 1e-4 if cfg["precision"] == "mixed" else 1e-8,
              "l2": "inputs (K*N*8 bytes FP64 u_kn) larger than the 126 MB L2; no flush",
              "step": "mbar_create + mbar_set_coordinate + mbar_solve + mbar_free_energies + mbar_destroy"}

    if args.impl == "reference":
        # the oracle (numpy, as it stands) on the host cores; rank 0 only
        if rank != 0:
            return 0
        p = reduced_problem(args.workload)
        secs = []
        for i in range(args.warmup + args.steps):
            t = oracle_solve_seconds(args.workload, p)
            if i >= args.warmup:
                secs.append(t)
        med = statistics.median(secs)
        val = 1.0 / med
        info = cpu_info()
        sample = (f"each step: the oracle's Algorithm 1 + Newton finish on the bounded sample {args.workload} "
                  f"K={p.K}, N_k={REDUCED_NK[args.workload]} (N={p.N} of {config['N']} samples, seed 1); "
                  f"value = solves/s of that sample, not scaled to the full size")
        line = {"impl": "reference", "metric": metric, "value": val, "unit": "solves/s", "n_gpus": args.gpus,
                "steps": args.steps, "warmup": args.warmup, "ms_per_step": med * 1e3,
                "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
                "data": "synthetic", "config": config,
                "cpu_baseline": {"value": val, "unit": "solves/s", "cores": info["cores_available"],
                                 "kind": "oracle", "sample": sample, **info},
                "e2e": {"value": val, "unit": "solves/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
        print(json.dumps(line), flush=True)
        return 0

    import torch
    from paper_2609_03541_b300 import mbar as M

    dist = None
    if world > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local_rank)
        dist.init_process_group("nccl")
    torch.cuda.set_device(local_rank)
    dev = torch.device("cuda", local_rank)
    prec = M.MBAR_MIXED if cfg["precision"] == "mixed" else M.MBAR_FP64

    prob = make_problem(args.workload, seed=rank, nk=args.nk)
    t0 = time.time()
    host = fill_pinned(prob, torch)
    phi_host = torch.from_numpy(np.ascontiguousarray(prob["phi"])).pin_memory() if prob["phi"] is not None else None
    Nk = prob["N_k"]
    u_dev = host.to(dev, non_blocking=False)
    phi_dev = phi_host.to(dev) if phi_host is not None else None
    log(f"[bench] rank {rank}: problem K={prob['K']} N={prob['N']} ready in {time.time() - t0:.1f}s")
    stream = torch.cuda.current_stream(dev)
    opts = M.default_opts(prec, h0=cfg["h0"])

    traces = []

    def step(u, phi, timing=False, acc=None):
        ctx = M.Context(u, Nk, prec, opts=opts, stream=stream.cuda_stream)
        if timing:
            ctx.set_timing(True)
        if phi is not None:
            ctx.set_coordinate(phi)
        rep = ctx.solve()
        f = ctx.free_energies()
        traces.append(ctx.trace())
        if timing and acc is not None:
            for kind in (0, 1, 2, 3, 4, 5):
                n, ms, by = ctx.timing(kind)
                a = acc.setdefault(kind, [0, 0.0, 0.0])
                a[0] += n
                a[1] += ms
                a[2] += by
        ctx.close()
        return f, rep

    for i in range(args.warmup):
        f_w, rep_w = step(u_dev, phi_dev)
        log(f"[bench] warmup {i}: report {rep_w.as_dict()}")
    if traces:
        tr = traces[-1]
        log(f"[bench] solve trace ({len(tr)} rows: phase, n, a, b):")
        for row in tr[:40]:
            log("   " + " ".join(f"{x:.6g}" for x in row))

    def barrier():
        if dist is not None:
            dist.barrier()
        torch.cuda.synchronize(dev)

    # ---- timed region: resident inputs ----
    acc = {}
    launches0 = M.kernel_launches()
    with ClockSampler(local_rank) as clk:
        barrier()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        marks = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps + 1)]
        e0.record(stream)
        marks[0].record(stream)
        for i in range(args.steps):
            f_last, rep = step(u_dev, phi_dev, timing=True, acc=acc)
            marks[i + 1].record(stream)
        e1.record(stream)
        barrier()
    launches = M.kernel_launches() - launches0
    ms_total = max_over_ranks(e0.elapsed_time(e1), dist, dev)
    ms_per_step = ms_total / args.steps
    lat = sorted(marks[i].elapsed_time(marks[i + 1]) for i in range(args.steps))
    latency = {"p50_ms": float(np.percentile(lat, 50)), "p99_ms": float(np.percentile(lat, 99)),
               "min_ms": lat[0], "max_ms": lat[-1], "samples": len(lat)}
    value = whole_job_rate(world, args.steps, ms_total)
    clocks = clk.summary()

    # ---- end to end: host buffers through the C ABI ----
    e2e = None
    if not args.no_e2e:
        hbytes = prob["K"] * prob["N"] * 8 + (prob["N"] * 8 if phi_host is not None else 0)
        barrier()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(args.steps):
            step(host.numpy(), phi_host.numpy() if phi_host is not None else None)
        e1.record(stream)
        barrier()
        ms_e2e = max_over_ranks(e0.elapsed_time(e1), dist, dev)
        e2e = {"value": whole_job_rate(world, args.steps, ms_e2e), "unit": "solves/s",
               "h2d_bytes_per_step": hbytes, "d2h_bytes_per_step": prob["K"] * 8}

    # ---- end to end from the factorised form: 2K + N numbers cross the link ----
    e2e_fact = None
    if not args.no_e2e and prob.get("fact") is not None:
        fa, fb, fp = (torch.from_numpy(np.ascontiguousarray(x, dtype=np.float64)).pin_memory().numpy()
                      for x in prob["fact"])

        def fstep():
            ctx = M.Context.factorised(fa, fb, fp, Nk, prec, opts=opts, stream=stream.cuda_stream)
            ctx.solve()
            f = ctx.free_energies()
            ctx.close()
            return f
        f_fact = fstep()   # warm-up
        barrier()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(args.steps):
            fstep()
        e1.record(stream)
        barrier()
        ms_f = max_over_ranks(e0.elapsed_time(e1), dist, dev)
        e2e_fact = {"value": whole_job_rate(world, args.steps, ms_f), "unit": "solves/s",
                    "h2d_bytes_per_step": (2 * prob["K"] + prob["N"]) * 8, "d2h_bytes_per_step": prob["K"] * 8,
                    "api": "mbar_create_factorised (u_kn = a_k + b_k phi_n generated on the device)",
                    "max_abs_df_vs_timed_solve_kT": float(np.max(np.abs(f_fact - f_last)))}

    # ---- accuracy of the timed solve against the FP64 GPU path (outside timing) ----
    accuracy = None
    if prec == M.MBAR_MIXED and rank == 0 and not args.no_accuracy:
        o64 = M.default_opts(M.MBAR_FP64, h0=cfg["h0"])
        ctx = M.Context(u_dev, Nk, M.MBAR_FP64, opts=o64, stream=stream.cuda_stream)
        if phi_dev is not None:
            ctx.set_coordinate(phi_dev)
        t1 = time.time()
        ctx.solve()
        f64 = ctx.free_energies()
        ctx.close()
        t_fp64 = time.time() - t1
        accuracy = {"max_abs_df_vs_fp64_gpu_kT": float(np.max(np.abs(f_last - f64))),
                    "fp64_gpu_solve_s": t_fp64,
                    "mixed_speedup_vs_fp64_gpu": t_fp64 / (ms_per_step / 1e3)}

    # ---- reweighting to a target state (Eqs. 5-6), outside the timed region ----
    rew = None
    if rank == 0 and not args.no_accuracy:
        ctx = M.Context(u_dev, Nk, prec, opts=opts, stream=stream.cuda_stream)
        if phi_dev is not None:
            ctx.set_coordinate(phi_dev)
        ctx.solve()
        u0 = u_dev[prob["K"] // 2].contiguous()
        ctx.reweight(u0)                                  # warm-up
        torch.cuda.synchronize()
        t1 = time.perf_counter()
        reps = 5
        for _ in range(reps):
            pw, logc = ctx.reweight(u0)
        torch.cuda.synchronize()
        dt = (time.perf_counter() - t1) / reps
        ctx.close()
        rew = {"target": "state K/2", "ms_per_call": dt * 1e3, "samples_per_s": prob["N"] / dt,
               "sum_p": float(pw.sum()),
               "note": "one unbinned LSE pass + weights, N doubles copied to the host per call"}

    # ---- roofline of the dominant kernel (unbinned fused LSE pass) ----
    peaks, peaks_src = load_peaks()
    # every unbinned pass: the exact-split passes that drive Newton steps
    # (kind 0) and the plain ones that only confirm a step below f_tol (3)
    n_x, ms_x, by_x = acc.get(0, [0, 0.0, 0.0])
    n_c, ms_c, by_c = acc.get(3, [0, 0.0, 0.0])
    n_l, ms_l, by_l = n_x + n_c, ms_x + ms_c, by_x + by_c
    roofline = None
    if n_l:
        achieved = by_l / (ms_l / 1e3) / 1e9
        # DRAM bytes per launch: the algorithmic bytes times the read+write
        # ratio of one ncu capture of the same kernel instance and padding
        # (MIXED, K = 500: 32 lanes x 16 states, n = 4e5, 804.7 MB for 800.0 MB;
        # K = 50: 4 lanes x 16 states, Kp = 52, n = 4e6, 849.0 MB for 800.0 MB);
        # other K and FP64 not captured
        smaj = prec == M.MBAR_MIXED and prob["K"] <= 1024
        ratio = {500: 804.7 / 800.0, 50: 849.0 / 800.0}.get(prob["K"]) if smaj else None
        traffic = (by_l / n_l) * ratio if ratio else None
        roofline = {"bound": "hbm", "achieved": achieved, "peak": peaks["hbm_gbs"], "unit": "GB/s",
                    "frac": achieved / peaks["hbm_gbs"], "traffic": traffic,
                    # the library's layout rule: sample-major for every MIXED unbinned pass
                    "kernel": ("lse_smaj_kernel (unbinned passes, sample-major FP32)" if smaj
                               else "lse_regs_kernel (unbinned passes, row-major FP32)" if prec == M.MBAR_MIXED
                               else "lse_pass_kernel<double> (unbinned passes)"), "launches": n_l,
                    "avg_launch_ms": ms_l / n_l, "bytes_per_launch": by_l / n_l,
                    "peak_source": f"{peaks_src} hbm_gbs",
                    "variants": {
                        "exact_split": {"launches": n_x, "avg_launch_ms": (ms_x / n_x) if n_x else None,
                                        "frac": (by_x / (ms_x / 1e3) / 1e9 / peaks["hbm_gbs"]) if n_x else None},
                        "confirm_plain": {"launches": n_c, "avg_launch_ms": (ms_c / n_c) if n_c else None,
                                          "frac": (by_c / (ms_c / 1e3) / 1e9 / peaks["hbm_gbs"]) if n_c else None}}}
    n_h, ms_h, by_h = acc.get(1, [0, 0.0, 0.0])
    hess = {"launches": n_h, "avg_ms": (ms_h / n_h) if n_h else None}
    # the binned LSE passes of Algorithm 1: second-loop rounds (each N_int + 2
    # passes with their epilogues, graph-launched) and one-launch first loops;
    # achieved = the passes' algorithmic bytes / the rounds' device time
    binned = {}
    for kind, name in ((4, "second_loop_rounds"), (5, "first_loop")):
        n_b, ms_b, by_b = acc.get(kind, [0, 0.0, 0.0])
        if n_b:
            gbs = by_b / (ms_b / 1e3) / 1e9
            binned[name] = {"launches": n_b, "avg_ms": ms_b / n_b, "bytes_per_launch": by_b / n_b,
                            "achieved_GBps": gbs, "frac": gbs / peaks["hbm_gbs"]}
    # shares of the timed step: the LSE family's device time per step
    lse_ms = (ms_l + acc.get(4, [0, 0.0, 0.0])[1] + acc.get(5, [0, 0.0, 0.0])[1]) / args.steps
    binned["lse_family_ms_per_step"] = lse_ms
    binned["lse_family_share_of_step"] = lse_ms / ms_per_step

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu:
        # the GPU on the oracle's bounded sample (same precision and options;
        # resident input, median of 5 event-timed solves), then the oracle
        pr = reduced_problem(args.workload)
        u_red = torch.from_numpy(np.ascontiguousarray(pr.u_kn)).to(dev)
        phi_red = torch.from_numpy(np.ascontiguousarray(pr.phi)).to(dev) if pr.phi is not None else None
        t_red = []
        for i in range(6):
            a0 = torch.cuda.Event(enable_timing=True)
            a1 = torch.cuda.Event(enable_timing=True)
            a0.record(stream)
            ctx = M.Context(u_red, pr.N_k, prec, opts=opts, stream=stream.cuda_stream)
            if phi_red is not None:
                ctx.set_coordinate(phi_red)
            ctx.solve()
            f_red = ctx.free_energies()
            ctx.close()
            a1.record(stream)
            torch.cuda.synchronize()
            if i:
                t_red.append(a0.elapsed_time(a1) / 1e3)
        gpu_iter = (ms_x / n_x / 1e3) if n_x else ((ms_l / n_l / 1e3) if n_l else None)
        cpu, f_red_ref = cpu_baseline_block(args.workload, pr, host.numpy(), Nk,
                                            gpu_solve_s=statistics.median(t_red), gpu_iter_s=gpu_iter)
        if accuracy is None:
            accuracy = {}
        accuracy["max_abs_df_vs_oracle_kT"] = float(np.max(np.abs(f_red - f_red_ref)))
        accuracy["oracle_config"] = cpu["solve_config"]

    # ---- the batched and served workloads on this GPU (single-process runs only) ----
    batch_blk, serve_blk = None, None
    if world == 1 and not args.no_extra:
        torch.cuda.empty_cache()
        budget_gb = args.budget_gb
        args.budget_gb = 140.0
        batch_blk = batch_block(args)
        log(f"[bench] batch: {batch_blk['solves_per_s']:.1f} solves/s")
        args.budget_gb = 160.0
        serve_blk = serve_block(args, args.requests, [0.5], poisson_requests=500)
        args.budget_gb = budget_gb

    if rank == 0:
        line = {"metric": metric, "value": value, "unit": "solves/s", "n_gpus": world, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": ms_per_step, "higher_is_better": True, "scaling": "weak",
                "vs_baseline": None, "dtype": "f32" if prec == M.MBAR_MIXED else "f64", "data": "synthetic",
                "config": config, "e2e": e2e, "e2e_factorised": e2e_fact, "gpu_launches": launches,
                "roofline": roofline, "binned_lse": binned,
                "latency": latency, "hessian": hess, "cpu_baseline": cpu, "clocks": clocks, "accuracy": accuracy,
                "reweight": rew,
                "report": rep.as_dict(), "batch": batch_blk, "serving": serve_blk}
        print(json.dumps(line), flush=True)
    if dist is not None:
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
