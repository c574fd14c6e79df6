"""LSE-pass autotuning (mbar_autotune_*): the search returns a compiled
shape that covers K, records it (and its cache line), and passes and solves
that take tuned shapes -- including a shape forced through the cache file
that the built-in rule never picks -- still match the oracle at the
tolerances of the untuned paths."""
import json
import os

import numpy as np
import pytest

import oracle as O
from paper_2609_03541_b300 import mbar as M
from paper_2609_03541_b300 import workloads as W

pytestmark = pytest.mark.gpu

HERE = os.path.dirname(os.path.abspath(__file__))


@pytest.fixture
def tuning(tmp_path):
    path = tmp_path / "tune.txt"
    M.autotune_clear()
    M.autotune_cache(path)
    yield path
    M.autotune_enable(False)
    M.autotune_cache(None)
    M.autotune_clear()


def _samples_pass(K, N, seed):
    import torch
    g = np.random.default_rng(seed)
    Nk = np.full(K, N // K, dtype=np.int64)
    Nk[: N - Nk.sum()] += 1
    u = g.uniform(0.0, 12.0, size=(K, N))
    f = g.uniform(-2.0, 2.0, size=K)
    f -= f[0]
    dev = torch.device("cuda")
    Kp = (K + 3) // 4 * 4
    v = torch.full((N, Kp), 7.0, dtype=torch.float32, device=dev)
    v[:, :K] = torch.from_numpy(np.ascontiguousarray(u.T)).to(dev, torch.float32)
    ft = torch.from_numpy(f).to(dev)
    lN = torch.from_numpy(np.log(Nk.astype(np.float64))).to(dev)
    Q = torch.empty(K, dtype=torch.float64, device=dev)
    logden = torch.empty(N, dtype=torch.float32, device=dev)
    scratch = torch.zeros(M.lse_samples_scratch_bytes(K, N), dtype=torch.uint8, device=dev)
    M.lse_pass_samples(v, K, ft, lN, Q, logden=logden, scratch=scratch)
    torch.cuda.synchronize()
    u32 = u.astype(np.float32).astype(np.float64)
    Q_ref = Nk * O.mbar_weights(u32, f, Nk).sum(axis=1)
    ld_ref = O.log_denominator(u32, f, Nk)
    return Q.cpu().numpy(), Q_ref, logden.cpu().numpy().astype(np.float64), ld_ref


def test_search_covers_K_and_is_cached(tuning):
    r = M.autotune_lse(M.TUNE_SAMPLES, 50, 1 << 18)
    assert r["cached"] == 0 and r["candidates"] >= 2
    assert 4 * r["lanes_per_sample"] * r["chunks_per_lane"] >= 64
    assert r["ms"] > 0 and r["heuristic_ms"] > 0
    assert r["ms"] <= 1.25 * r["heuristic_ms"]       # the rule's shape is among the candidates (timing noise aside)
    again = M.autotune_lse(M.TUNE_SAMPLES, 60, (1 << 18) + 5)  # same key: K 60 -> 64, same log2 n
    assert again["cached"] == 1 and again["lanes_per_sample"] == r["lanes_per_sample"]
    lines = tuning.read_text().split("\n")
    assert lines[0].split()[1:4] == ["0", "64", "18"]


def test_tuned_and_forced_shapes_match_the_oracle(tuning):
    K, N = 50, 1 << 18
    M.autotune_lse(M.TUNE_SAMPLES, K, N)
    dev_name = tuning.read_text().split()[0]
    # force the 32-lane shape with 32 KB stages (the rule picks 4 lanes for K = 50)
    with open(tuning, "a") as fh:
        fh.write(f"{dev_name} 0 64 18 32 3 512 32768 1 1.0 1.0\n")
    M.autotune_clear()
    M.autotune_cache(tuning)
    M.autotune_enable(True)
    r = M.autotune_lse(M.TUNE_SAMPLES, K, N)
    assert (r["lanes_per_sample"], r["chunks_per_lane"], r["cached"]) == (32, 3, 1)
    Q, Q_ref, ld, ld_ref = _samples_pass(K, N, seed=3)
    assert np.max(np.abs(Q - Q_ref) / Q_ref) < 1e-5
    assert np.max(np.abs(ld - ld_ref)) < 1e-4


def test_tuned_factorised_pass_matches_the_oracle(tuning):
    import torch
    K, N = 130, 1 << 17
    M.autotune_lse(M.TUNE_FACTORISED, K, N)
    M.autotune_enable(True)
    g = np.random.default_rng(9)
    a = g.uniform(-1, 1, K)
    b = np.linspace(0.5, 2.0, K)
    phi = g.uniform(-10, 0, N)
    Nk = np.full(K, N // K, dtype=np.int64)
    Nk[: N - Nk.sum()] += 1
    f = O.gauge(g.uniform(-3, 3, K))
    td = lambda x: torch.from_numpy(np.ascontiguousarray(x, dtype=np.float64)).cuda()
    Q = torch.empty(K, dtype=torch.float64, device="cuda")
    scratch = torch.zeros(M.lse_factorised_scratch_bytes(K, N), dtype=torch.uint8, device="cuda")
    M.lse_pass_factorised(td(a), td(b), td(phi), td(f), td(np.log(Nk.astype(np.float64))), Q, scratch=scratch)
    torch.cuda.synchronize()
    u = O.factorised_u(a, b, phi)
    Q_ref = Nk * O.mbar_weights(u, f, Nk).sum(axis=1)
    assert np.max(np.abs(Q.cpu().numpy() - Q_ref) / Q_ref) < 1e-5


def test_solve_with_tuned_shapes_reaches_the_oracle_root(tuning):
    with open(os.path.join(HERE, "golden", "solve_refs.json")) as fh:
        case = {c["name"]: c for c in json.load(fh)["cases"]}["harmonic_K130"]
    p = W.harmonic(d=3, **case["args"])
    M.autotune_lse(M.TUNE_SAMPLES, len(p.N_k), int(p.N_k.sum()))
    M.autotune_enable(True)
    with M.Context(p.u_kn, p.N_k, M.MBAR_MIXED) as ctx:
        rep = ctx.solve().as_dict()
        f = ctx.free_energies()
    assert np.max(np.abs(f - np.asarray(case["f"]))) < 1e-4, rep
