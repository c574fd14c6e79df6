"""Serving and batching (mbar_server_*, mbar_batch_solve): results against
the oracle, identity with the same problem solved alone, admission within
the memory budget with overlap on the device, and rejection of requests
that could never be admitted."""
import numpy as np
import pytest

import oracle as O
from paper_2609_03541_b300 import mbar as M
from paper_2609_03541_b300 import workloads as W

pytestmark = pytest.mark.gpu

TOL = {M.MBAR_FP64: 1e-8, M.MBAR_MIXED: 1e-4}


def _mix():
    """Uneven problems: (u_kn, N_k, phi, oracle f)."""
    probs = []
    for seed, K in enumerate([4, 8, 12]):
        p = W.harmonic(K=K, d=3, N_k=300 + 200 * seed, seed=seed)
        probs.append((p.u_kn, p.N_k, None))
    for seed, K in enumerate([10, 16]):
        p = W.umbrella(K=K, N_k=400, seed=seed, grid_points=1 << 12)
        probs.append((p.u_kn, p.N_k, p.phi))
    p = W.gaussian_overlap(M=6, N_0=1000, seed=3)
    probs.append((p.u_kn, p.N_k, p.phi))
    p = W.alchemical(K=20, N_k=200, seed=5)
    probs.append((p.u_kn, p.N_k, p.phi))
    return [(u, nk, phi, O.solve_mbar(u, nk)) for u, nk, phi in probs]


def _alone(u, nk, phi, prec):
    """The same solve alone, set up as a server worker sets up its contexts
    (a device shared with other solves: no graphs, cluster-sized loops)."""
    ctx = M.Context(u, nk, prec, opts=M.default_opts(prec))
    ctx.set_exclusive(False)
    if phi is not None:
        ctx.set_coordinate(phi)
    ctx.solve()
    f = ctx.free_energies()
    ctx.close()
    return f


@pytest.mark.parametrize("prec", [M.MBAR_FP64, M.MBAR_MIXED])
def test_server_results_equal_the_same_solves_alone(prec):
    mix = _mix()
    alone = [_alone(u, nk, phi, prec) for u, nk, phi, _ in mix]
    with M.Server(M.server_config(workers=4, hbm_budget_bytes=8 << 30, precision=prec)) as srv:
        ids = [srv.submit(u, nk, phi) for u, nk, phi, _ in mix]
        out = [srv.wait(i) for i in ids]
        st = srv.stats()
    assert st["completed"] == len(mix)
    assert st["peak_running"] >= 2          # requests were on the GPU together
    for (f, rep, lat, run), f1, (_, _, _, f_ref) in zip(out, alone, mix):
        assert np.array_equal(f, f1)        # same kernels, same order: identical bits
        assert np.max(np.abs(f - f_ref)) < TOL[prec]
        assert f[0] == 0.0
        assert lat >= run >= 0.0


def test_server_admission_keeps_within_the_budget():
    mix = _mix()
    prec = M.MBAR_MIXED
    foot = [M.footprint_bytes(len(nk), u.shape[1], prec) for u, nk, _, _ in mix]
    budget = int(2.2 * max(foot))            # at most about two at a time
    with M.Server(M.server_config(workers=6, hbm_budget_bytes=budget, precision=prec)) as srv:
        ids = [srv.submit(u, nk, phi) for u, nk, phi, _ in mix]
        states = [srv.poll(i) for i in ids]
        out = [srv.wait(i) for i in ids]
        st = srv.stats()
    assert all(s in (0, 1, 2) for s in states)
    assert st["peak_bytes"] <= budget
    assert st["completed"] == len(mix)
    for (f, _, _, _), (_, _, _, f_ref) in zip(out, mix):
        assert np.max(np.abs(f - f_ref)) < TOL[prec]


def test_server_rejects_a_request_larger_than_its_budget():
    p = W.harmonic(K=8, d=3, N_k=1000, seed=0)
    with M.Server(M.server_config(workers=2, hbm_budget_bytes=1 << 20)) as srv:
        with pytest.raises(M.MbarError) as e:
            srv.submit(p.u_kn, p.N_k)
    assert e.value.name == "MBAR_EUNSUPPORTED"


def test_server_reads_device_inputs():
    import torch
    mix = _mix()[:4]
    dev = [(torch.from_numpy(np.ascontiguousarray(u)).cuda(), nk,
            torch.from_numpy(np.ascontiguousarray(phi)).cuda() if phi is not None else None, f_ref)
           for u, nk, phi, f_ref in mix]
    with M.Server(M.server_config(workers=3, hbm_budget_bytes=4 << 30)) as srv:
        ids = [srv.submit(u, nk, phi) for u, nk, phi, _ in dev]
        out = [srv.wait(i) for i in ids]
    for (f, _, _, _), (_, _, _, f_ref) in zip(out, dev):
        assert np.max(np.abs(f - f_ref)) < TOL[M.MBAR_MIXED]


@pytest.mark.parametrize("prec", [M.MBAR_FP64, M.MBAR_MIXED])
def test_batch_solve_matches_the_oracle_and_the_single_solves(prec):
    mix = _mix()
    fs, reps, sts = M.batch_solve([(u, nk, phi) for u, nk, phi, _ in mix],
                                  M.server_config(workers=5, hbm_budget_bytes=8 << 30, precision=prec))
    assert sts == [0] * len(mix)
    for f, (u, nk, phi, f_ref) in zip(fs, mix):
        assert np.max(np.abs(f - f_ref)) < TOL[prec]
        assert np.array_equal(f, _alone(u, nk, phi, prec))


def test_server_tolerates_device_synchronisation_by_other_threads():
    """Workers never capture streams, so the caller's device-wide syncs
    (e.g. torch.cuda.synchronize while drawing the next inputs) do not fail
    and do not disturb the solves."""
    import torch
    mix = _mix()
    with M.Server(M.server_config(workers=4, hbm_budget_bytes=8 << 30)) as srv:
        ids = [srv.submit(u, nk, phi) for u, nk, phi, _ in mix]
        for _ in range(200):
            torch.cuda.synchronize()
            x = torch.ones(1 << 16, device="cuda")
            torch.cuda.synchronize()
            del x
        out = [srv.wait(i) for i in ids]
    for (f, _, _, _), (_, _, _, f_ref) in zip(out, mix):
        assert np.max(np.abs(f - f_ref)) < TOL[M.MBAR_MIXED]


def _factorised_mix():
    """Factorised requests of the serving stream's two kinds (umbrella
    windows with the per-sample terms dropped; the Sec. IV replicas,
    u = beta_k E), K from 5 to 700, with host copies for the oracle."""
    import torch
    out = []
    for kind, K, Nk, seed in [("umbrella", 5, 800, 11), ("gaussian", 9, 1000, 12), ("umbrella", 40, 300, 13),
                              ("gaussian", 130, 60, 14), ("umbrella", 700, 12, 15)]:
        if kind == "umbrella":
            a, b, phi, nk = W.umbrella_factorised_device(K, Nk, seed)
        else:
            b, phi, nk = W.gaussian_overlap_device(K, Nk, seed)
            a = torch.zeros_like(b)
        out.append((a, b, phi, nk))
    torch.cuda.synchronize()
    return out


def test_server_factorised_requests_equal_the_same_solves_alone():
    """mbar_server_submit_factorised: the store-free MIXED solves, several on
    the GPU together, give the bits of the same solves run alone, and the
    oracle's MBAR root within the mixed tolerance."""
    mix = _factorised_mix()
    prec = M.MBAR_MIXED
    alone = []
    for a, b, phi, nk in mix:
        with M.Context.factorised(a, b, phi, nk, prec) as ctx:
            ctx.set_exclusive(False)  # as the server's workers run them
            ctx.solve()
            alone.append(ctx.free_energies())
    with M.Server(M.server_config(workers=4, hbm_budget_bytes=8 << 30, precision=prec)) as srv:
        ids = [srv.submit_factorised(a, b, phi, nk) for a, b, phi, nk in mix]
        out = [srv.wait(i) for i in ids]
        st = srv.stats()
    assert st["completed"] == len(mix)
    assert st["peak_running"] >= 2
    for (f, rep, lat, run), f1, (a, b, phi, nk) in zip(out, alone, mix):
        assert np.array_equal(f, f1)
        u = O.factorised_u(a.cpu().numpy(), b.cpu().numpy(), phi.cpu().numpy())
        f_ref = O.solve_mbar(u, nk)
        assert np.max(np.abs(f - f_ref)) < TOL[prec], (len(nk), rep.as_dict())
