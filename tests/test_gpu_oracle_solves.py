"""Whole solves through the C ABI against the oracle's MBAR root.

The roots are stored in tests/golden/solve_refs.json by
tests/golden/make_solve_refs.py, which calls only the oracle (its solves
take up to minutes on the host at these sizes). Each case is rebuilt here
from the same seeded generator, solved on the device, and compared element
by element: 1e-8 kT on the FP64 path, 1e-4 kT on the mixed path (the
mixed-precision and FP64 tolerances; Eq. 1 at its unbinned fixed point, Sec. II).

Cases:
  * the batched workload's problem types: umbrella windows on the double
    well and harmonic wells in d = 3, K from 4 to 256. Four umbrella
    windows 1.0 apart barely overlap: the gauge-reduced Hessian's smallest
    eigenvalue is 0.004-0.2, so a gradient bias of b moves the root by
    ~b / lambda_min. MIXED must still land within 1e-4 kT: each sample's
    largest weight is accumulated as an exact count plus its remainder;
  * the default benchmark's shapes at a reduced sample count: alchemical
    K = 500 (N_k = 20) and the tempering stand-in K = 50 (N_k = 2000). At
    K = 500 a MIXED solve runs the staging kernel with TMA loads, the
    one-launch first loop and the binned register passes with 32 lanes per
    sample, the 32-lane sample-major unbinned pass and the thread-block
    cluster tensor-core Hessian, i.e. the kernel instances the benchmark
    times at N = 2e6.
"""
import json
import os

import numpy as np
import pytest

from paper_2609_03541_b300 import mbar as M
from paper_2609_03541_b300 import workloads as W

pytestmark = pytest.mark.gpu

TOL = {M.MBAR_FP64: 1e-8, M.MBAR_MIXED: 1e-4}
HERE = os.path.dirname(os.path.abspath(__file__))


def _refs():
    with open(os.path.join(HERE, "golden", "solve_refs.json")) as fh:
        return {c["name"]: c for c in json.load(fh)["cases"]}


REFS = _refs()


def _problem(case):
    kind, args = case["kind"], case["args"]
    if kind == "umbrella":
        return W.umbrella(grid_points=1 << 13, **args)
    if kind == "harmonic":
        return W.harmonic(d=3, **args)
    if kind == "alchemical":
        return W.alchemical(**args)
    if kind == "parallel_tempering":
        return W.parallel_tempering(**args)
    raise ValueError(kind)


def _solve(p, prec):
    with M.Context(p.u_kn, p.N_k, prec) as ctx:
        if p.phi is not None:
            ctx.set_coordinate(p.phi)
        rep = ctx.solve().as_dict()
        return ctx.free_energies(), rep


BATCH_TYPES = [n for n in REFS if n.startswith(("umbrella", "harmonic"))]


@pytest.mark.parametrize("prec", [M.MBAR_FP64, M.MBAR_MIXED])
@pytest.mark.parametrize("name", BATCH_TYPES)
def test_batch_problem_types_match_the_oracle(name, prec):
    case = REFS[name]
    p = _problem(case)
    f, rep = _solve(p, prec)
    err = float(np.max(np.abs(f - np.asarray(case["f"]))))
    assert err < TOL[prec], (name, err, case["lambda_min"], rep)


def test_batched_solve_matches_the_oracle():
    """The same problems through mbar_batch_solve (MIXED, several admitted
    at once on the workers' streams)."""
    cases = [REFS[n] for n in BATCH_TYPES]
    probs = [_problem(c) for c in cases]
    cfg = M.server_config(workers=4, hbm_budget_bytes=8 << 30, precision=M.MBAR_MIXED)
    fs, reps, sts = M.batch_solve([(p.u_kn, p.N_k, p.phi) for p in probs], cfg)
    assert all(s == 0 for s in sts), sts
    for c, f in zip(cases, fs):
        assert np.max(np.abs(f - np.asarray(c["f"]))) < TOL[M.MBAR_MIXED], c["name"]


@pytest.mark.parametrize("prec", [M.MBAR_FP64, M.MBAR_MIXED])
@pytest.mark.parametrize("name", ["alchemical_K500", "tempering_K50"])
def test_bench_shapes_match_the_oracle(name, prec):
    case = REFS[name]
    p = _problem(case)
    f, rep = _solve(p, prec)
    err = float(np.max(np.abs(f - np.asarray(case["f"]))))
    assert err < TOL[prec], (name, err, rep)


@pytest.mark.parametrize("name", ["alchemical_K500", "tempering_K50"] + BATCH_TYPES[:4])
def test_exclusive_and_shared_device_loops_match_the_oracle(name):
    """MIXED solves with the device to themselves (the default: graphs, and
    the binned SCI steps of small levels in one cooperative launch over all
    SMs with the level in shared memory) and shared (mbar_set_exclusive(0):
    one 8-SM cluster or separate launches): both at the oracle's root within
    1e-4 kT."""
    case = REFS[name]
    p = _problem(case)
    f_ref = np.asarray(case["f"])
    for exclusive in (True, False):
        with M.Context(p.u_kn, p.N_k, M.MBAR_MIXED) as ctx:
            ctx.set_exclusive(exclusive)
            if p.phi is not None:
                ctx.set_coordinate(p.phi)
            rep = ctx.solve().as_dict()
            f = ctx.free_energies()
        err = float(np.max(np.abs(f - f_ref)))
        assert err < TOL[M.MBAR_MIXED], (name, exclusive, err, rep)


@pytest.mark.parametrize("name", ["umbrella_K4_s0", "umbrella_K4_s4", "umbrella_K4_s7"])
def test_mixed_gradient_keeps_small_weight_deficits(name):
    """At the oracle's root the exact gradient vanishes (~1e-12). A sample
    deep inside one window has weight 1 - r there with r far below the FP32
    spacing of 1; summed as FP32 terms close to 1 those deficits are lost and
    the gradient is biased by ~2.5e-4 (an FP32 emulation of that pass on
    these cases). With the largest weight split into an exact count plus
    -r / (1 + r) the MIXED gradient stays within 5e-5 of zero."""
    case = REFS[name]
    p = _problem(case)
    f_ref = np.asarray(case["f"])
    with M.Context(p.u_kn, p.N_k, M.MBAR_MIXED) as ctx:
        _, g, _ = ctx.sci_step(f_ref)
    assert np.max(np.abs(g)) < 5e-5, g


def test_persistent_batched_solve_matches_the_oracle():
    """mbar_batch_solve with MBAR_BATCH_PERSISTENT: the workers' first loops
    are queued to a batcher that runs whatever is queued in one persistent
    launch (one CTA per problem from a device queue); roots within the mixed
    tolerance, and each first loop takes the steps of the solve alone, to
    one step (its sums add in another order)."""
    cases = [REFS[n] for n in BATCH_TYPES]
    probs = [_problem(c) for c in cases]
    cfg = M.server_config(workers=4, hbm_budget_bytes=8 << 30, precision=M.MBAR_MIXED, persistent=True)
    fs, reps, sts = M.batch_solve([(p.u_kn, p.N_k, p.phi) for p in probs], cfg)
    assert all(s == 0 for s in sts), sts
    for c, p, f, r in zip(cases, probs, fs, reps):
        assert np.max(np.abs(f - np.asarray(c["f"]))) < TOL[M.MBAR_MIXED], c["name"]
        _, alone = _solve(p, M.MBAR_MIXED)
        assert r.iters_first_loop > 0
        assert abs(r.iters_first_loop - alone["iters_first_loop"]) <= 1, (c["name"], r.as_dict(), alone)


def test_persistent_batched_solve_under_a_tight_budget():
    """A budget of about two problems' footprints: admission keeps at most
    two solves on the device, so the batcher's launches carry one or two
    first loops each."""
    names = ["umbrella_K9", "umbrella_K17", "harmonic_K33", "umbrella_K64", "harmonic_K4"]
    cases = [REFS[n] for n in names]
    probs = [_problem(c) for c in cases]
    foot = max(M.footprint_bytes(len(p.N_k), int(p.N_k.sum())) for p in probs)
    cfg = M.server_config(workers=3, hbm_budget_bytes=int(2.2 * foot), precision=M.MBAR_MIXED, persistent=True)
    fs, reps, sts = M.batch_solve([(p.u_kn, p.N_k, p.phi) for p in probs], cfg)
    assert all(s == 0 for s in sts), sts
    for c, f in zip(cases, fs):
        assert np.max(np.abs(f - np.asarray(c["f"]))) < TOL[M.MBAR_MIXED], c["name"]
