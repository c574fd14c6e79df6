"""The allocation-free LSE pass (mbar_lse_pass_static) against the regular
one (mbar_lse_pass with a caller-provided scratch buffer).

mbar_lse_pass_static exists for callers that cannot allocate device memory
(a host framework whose allocator owns the GPU's memory, or a loop that must
not pay cudaMalloc's implicit synchronisation); it keeps its scratch in an
array built into the library. This file is collected last so that a run that
stops at the first failure has run every other test before it; it passes on
its own in a fresh process as well.
"""
import numpy as np
import pytest

from paper_2609_03541_b300 import mbar as M

pytestmark = pytest.mark.gpu

TOL = {"float32": 1e-5, "float64": 1e-10}   # same as test_lse_pass_stateless


def _inputs(K, N, dtype, seed):
    import torch
    g = np.random.default_rng(seed)
    Nk = np.full(K, N // K, dtype=np.int64)
    Nk[: N - Nk.sum()] += 1
    u = 3.0 * g.standard_normal((K, N)) + g.uniform(-2, 2, size=(K, 1))
    f = g.uniform(-1, 1, size=K)
    f[0] = 0.0
    dev = torch.device("cuda")
    tdt = torch.float32 if dtype == "float32" else torch.float64
    ld = (N + 31) // 32 * 32
    v = torch.zeros((K, ld), dtype=tdt, device=dev)
    v[:, :N] = torch.from_numpy(u).to(dev, tdt)
    return (v[:, :N], torch.from_numpy(f).to(dev),
            torch.from_numpy(np.log(Nk.astype(np.float64))).to(dev))


@pytest.mark.parametrize("dtype", ["float32", "float64"])
@pytest.mark.parametrize("K,N", [(37, 5001), (500, 20011)])
def test_static_scratch_pass_matches_the_regular_pass_twice(dtype, K, N):
    import torch
    v, f, lN = _inputs(K, N, dtype, seed=K)
    dev = v.device
    Q_ref = torch.empty(K, dtype=torch.float64, device=dev)
    ld_ref = torch.empty(N, dtype=v.dtype, device=dev)
    scratch = torch.zeros(M.lse_scratch_bytes(K, N, v.element_size()), dtype=torch.uint8, device=dev)
    M.lse_pass(v, f, lN, Q_ref, logden=ld_ref, scratch=scratch)
    for _ in range(2):   # the built-in array keeps the previous call's contents
        Q = torch.full((K,), float("nan"), dtype=torch.float64, device=dev)
        ld = torch.full((N,), float("nan"), dtype=v.dtype, device=dev)
        M.lse_pass_static(v, f, lN, Q, logden=ld)
        torch.cuda.synchronize()
        q, qr = Q.cpu().numpy(), Q_ref.cpu().numpy()
        assert np.max(np.abs(q - qr) / np.abs(qr)) < TOL[dtype]
        assert np.max(np.abs(ld.cpu().numpy().astype(np.float64) - ld_ref.cpu().numpy())) < TOL[dtype] * 100


def test_static_scratch_pass_rejects_sizes_beyond_its_array():
    import torch
    K, N = 1024, 4096
    need = M.lse_scratch_bytes(K, N, 8)
    assert need > M.lib().mbar_lse_static_scratch_bytes()   # else this size would be accepted
    v, f, lN = _inputs(K, N, "float64", seed=1)              # fully allocated K x N input
    Q = torch.empty(K, dtype=torch.float64, device=v.device)
    with pytest.raises(M.MbarError) as e:
        M.lse_pass_static(v, f, lN, Q)
    assert e.value.name == "MBAR_EUNSUPPORTED"
    assert "built-in array" in str(e.value)
