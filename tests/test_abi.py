"""CPU-side checks of the C ABI: the library builds, loads, exports every
symbol the header declares, its structs match the binding, and the host-side
argument checks answer without touching a GPU."""
import ctypes
import os
import re
import subprocess
import tempfile

import numpy as np
import pytest

from paper_2609_03541_b300 import build as B
from paper_2609_03541_b300 import mbar as M

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "bumbar.h")


@pytest.fixture(scope="module")
def L():
    B.build()
    return M.lib()


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(mbar_[a-z0-9_]+)\s*\(", text)))


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ["mbar_create", "mbar_bin", "mbar_solve", "mbar_free_energies", "mbar_destroy",
                     "mbar_sci_step", "mbar_hessian", "mbar_newton_step", "mbar_lse_pass"]:
        assert required in names


def test_library_exports_every_declared_symbol(L):
    out = subprocess.run(["nm", "-D", "--defined-only", M.LIB_PATH], capture_output=True, text=True, check=True).stdout
    exported = set(re.findall(r"\sT\s(mbar_[a-z0-9_]+)", out))
    missing = [n for n in declared_functions() if n not in exported]
    assert not missing, missing
    assert set(M._SIGNATURES) <= exported


def test_struct_layout_matches_binding():
    src = r'''
#include <stdio.h>
#include <stddef.h>
#include "bumbar.h"
int main(void){
  printf("%zu %zu %zu %zu %zu %zu %zu %zu %zu %zu\n", sizeof(mbar_opts), offsetof(mbar_opts, f_tol),
         offsetof(mbar_opts, max_sci), offsetof(mbar_opts, noise_floor),
         sizeof(mbar_report), offsetof(mbar_report, max_abs_grad), offsetof(mbar_report, last_step),
         sizeof(mbar_server_config), offsetof(mbar_server_config, hbm_budget_bytes),
         offsetof(mbar_server_config, opts));
  return 0;
}'''
    with tempfile.TemporaryDirectory() as d:
        c = os.path.join(d, "t.c")
        open(c, "w").write(src)
        exe = os.path.join(d, "t")
        subprocess.run(["gcc", "-I", os.path.join(ROOT, "include"), c, "-o", exe], check=True)
        vals = list(map(int, subprocess.run([exe], capture_output=True, text=True, check=True).stdout.split()))
    assert vals == [ctypes.sizeof(M.Opts), M.Opts.f_tol.offset, M.Opts.max_sci.offset, M.Opts.noise_floor.offset,
                    ctypes.sizeof(M.Report), M.Report.max_abs_grad.offset, M.Report.last_step.offset,
                    ctypes.sizeof(M.ServerConfig), M.ServerConfig.hbm_budget_bytes.offset,
                    M.ServerConfig.opts.offset]


def test_opts_default_are_the_papers(L):
    o = M.default_opts(M.MBAR_MIXED)
    assert (o.n0, o.eps, o.inc, o.n_intermediate) == (100, 1e-3, 10, 20)
    assert o.use_binning == 1 and o.h0 == 0.0
    with pytest.raises(M.MbarError):
        M.default_opts(7)


def test_status_strings(L):
    for code in range(8):
        assert L.mbar_status_string(code)


@pytest.mark.parametrize("K,N,Nk,code", [
    (0, 4, [], "MBAR_EINVAL"),
    (2, 4, [1, 2], "MBAR_EINVAL"),           # counts do not sum to N
    (2, 4, [0, 4], "MBAR_EINVAL"),           # empty state
    (2000, 4000, [2] * 2000, "MBAR_EUNSUPPORTED"),
])
def test_create_rejects_bad_sizes_before_any_device_work(L, K, N, Nk, code):
    u = np.zeros((max(K, 1), N))
    Nk = np.asarray(Nk if Nk else [1], dtype=np.int64)
    h = ctypes.c_void_p()
    st = L.mbar_create(ctypes.byref(h), K, N, Nk.ctypes.data_as(M._i64p), ctypes.c_void_p(u.ctypes.data), 0, None, None)
    assert M.STATUS[st] == code
    assert not h.value


def test_destroy_null_is_ok(L):
    assert L.mbar_destroy(None) == 0


def test_exclusive_needs_a_context(L):
    assert M.STATUS[L.mbar_set_exclusive(None, 1)] == "MBAR_EINVAL"


def test_footprint_estimate_grows_with_the_problem(L):
    small = M.footprint_bytes(8, 8000)
    big = M.footprint_bytes(500, 2_000_000)
    assert 0 < small < big
    assert big >= 500 * 2_000_000 * 12          # FP64 staging + FP32 data at creation
    assert M.footprint_bytes(500, 2_000_000, M.MBAR_FP64) > big
    assert M.footprint_bytes(0, 10) == 0


def test_factorised_footprint_holds_no_store(L):
    """A store-free (MIXED, binned) factorised solve is charged less than
    the FP32 K x N store at the largest served size; on the FP64 path the
    charge carries the K x N FP64 buffer of u."""
    K, N = 1024, 20_000 * 1024
    mixed = M.footprint_factorised_bytes(K, N, M.MBAR_MIXED)
    assert 0 < mixed < K * N * 4
    assert M.footprint_factorised_bytes(K, N, M.MBAR_FP64) > K * N * 8
    assert M.footprint_factorised_bytes(K, N, M.MBAR_MIXED, use_binning=0) > K * N * 8
    assert M.footprint_factorised_bytes(0, 10) == 0


def test_autotune_rejects_bad_arguments_without_a_gpu(L):
    for fam, K, n, code in [(7, 50, 1000, "MBAR_EINVAL"), (M.TUNE_SAMPLES, 0, 1000, "MBAR_EINVAL"),
                            (M.TUNE_SAMPLES, 2000, 1000, "MBAR_EUNSUPPORTED"),
                            (M.TUNE_FACTORISED, 50, 0, "MBAR_EINVAL")]:
        with pytest.raises(M.MbarError) as e:
            M.autotune_lse(fam, K, n)
        assert e.value.name == code


def test_autotune_cache_file_is_read_back(L, tmp_path):
    """A cache line is served without timing anything (cached = 1). Without
    a GPU the device name is "unknown", so a line for that name is found;
    the key is K rounded up to a power of two and floor(log2 n)."""
    path = tmp_path / "tune.txt"
    path.write_text("unknown 0 64 17 8 4 512 65536 20 0.5 0.6\n"
                    "unknown 1 512 20 32 4 384 0 6 1.0 1.1\n")
    M.autotune_clear()
    M.autotune_cache(path)
    try:
        r = M.autotune_lse(M.TUNE_SAMPLES, 50, 200_000)      # 50 -> 64, log2(2e5) -> 17
        assert r["cached"] == 1
        assert (r["lanes_per_sample"], r["chunks_per_lane"], r["stage_bytes"]) == (8, 4, 65536)
        r = M.autotune_lse(M.TUNE_FACTORISED, 500, 2_000_000)  # 500 -> 512, log2(2e6) -> 20
        assert (r["lanes_per_sample"], r["chunks_per_lane"], r["threads"]) == (32, 4, 384)
        assert r["ms"] == 1.0 and r["heuristic_ms"] == 1.1
    finally:
        M.autotune_cache(None)
        M.autotune_clear()


def test_server_rejects_bad_configuration_without_a_gpu(L):
    cfg = M.server_config(workers=0, hbm_budget_bytes=1 << 30)
    with pytest.raises(M.MbarError) as e:
        M.Server(cfg)
    assert e.value.name == "MBAR_EINVAL"
    cfg = M.server_config(workers=2, hbm_budget_bytes=0)
    with pytest.raises(M.MbarError):
        M.Server(cfg)


@pytest.mark.parametrize("K,N,code", [(0, 4, "MBAR_EINVAL"), (2, 0, "MBAR_EINVAL"), (2000, 4, "MBAR_EUNSUPPORTED")])
def test_create_factorised_rejects_bad_sizes_before_any_device_work(L, K, N, code):
    a = np.zeros(max(K, 1))
    phi = np.zeros(max(N, 1))
    Nk = np.ones(max(K, 1), dtype=np.int64)
    h = ctypes.c_void_p()
    p = lambda x: ctypes.c_void_p(x.ctypes.data)
    st = L.mbar_create_factorised(ctypes.byref(h), K, N, Nk.ctypes.data_as(M._i64p), p(a), p(a), p(phi), 0, None,
                                  None)
    assert M.STATUS[st] == code
    assert not h.value
    st = L.mbar_create_factorised(ctypes.byref(h), 2, 4, Nk.ctypes.data_as(M._i64p), None, p(a), p(phi), 0, None,
                                  None)
    assert M.STATUS[st] == "MBAR_EINVAL"


def test_factorised_pass_rejects_bad_arguments_before_any_device_work(L):
    assert L.mbar_lse_factorised_scratch_bytes(0, 10) == 0
    assert L.mbar_lse_factorised_scratch_bytes(2000, 10) == 0
    x = np.zeros(16)
    p = ctypes.c_void_p(x.ctypes.data)
    st = L.mbar_lse_pass_factorised(None, p, p, 2, 4, p, p, None, p, None, p, 4096, None)
    assert M.STATUS[st] == "MBAR_EINVAL"
    st = L.mbar_lse_pass_factorised(p, p, p, 2000, 4, p, p, None, p, None, p, 4096, None)
    assert M.STATUS[st] == "MBAR_EUNSUPPORTED"
    st = L.mbar_lse_pass_factorised(p, p, p, 0, 4, p, p, None, p, None, p, 4096, None)
    assert M.STATUS[st] == "MBAR_EINVAL"
