"""Autotuner candidates and batch argument checks: host logic, no GPU.

The measured choice itself needs a GPU (tests/test_gpu_batch.py); here the
candidate set is checked against the planner it derives from: every entry
meets the same error bound as the planner's own choice (Sec. 2.4: each term
of eq. (ese) below tol/10), grid sizes are cuFFT-friendly multiples of 8, and
the model choice comes first.
"""
import ctypes

import numpy as np
import pytest

from paper_2606_19059_gb300 import ewald, workloads

F32, F64 = ewald.EWALD_F32_BULK, ewald.EWALD_F64


def _friendly(m):
    if m % 2:
        return False
    for p in (2, 3, 5, 7):
        while m % p == 0:
            m //= p
    return m == 1


@pytest.mark.parametrize("N,tol", [(1000, 1e-4), (20000, 1e-6), (100000, 1e-8), (3000, 1e-8)])
def test_candidates_meet_the_planner_bound(N, tol):
    c = ewald.ewald_autotune_candidates(N, 1.0, tol, F32, cap=32)
    base = ewald.ewald_choose_params(N, 1.0, tol, F32)
    assert len(c) >= 2
    assert (c[0].M, c[0].P, c[0].tile) == (base.M, base.P, base.tile)
    seen = set()
    for q in c:
        assert q.est_err <= 0.3 * tol * (1 + 1e-12)
        assert q.P == base.P and q.tile in (4, 8) and q.M % q.tile == 0
        assert q.M % 8 == 0 and _friendly(q.M) and q.M >= q.P
        assert q.cell >= q.rc * (1 - 1e-12)
        key = (q.M, q.tile)
        assert key not in seen
        seen.add(key)
    Ms = [q.M for q in c[1:]]
    assert min(Ms) >= 0.6 * base.M - 8 and max(Ms) <= 1.7 * base.M + 8


@pytest.mark.parametrize("N", [1000, 3000, 20000, 100000])
def test_double_single_candidates_keep_the_double_single_grid(N):
    # FP32 bulk at tol <= 1e-7 runs double-single grid kernels, which take 8^3
    # tiles only; a 4^3-tile candidate would run FP64 P2G/G2P instead
    c = ewald.ewald_autotune_candidates(N, 1.0, 1e-8, F32, cap=32)
    assert all(q.near_ds == 1 for q in c)
    assert all(q.tile == 8 for q in c), [(q.M, q.tile) for q in c]
    # the FP32 plans still get the 4^3 candidate
    c6 = ewald.ewald_autotune_candidates(N, 1.0, 1e-6, F32, cap=32)
    assert any(q.tile == 4 for q in c6)


def test_candidates_cap_and_model_mode():
    c = ewald.ewald_autotune_candidates(5000, 1.0, 1e-6, F32, cap=1)
    assert len(c) == 1
    q, ms = ewald.ewald_autotune(5000, 1.0, 1e-6, F32, mode=ewald.EWALD_TUNE_MODEL)
    base = ewald.ewald_choose_params(5000, 1.0, 1e-6, F32)
    assert (q.M, q.P, q.tile, q.xi) == (base.M, base.P, base.tile, base.xi) and ms == -1.0


def test_batch_and_tuner_reject_bad_arguments():
    lib = ewald.load()
    arr = (ewald.ewald_params * 4)()
    n = ctypes.c_int32(0)
    assert lib.ewald_autotune_candidates(1000, 1.0, 1e-6, F32, 0, arr, ctypes.byref(n)) == ewald.EWALD_EINVAL
    assert lib.ewald_autotune_candidates(0, 1.0, 1e-6, F32, 4, arr, ctypes.byref(n)) == ewald.EWALD_EINVAL
    out = ewald.ewald_params()
    assert lib.ewald_autotune(1000, 1.0, 1e-6, F32, 7, ctypes.byref(out), None) == ewald.EWALD_EINVAL
    h = ctypes.c_void_p()
    N = np.array([1000, 2000], dtype=np.int64)
    L = np.ones(2)
    tol = np.array([1e-6, 1e-6])
    bad_tol = np.array([1e-6, 0.5])
    for args in [(0, N, L, tol, 1), (2, N, L, bad_tol, 1), (2, N, L, tol, 0), (2, N, L, tol, 65),
                 (2, np.array([1000, 0], dtype=np.int64), L, tol, 1)]:
        nb, n_, l_, t_, ns = args
        st = lib.ewald_batch_create(nb, n_.ctypes.data, l_.ctypes.data, t_.ctypes.data, F32,
                                    ewald.EWALD_TUNE_MODEL, ns, ctypes.byref(h))
        assert st == ewald.EWALD_EINVAL
    assert lib.ewald_batch_apply(None, None) == ewald.EWALD_EINVAL
    assert lib.ewald_batch_buffers(None, 0, None, None, None) == ewald.EWALD_EINVAL
    lib.ewald_batch_destroy(None)


def test_batch_workload_generator():
    N, tol = workloads.batch_boxes(512, seed=1004)
    assert N.dtype == np.int64 and N.min() >= 1000 and N.max() <= 100000
    assert set(np.unique(tol)) <= set(workloads.BATCH_TOLS)
    # log-uniform sizes: about half the boxes below 1e4
    assert 0.35 < np.mean(N < 10_000) < 0.65
    N2, tol2 = workloads.batch_boxes(512, seed=1004)
    assert np.array_equal(N, N2) and np.array_equal(tol, tol2)
    x, f = workloads.batch_box(1004, 3, 1234)
    assert x.shape == (1234, 3) and abs(f.mean(axis=0)).max() < 1e-12
