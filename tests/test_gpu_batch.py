"""Batched boxes through the C ABI: graph-captured batch applies against the
same boxes applied one at a time, and against the oracle.

A batch box runs the same kernels with the same parameters as a standalone
plan.  Binning places points within a cell in the order the device's atomic
counters hand out slots, so summation order -- and only that -- may differ
between two applies: the batch must reproduce the standalone result to
rounding (the box's own arithmetic precision), on the capturing call and on
graph replays.  Accuracy is then the oracle's business: a seeded subset of
boxes is checked at 64 targets each against the direct Ewald sum, both error
measures within the box's own tolerance.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover - CPU container
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import oracle  # noqa: E402
from paper_2606_19059_gb300 import ewald, workloads  # noqa: E402

pytestmark = pytest.mark.gpu
DEV = torch.device("cuda:0")
F32 = ewald.EWALD_F32_BULK
SEED = 1004


def dev(a):
    return torch.as_tensor(np.ascontiguousarray(a), dtype=torch.float64, device=DEV)


@pytest.fixture(scope="module")
def batch():
    N, tol = workloads.batch_boxes(12, seed=SEED, n_hi=3e4)
    b = ewald.Batch(N, 1.0, tol, F32, tune=ewald.EWALD_TUNE_MEASURE, nstreams=4)
    data = [workloads.batch_box(SEED, i, int(n)) for i, n in enumerate(N)]
    for i, (x, f) in enumerate(data):
        bx, bf, _ = b.buffers(i)
        bx.copy_(dev(x))
        bf.copy_(dev(f))
    yield b, N, tol, data
    b.close()


def same_to_rounding(u, v, q):
    """Two applies of one plan: equal up to summation order in the plan's precision
    (double-single plans: the FP32 pairs of their split near field, ~tol/20)."""
    bound = 2e-6 if q.near_f64 == 0 else (q.tol / 20 if q.near_ds else 1e-11)
    d = (u - v).abs().max().item() / v.abs().max().item()
    return d <= bound, d


def standalone(b, i, x, f):
    q = b.params(i)
    p = ewald.Plan(int(b.N[i]), 1.0, float(q.tol), F32, M=q.M, P=q.P, tile=q.tile, poly_deg=q.poly_deg)
    assert (p.params.xi, p.params.rc, p.params.n_c) == (q.xi, q.rc, q.n_c)
    u = p.apply(dev(x), dev(f))
    torch.cuda.synchronize()
    return u


def test_batch_equals_boxes_one_at_a_time(batch):
    b, N, tol, data = batch
    b.apply()
    torch.cuda.synchronize()
    for i, (x, f) in enumerate(data):
        u_b = b.buffers(i)[2].clone()
        ok, d = same_to_rounding(u_b, standalone(b, i, x, f), b.params(i))
        assert ok, (i, d)


def test_graph_replay_with_new_forces(batch):
    b, N, tol, data = batch
    rng = np.random.default_rng(7)
    new = []
    for i, (x, f) in enumerate(data):
        f2 = workloads.forces(rng, int(N[i]))
        b.buffers(i)[1].copy_(dev(f2))
        new.append(f2)
    for _ in range(2):  # replays of the captured graph
        b.apply()
    torch.cuda.synchronize()
    for i, (x, f) in enumerate(data):
        ok, d = same_to_rounding(b.buffers(i)[2], standalone(b, i, x, new[i]), b.params(i))
        assert ok, (i, d)
    for i, (x, f) in enumerate(data):  # restore for the other tests
        b.buffers(i)[1].copy_(dev(f))


def test_batch_boxes_match_oracle(batch):
    b, N, tol, data = batch
    b.apply()
    torch.cuda.synchronize()
    rng = np.random.default_rng(11)
    # one box per tolerance present, 64 seeded targets each
    for t in sorted(set(tol.tolist())):
        i = int(np.flatnonzero(tol == t)[0])
        x, f = data[i]
        tg = np.sort(rng.choice(int(N[i]), size=min(64, int(N[i])), replace=False))
        ref = oracle.ewald(x, f, 1.0, targets=tg)
        u = b.buffers(i)[2].cpu().numpy()[tg]
        d = u - ref
        l2 = np.linalg.norm(d) / np.linalg.norm(ref)
        mx = np.abs(d).max() / np.abs(ref).max()
        assert l2 <= t and mx <= t, (i, t, l2, mx)


def test_autotune_picks_a_candidate_and_caches():
    ewald.ewald_autotune_clear()
    q, ms = ewald.ewald_autotune(8000, 1.0, 1e-6, F32)
    cands = ewald.ewald_autotune_candidates(8000, 1.0, 1e-6, F32, cap=24)
    assert any((c.M, c.tile) == (q.M, q.tile) for c in cands)
    assert ms > 0 and q.est_err <= 0.3e-6 * (1 + 1e-12)
    q2, ms2 = ewald.ewald_autotune(8000, 1.0, 1e-6, F32)
    assert (q2.M, q2.tile, ms2) == (q.M, q.tile, ms)


def test_batch_is_one_launch_per_stage_and_variant(batch):
    # every stage of every box in one launch per kernel instantiation, the FFTs
    # of the boxes that share a grid size and precision in one batched plan
    b, N, tol, data = batch
    k, f = b.launch_counts()
    groups = {(b.params(i).M, b.params(i).fft_f64) for i in range(len(N))}
    assert f == 2 * len(groups)
    per_box = sum(ewald.ewald_launch_counts(_plan(b, i))[0] for i in range(len(N)))
    assert k <= 40 and k < per_box, (k, per_box)


def _plan(b, i):
    import ctypes

    h = ctypes.c_void_p()
    ewald._check(ewald.load().ewald_batch_plan(b.handle, int(i), ctypes.byref(h)), "ewald_batch_plan")
    return h.value
