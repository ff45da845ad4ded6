"""GPU parity of the combined single and double layer apply (Sec. 2.3),
through the C ABI, against the CPU oracle (oracle/stresslet.py).

Error measures as in test_gpu_parity.py (relative to the reference's size).
Bounds: against the direct Ewald sum, the plan's tol (the double layer's
discretisation error at the plan's xi, rc, M, P was measured on the CPU,
oracle alone, at 2e-10 for tol 1e-8 and 3e-8 for tol 1e-6 on uniform
points); against the oracle's own near field + grid pipeline at the plan's
parameters, 1e-9 in FP64 (the kernels' window polynomial against the exact
window, and rounding).
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover - CPU container
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from oracle import stresslet as dl  # noqa: E402
import oracle  # noqa: E402
from paper_2606_19059_gb300 import ewald, workloads  # noqa: E402

pytestmark = pytest.mark.gpu
DEV = torch.device("cuda:0")
F64, F32 = ewald.EWALD_F64, ewald.EWALD_F32_BULK


def dev(a):
    return torch.as_tensor(np.ascontiguousarray(a), dtype=torch.float64, device=DEV)


def host(t):
    torch.cuda.synchronize()
    return t.detach().cpu().numpy()


def errs(u, ref):
    d = u - ref
    return (np.linalg.norm(d) / np.linalg.norm(ref), np.abs(d).max() / np.abs(ref).max())


def _case(kind, N, seed, L=1.0):
    x, f = workloads.make(kind, N, seed=seed, L=L)
    rng = np.random.default_rng(seed + 1)
    q, n = rng.standard_normal((N, 3)), rng.standard_normal((N, 3))
    return x, f, q, n


def _combined(p, x, f, q, n):
    return host(p.apply_combined(dev(x), dev(f), dev(q), dev(n)))


def test_double_layer_fp64_matches_oracle_pipeline_and_direct_sum():
    N = 1200
    x, _, q, n = _case("uniform", N, 401)
    p = ewald.Plan(N, 1.0, 1e-8, F64)
    prm = p.params.as_dict()
    u = _combined(p, x, np.zeros((N, 3)), q, n)
    D = dl.densities(q, n)
    tid = np.arange(0, N, 13)
    near = dl.near_field(x, D, 1.0, prm["xi"], prm["rc"], targets=tid)
    far = dl.far_field_spectral(x, D, 1.0, prm["M"], prm["P"], prm["xi"])[tid]
    assert errs(u[tid], near + far)[1] < 1e-9
    ref = dl.ewald(x, D, 1.0, targets=tid)
    l2, mx = errs(u[tid], ref)
    assert l2 < 1e-8 and mx < 1e-8


def test_combined_is_stokeslet_plus_double_layer():
    N = 3000
    x, f, q, n = _case("uniform", N, 402)
    p = ewald.Plan(N, 1.0, 1e-8, F64)
    uc = _combined(p, x, f, q, n)
    us = host(p.apply(dev(x), dev(f)))
    ud = _combined(p, x, np.zeros((N, 3)), q, n)
    assert errs(uc, us + ud)[1] < 1e-12
    # and the Stokeslet part alone is unchanged by the double layer's buffers
    tid = np.arange(0, N, 97)
    ref = oracle.ewald(x, f, 1.0, targets=tid)
    assert errs(us[tid], ref)[1] < 1e-8


def test_double_layer_fp32_bulk_within_tolerance():
    N = 1500
    x, _, q, n = _case("uniform", N, 403)
    p = ewald.Plan(N, 1.0, 1e-6, F32)
    u = _combined(p, x, np.zeros((N, 3)), q, n)
    tid = np.arange(0, N, 17)
    ref = dl.ewald(x, dl.densities(q, n), 1.0, targets=tid)
    l2, mx = errs(u[tid], ref)
    assert l2 < 1e-6 and mx < 1e-6


@pytest.mark.parametrize("tile,P", [(4, 12), (8, 11)])
def test_combined_fp32_other_tile_and_odd_support(tile, P):
    # 4^3 tiles take the per-triple P2G passes instead of the one-pass
    # nine-component kernel; an odd support puts a bin on the window's axis of
    # symmetry (the P2G rows of bins l and P-1-l come from one polynomial)
    N = 1500
    x, f, q, n = _case("uniform", N, 409)
    p = ewald.Plan(N, 1.0, 1e-6, F32, M=32, P=P, tile=tile)
    assert (p.params.tile, p.params.P) == (tile, P)
    u = _combined(p, x, f, q, n)
    tid = np.arange(0, N, 13)
    ref = oracle.ewald(x, f, 1.0, targets=tid) + dl.ewald(x, dl.densities(q, n), 1.0, targets=tid)
    l2, mx = errs(u[tid], ref)
    assert l2 < 1e-6 and mx < 1e-6, (l2, mx)


@pytest.mark.parametrize("M", [64, 256])
def test_combined_fp32_z_kernels_at_other_grid_sizes(M):
    # FP32 spectra at M = 64 and 256 take the 2-D transforms around the z
    # kernels (Stokeslet alone, and with the double layer's nine components),
    # whose splits M = R1 R2 and block shapes differ from M = 128's
    N = 1500
    x, f, q, n = _case("uniform", N, 410)
    p = ewald.Plan(N, 1.0, 1e-6, F32, M=M, P=12)
    assert p.params.fft_f64 == 0 and p.params.M == M and p.params.tile == 8
    tid = np.arange(0, N, 13)
    ref_s = oracle.ewald(x, f, 1.0, targets=tid)
    us = host(p.apply(dev(x), dev(f)))
    l2, mx = errs(us[tid], ref_s)
    assert l2 < 1e-6 and mx < 1e-6, (l2, mx)
    u = _combined(p, x, f, q, n)
    ref = ref_s + dl.ewald(x, dl.densities(q, n), 1.0, targets=tid)
    l2, mx = errs(u[tid], ref)
    assert l2 < 1e-6 and mx < 1e-6, (l2, mx)


def test_double_layer_fp32_pairs_fp64_fft_two_cells_per_side():
    # FP32 bulk at 1e-7 < tol < 1e-6: FP32 densities spread onto FP64 grids,
    # FP64 CNV and FP64 near-field pairs; n_c = 2, so the 27 neighbour offsets
    # reach one cell through several images
    N, tol = 1500, 3e-7
    x, _, q, n = _case("uniform", N, 408)
    p = ewald.Plan(N, 1.0, tol, F32)
    prm = p.params
    assert prm.near_f64 == 0 and prm.near_ds == 0 and prm.fft_f64 == 1 and prm.n_c == 2
    u = _combined(p, x, np.zeros((N, 3)), q, n)
    tid = np.arange(0, N, 17)
    ref = dl.ewald(x, dl.densities(q, n), 1.0, targets=tid)
    l2, mx = errs(u[tid], ref)
    assert l2 <= tol and mx <= tol, (l2, mx)


def test_double_layer_fp32_cutoff_reaching_two_cells():
    # FP32 pairs with cells narrower than rc (K = 2: 125 neighbour cells)
    N, tol = 1500, 1e-6
    x, _, q, n = _case("uniform", N, 409)
    rc = ewald.ewald_choose_params(N, 1.0, tol, F32).rc
    p = ewald.Plan(N, 1.0, tol, F32, n_c=int(1.5 / rc))
    prm = p.params
    assert prm.fft_f64 == 0 and 1.0 < prm.rc / prm.cell <= 2.0
    u = _combined(p, x, np.zeros((N, 3)), q, n)
    tid = np.arange(0, N, 17)
    ref = dl.ewald(x, dl.densities(q, n), 1.0, targets=tid)
    l2, mx = errs(u[tid], ref)
    assert l2 <= tol and mx <= tol, (l2, mx)


def test_combined_at_the_benchmark_workload():
    # The combined apply as the benchmark times it (uniform N = 1e5, M = 128,
    # P = 12, FP32 bulk, tol 1e-6) at 256 seeded targets: the Stokeslet part
    # from the C oracle, the double layer from stored oracle values
    # (tests/golden/make_stresslet_uniform_1e5.py, oracle/stresslet.py)
    import os

    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "stresslet_uniform_1e5_256.txt")
    tab = np.loadtxt(path)
    idx, ref_dl = tab[:, 0].astype(np.int64), tab[:, 1:]
    kind, N, L, tol, M, P, seed = workloads.WORKLOADS["uniform_1e5_tol1e-6_M128_P12"]
    x, f = workloads.make(kind, N, seed, L)
    rng = np.random.default_rng(1009)
    q = rng.standard_normal((N, 3))
    n = rng.standard_normal((N, 3))
    assert np.array_equal(idx, np.sort(np.random.default_rng(7).choice(N, 256, replace=False)))
    p = ewald.Plan(N, L, tol, F32, M=M, P=P)
    u = _combined(p, x, f, q, n)
    ref = oracle.ewald(x, f, L, targets=idx) + ref_dl
    l2, mx = errs(u[idx], ref)
    assert l2 <= tol and mx <= tol, (l2, mx)
    # the double layer alone, relative to its own size
    ud = _combined(p, x, np.zeros((N, 3)), q, n)
    l2, mx = errs(ud[idx], ref_dl)
    assert l2 <= tol and mx <= tol, (l2, mx)


def test_double_layer_clustered_and_nonunit_box():
    N, L = 1000, 2.0
    x, _, q, n = _case("clustered", N, 404, L=L)
    p = ewald.Plan(N, L, 1e-8, F64)
    u = _combined(p, x, np.zeros((N, 3)), q, n)
    tid = np.arange(0, N, 11)
    ref = dl.ewald(x, dl.densities(q, n), L, targets=tid)
    l2, mx = errs(u[tid], ref)
    assert l2 < 1e-8 and mx < 1e-8


def test_double_layer_wraps_positions_and_ignores_antisymmetric_part():
    N = 2000
    x, _, q, n = _case("uniform", N, 405)
    p = ewald.Plan(N, 1.0, 1e-6, F64)
    z = np.zeros((N, 3))
    ua = _combined(p, x, z, q, n)
    shift = np.random.default_rng(9).integers(-2, 3, size=(N, 3)).astype(np.float64)
    ub = _combined(p, x + shift, z, q, n)          # the same points, other images
    assert errs(ub, ua)[1] < 1e-12
    uc = _combined(p, x, z, n, q)                   # q (x) n and n (x) q: same symmetric part
    assert errs(uc, ua)[1] < 1e-12


@pytest.mark.parametrize("kind,N,tol", [("uniform", 1500, 1e-8), ("clustered", 1200, 1e-7)])
def test_double_layer_on_double_single_plans(kind, N, tol):
    # FP32 bulk at tol <= 1e-7: the densities spread by the double-single P2G
    # onto FP64 grids, FP64 FFTs and CNV, double-single G2P, FP64 near pairs
    x, f, q, n = _case(kind, N, 406)
    p = ewald.Plan(N, 1.0, tol, F32)
    assert p.params.near_ds == 1 and p.params.tile == 8 and p.params.P >= 8
    tid = np.arange(0, N, 13)
    u = _combined(p, x, np.zeros((N, 3)), q, n)
    ref = dl.ewald(x, dl.densities(q, n), 1.0, targets=tid)
    l2, mx = errs(u[tid], ref)
    assert l2 <= tol and mx <= tol, (l2, mx)
    uc = _combined(p, x, f, q, n)  # and with the Stokeslet part
    refc = ref + oracle.ewald(x, f, 1.0, targets=tid)
    l2, mx = errs(uc[tid], refc)
    assert l2 <= tol and mx <= tol, (l2, mx)


def test_double_layer_nan_density_sets_status():
    N = 400
    x, f, q, n = _case("uniform", N, 407)
    q[7, 1] = np.nan
    p = ewald.Plan(N, 1.0, 1e-6, F64)
    p.apply_combined(dev(x), dev(f), dev(q), dev(n))
    assert p.sync_status() == ewald.EWALD_EINVAL


def test_combined_allocation_failure_leaves_the_plan_usable():
    # The combined apply allocates its four double-layer workspaces on first
    # use.  A failure at any of them returns ENOMEM and commits none of them,
    # so the next call allocates afresh instead of launching on a partial set.
    N = 1000
    x, f, q, n = _case("uniform", N, 431)
    ref = _combined(ewald.Plan(N, 1.0, 1e-6, F32), x, f, q, n)
    for nth in (1, 2, 4):
        p = ewald.Plan(N, 1.0, 1e-6, F32)
        ewald.ewald_debug_fail_alloc(nth)
        try:
            with pytest.raises(ewald.EwaldError) as e:
                _combined(p, x, f, q, n)
        finally:
            ewald.ewald_debug_fail_alloc(0)
        assert e.value.status == ewald.EWALD_ENOMEM
        assert p.sync_status() == ewald.EWALD_OK
        u = _combined(p, x, f, q, n)  # FP32 pairs: equal to rounding (cell order may differ)
        assert np.abs(u - ref).max() <= 1e-6 * np.abs(ref).max()
        p.close()


def test_plan_allocation_failure_returns_enomem():
    ewald.ewald_debug_fail_alloc(7)
    try:
        with pytest.raises(ewald.EwaldError) as e:
            ewald.Plan(2000, 1.0, 1e-6, F32)
    finally:
        ewald.ewald_debug_fail_alloc(0)
    assert e.value.status == ewald.EWALD_ENOMEM
    x, f = workloads.make("uniform", 2000, seed=432)
    p = ewald.Plan(2000, 1.0, 1e-6, F32)
    u = host(p.apply(dev(x), dev(f)))
    ref = oracle.ewald(x, f, 1.0, targets=np.arange(0, 2000, 20))
    assert errs(u[::20], ref)[0] <= 1e-6
