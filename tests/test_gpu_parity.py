"""GPU parity: the CUDA library (through its C ABI) against the CPU oracle.

Error measures (relative to the reference's size):
  rel_l2  = ||u - u_ref||_2 / ||u_ref||_2 over all components,
  rel_max = max |u - u_ref| / max |u_ref|.
A full apply passes when both are <= tol (the requested tolerance).  Stage
tests hold each stage to its own bound: rounding for the near field and the
convolution, the window-polynomial error for P2G/G2P, the window (aliasing)
error for the far field.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover - CPU container
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import oracle  # noqa: E402
from oracle import spectral  # noqa: E402
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


def plan(N, L, tol, dtype, **ov):
    return ewald.Plan(N, L, tol, dtype, **ov)


# ---------------------------------------------------------------- stages ----

@pytest.mark.parametrize("dtype,bound", [(F64, 1e-12), (F32, 2e-6)])
def test_near_field_matches_oracle(dtype, bound):
    x, f = workloads.make("uniform", 3000, seed=101)
    p = plan(3000, 1.0, 1e-8 if dtype == F64 else 1e-6, dtype, M=32, P=8)
    u = host(p.near_field(dev(x), dev(f)))
    ref = oracle.near_field(x, f, 1.0, p.params.xi, p.params.rc)
    l2, mx = errs(u, ref)
    assert l2 <= bound and mx <= 5 * bound, (l2, mx)


def test_near_field_small_box_explicit_images():
    # rc > L/3: fewer than three cells per side, colleague cells alias and
    # images must be enumerated explicitly
    x, f = workloads.make("uniform", 40, seed=102, L=1.0)
    p = plan(40, 1.0, 1e-3, F64, M=16, P=6)
    assert p.params.n_c < 3
    u = host(p.near_field(dev(x), dev(f)))
    ref = oracle.near_field(x, f, 1.0, p.params.xi, p.params.rc)
    assert errs(u, ref)[1] < 1e-11


def _support_sums(x, f, L, M, P):
    """Per grid point g and component c: n(g), the number of points whose
    window support (|g_d - x_d| < P h / 2 on every axis, periodic) holds g, and
    A_c(g), the sum of |f_c| over them."""
    h = L / M
    grid = np.arange(M) * h
    ins = []
    for d in range(3):
        r = np.abs(grid[None, :] - np.mod(x[:, d], L)[:, None])
        ins.append((np.minimum(r, L - r) < P * h / 2).astype(np.float64))
    n = np.einsum("pi,pj,pk->ijk", ins[2], ins[1], ins[0])
    A = np.stack([np.einsum("p,pi,pj,pk->ijk", np.abs(f[:, c]), ins[2], ins[1], ins[0]) for c in range(3)])
    return n, A


# FP32 P2G evaluates bins l and P-1-l from bin l's even and odd parts: odd P
# (a bin on the axis of symmetry) and even P both.
# Bound, per grid point and component: each term w_x w_y w_z f_c carries three
# window values off by at most werr (the polynomial against the exact window)
# and, in the kernels' precision u, the rounding of a degree-nu polynomial in
# its even/odd form (2 nu + 2 roundings) and of the products (2 more); the n(g)
# terms are then summed in an order the kernel does not fix (first-order
# forward error of a sum: (n - 1) u times the sum of the terms' sizes).  So
# |g - ref| <= 3 werr A(g) + (2 nu + 4 + n(g)) u B(g), B = spread of |f|
# (the window is nonnegative).
@pytest.mark.parametrize("dtype,P,M", [(F64, 8, 32), (F64, 7, 24), (F32, 12, 32), (F32, 11, 32), (F32, 7, 24)])
def test_spread_matches_exact_window(dtype, P, M):
    x, f = workloads.make("uniform", 400, seed=103)
    p = plan(400, 1.0, 1e-8 if dtype == F64 else 1e-6, dtype, M=M, P=P)
    g = host(p.spread(dev(x), dev(f)))
    ref = spectral.spread(x, f, 1.0, M, P)
    B = spectral.spread(x, np.abs(f), 1.0, M, P)
    n, A = _support_sums(x, f, 1.0, M, P)
    _, werr = ewald.ewald_window_eval(P, p.params.poly_deg, np.zeros(1))
    u = 2.0 ** -24 if dtype == F32 else 2.0 ** -53
    bound = 3 * werr * A + (2 * p.params.poly_deg + 4 + n[None]) * u * B + 1e-300
    err = np.abs(g - ref)
    assert np.all(err <= bound), (err.max(), (err / bound).max())
    assert n.max() > 0 and err.max() < 1e-3 * np.abs(ref).max()


@pytest.mark.parametrize("dtype", [F64, F32])
def test_interp_matches_exact_window(dtype):
    rng = np.random.default_rng(104)
    M, P = 32, 9
    x = workloads.uniform(rng, 300)
    v = rng.standard_normal((3, M, M, M))
    p = plan(300, 1.0, 1e-8 if dtype == F64 else 1e-6, dtype, M=M, P=P)
    u = host(p.interp(dev(x), dev(v)))
    ref = spectral.gather(x, v, 1.0, M, P)
    _, werr = ewald.ewald_window_eval(P, p.params.poly_deg, np.zeros(1))
    h3 = (1.0 / M) ** 3
    bound = 3 * werr * P ** 3 * h3 * np.abs(v).max() + (1e-6 if dtype == F32 else 1e-13) * np.abs(ref).max()
    assert np.abs(u - ref).max() <= bound


def test_spread_interp_adjoint_on_gpu():
    rng = np.random.default_rng(105)
    M, P = 24, 8
    x = workloads.uniform(rng, 500)
    f = workloads.forces(rng, 500, zero_mean=False)
    v = rng.standard_normal((3, M, M, M))
    p = plan(500, 1.0, 1e-8, F64, M=M, P=P)
    g = host(p.spread(dev(x), dev(f)))
    u = host(p.interp(dev(x), dev(v)))
    h3 = (1.0 / M) ** 3
    lhs, rhs = h3 * np.sum(g * v), np.sum(f * u)
    assert abs(lhs - rhs) <= 1e-12 * abs(lhs)


# M = 64, 128 and 256: 2-D (y, x) transforms around one kernel for the z
# transforms and the CNV (FP32, or double-single for FP64 spectra: unit
# roundoff 2^-44 over 2 log2 M <= 16 radix-2 stages each way and the CNV's
# ~10 operations, ~40 x 5.7e-14 of the spectrum's scale, x4 for the maximum
# against the norm: 1e-11); M = 32 and 36: the 3-D transforms and the CNV pass
@pytest.mark.parametrize("dtype,M,bound", [(F64, 32, 1e-12), (F64, 36, 1e-12), (F64, 64, 1e-11), (F64, 128, 1e-11),
                                           (F64, 256, 1e-11), (F32, 32, 2e-6), (F32, 64, 2e-6),
                                           (F32, 128, 3e-6), (F32, 256, 4e-6)])
def test_fourier_convolve_matches_numpy(dtype, M, bound):
    rng = np.random.default_rng(106)
    P = 8
    tol = 1e-8 if dtype == F64 else 1e-6
    p = plan(10, 1.0, tol, dtype, M=M, P=P)
    phi = rng.standard_normal((3, M, M, M))
    out = host(p.fourier_convolve(dev(phi)))
    ref = spectral.fourier_convolve(phi, 1.0, M, P, p.params.xi)
    assert np.abs(out - ref).max() <= bound * np.abs(ref).max()


@pytest.mark.parametrize("dtype,bound", [(F64, 1e-8), (F32, 2e-6)])
def test_far_field_matches_direct_k_sum(dtype, bound):
    x, f = workloads.make("uniform", 2000, seed=107)
    M = 48
    p = plan(2000, 1.0, 1e-8 if dtype == F64 else 1e-6, dtype, M=M, P=12)
    u = host(p.far_field(dev(x), dev(f)))
    ref = oracle.far_field(x, f, 1.0, p.params.xi, kbox=M // 2 - 1)
    l2, mx = errs(u, ref)
    assert l2 <= bound and mx <= 5 * bound, (l2, mx)


# ----------------------------------------------------------- full apply -----

def test_hasimoto_single_point_on_gpu():
    xi_sc = 2.8372974794806  # tests/golden/hasimoto_sc.txt
    x = np.array([[0.3, 0.6, 0.1]])
    f = np.array([[0.2, -1.0, 0.5]])
    p = plan(1, 1.0, 1e-10, F64)
    u = host(p.apply(dev(x), dev(f)))
    assert np.abs(u - (-(8 / 6) * xi_sc * f)).max() <= 1e-9 * np.abs(f).max()


def test_uniform_1e3_tol1e8_fp64_all_targets():
    name = "uniform_1e3_tol1e-8"
    kind, N, L, tol, M, P, seed = workloads.WORKLOADS[name]
    x, f = workloads.make(kind, N, seed, L)
    p = plan(N, L, tol, F64)
    u = host(p.apply(dev(x), dev(f)))
    ref = oracle.ewald(x, f, L)
    l2, mx = errs(u, ref)
    assert l2 <= tol and mx <= tol, (l2, mx, p.params.as_dict())


@pytest.mark.parametrize("dtype", [F32, F64])
def test_uniform_1e5_tol1e6_sampled(dtype):
    kind, N, L, tol, M, P, seed = workloads.WORKLOADS["uniform_1e5_tol1e-6_M128_P12"]
    x, f = workloads.make(kind, N, seed, L)
    p = plan(N, L, tol, dtype, M=M, P=P)
    u = host(p.apply(dev(x), dev(f)))
    idx = np.random.default_rng(7).choice(N, 256, replace=False)
    ref = oracle.ewald(x, f, L, targets=idx)
    l2, mx = errs(u[idx], ref)
    assert l2 <= tol and mx <= tol, (l2, mx)


@pytest.fixture(scope="module")
def clustered_2e6():
    kind, N, L, tol, M, P, seed = workloads.WORKLOADS["clustered_2e6_tol1e-7_M256_P14"]
    x, f = workloads.make(kind, N, seed, L)
    idx = np.random.default_rng(8).choice(N, 64, replace=False)
    ref = oracle.ewald(x, f, L, targets=idx)
    return x, f, idx, ref, (N, L, tol, M, P)


def test_clustered_2e6_tol1e7_fp32_sampled(clustered_2e6):
    # FP32 bulk at tol 1e-7: plain FP32 pairs sit at the tolerance on this
    # workload (max error over all points 1.03e-7 of max |u|), so the planner
    # takes the double-single near field and grid kernels here
    x, f, idx, ref, (N, L, tol, M, P) = clustered_2e6
    p = plan(N, L, tol, F32, M=M, P=P)
    assert p.params.near_ds == 1 and p.params.fft_f64 == 1
    u = host(p.apply(dev(x), dev(f)))
    l2, mx = errs(u[idx], ref)
    assert l2 <= tol and mx <= tol, (l2, mx)


def test_clustered_2e6_tol1e7_fp64_sampled(clustered_2e6):
    x, f, idx, ref, (N, L, tol, M, P) = clustered_2e6
    p = plan(N, L, tol, F64, M=M, P=P)
    u = host(p.apply(dev(x), dev(f)))
    l2, mx = errs(u[idx], ref)
    assert l2 <= tol and mx <= tol, (l2, mx)


@pytest.mark.parametrize("dtype", [F64, F32])
def test_clustered_small_all_targets(dtype):
    x, f = workloads.make("clustered", 4000, seed=109)
    tol = 1e-8 if dtype == F64 else 1e-6
    p = plan(4000, 1.0, tol, dtype)
    u = host(p.apply(dev(x), dev(f)))
    ref = oracle.ewald(x, f, 1.0)
    l2, mx = errs(u, ref)
    assert l2 <= tol and mx <= tol, (l2, mx)


# ------------------------------------------------------------ edge cases ----

def test_two_points_and_odd_grid():
    x = np.array([[0.1, 0.2, 0.3], [0.8, 0.75, 0.05]])
    f = np.array([[1.0, 0.0, 0.0], [0.0, -1.0, 0.5]])
    p = plan(2, 1.0, 1e-7, F64, M=40, P=11)
    u = host(p.apply(dev(x), dev(f)))
    ref = oracle.ewald(x, f, 1.0)
    assert errs(u, ref)[1] <= 1e-7


def test_positions_outside_box_are_wrapped():
    x, f = workloads.make("uniform", 500, seed=110)
    shift = np.random.default_rng(1).integers(-3, 4, size=x.shape).astype(float)
    p = plan(500, 1.0, 1e-8, F64)
    u1 = host(p.apply(dev(x), dev(f)))
    u2 = host(p.apply(dev(x + shift), dev(f)))
    assert errs(u2, u1)[1] < 1e-12


def test_all_points_in_one_cell():
    rng = np.random.default_rng(111)
    x = 0.5 + 0.01 * rng.standard_normal((600, 3))
    f = workloads.forces(rng, 600)
    p = plan(600, 1.0, 1e-8, F64)
    u = host(p.apply(dev(x), dev(f)))
    ref = oracle.ewald(x, f, 1.0)
    l2, mx = errs(u, ref)
    assert l2 <= 1e-8 and mx <= 1e-8


def test_coincident_points_are_skipped():
    x, f = workloads.make("uniform", 300, seed=112)
    x[7] = x[3]  # an exact duplicate position
    p = plan(300, 1.0, 1e-8, F64)
    u = host(p.apply(dev(x), dev(f)))
    ref = oracle.ewald(x, f, 1.0)
    assert np.all(np.isfinite(u))
    assert errs(u, ref)[1] <= 1e-8


def test_nonunit_box_and_net_force():
    rng = np.random.default_rng(113)
    L = 2.5
    x = workloads.uniform(rng, 800, L)
    f = rng.standard_normal((800, 3)) + 0.3  # net force: k = 0 dropped
    p = plan(800, L, 1e-7, F64)
    u = host(p.apply(dev(x), dev(f)))
    ref = oracle.ewald(x, f, L)
    l2, mx = errs(u, ref)
    assert l2 <= 1e-7 and mx <= 1e-7


def test_nan_input_sets_status_without_fault():
    x, f = workloads.make("uniform", 200, seed=114)
    x[5, 1] = np.nan
    p = plan(200, 1.0, 1e-6, F32)
    p.apply(dev(x), dev(f))
    assert p.sync_status() == ewald.EWALD_EINVAL
    x[5, 1] = 0.5
    p.apply(dev(x), dev(f))
    assert p.sync_status() == ewald.EWALD_OK


def test_bad_arguments_return_status():
    with pytest.raises(ewald.EwaldError) as e:
        ewald.ewald_plan(0, 1.0, 1e-6)
    assert e.value.status == ewald.EWALD_EINVAL
    p = plan(10, 1.0, 1e-6, F32)
    with pytest.raises(ewald.EwaldError) as e:
        ewald.ewald_apply(p.handle, 0, 0, 0, 0)
    assert e.value.status == ewald.EWALD_EINVAL
    with pytest.raises(ewald.EwaldError) as e:
        ewald.ewald_apply_forces(ewald.ewald_plan(10, 1.0, 1e-6), 1, 1, 0)  # no positions yet
    assert e.value.status == ewald.EWALD_EINVAL


def test_set_positions_then_apply_forces_equals_apply():
    x, f = workloads.make("uniform", 5000, seed=115)
    g = workloads.forces(np.random.default_rng(3), 5000)
    p = plan(5000, 1.0, 1e-6, F32)
    ua = host(p.apply(dev(x), dev(g)))
    p.set_positions(dev(x))
    p.apply_forces(dev(f))
    ub = host(p.apply_forces(dev(g)))
    assert errs(ub, ua)[1] < 1e-6


def test_apply_host_equals_device_apply():
    x, f = workloads.make("uniform", 3000, seed=116)
    p = plan(3000, 1.0, 1e-6, F32)
    ud = host(p.apply(dev(x), dev(f)))
    xh = torch.from_numpy(x.copy()).pin_memory()
    fh = torch.from_numpy(f.copy()).pin_memory()
    uh = torch.empty_like(xh).pin_memory()
    for _ in range(4):  # direct, captured, direct again, then the faster
        uh.zero_()
        ewald.ewald_apply_host(p.handle, xh.data_ptr(), fh.data_ptr(), uh.data_ptr(),
                               torch.cuda.current_stream().cuda_stream)
        assert errs(uh.numpy(), ud)[1] < 5e-6


def test_apply_host_pageable_equals_device_apply():
    """Pageable host arrays take the staged-copy path (page-locked ones are
    read and written in place by the kernels)."""
    x, f = workloads.make("uniform", 3000, seed=120)
    p = plan(3000, 1.0, 1e-6, F32)
    ud = host(p.apply(dev(x), dev(f)))
    xh, fh = np.ascontiguousarray(x), np.ascontiguousarray(f)
    uh = np.zeros_like(xh)
    for _ in range(3):
        ewald.ewald_apply_host(p.handle, xh.ctypes.data, fh.ctypes.data, uh.ctypes.data,
                               torch.cuda.current_stream().cuda_stream)
        assert errs(uh, ud)[1] < 5e-6
        uh[:] = 0.0


def test_repeated_apply_sees_new_buffer_contents():
    """Repeated applies on the same buffers replay a captured graph; the
    replay must read the buffers' current contents, and new buffers must
    capture again.  Binning orders each cell's points by atomics, so two
    applies of the same input differ by FP32 rounding (a few 1e-7); a stale
    replay would be off by O(1)."""
    N = 4000
    x, f = workloads.make("uniform", N, seed=118)
    x2, g = workloads.make("uniform", N, seed=119)
    p = plan(N, 1.0, 1e-6, F32)
    s = torch.cuda.current_stream().cuda_stream
    xd, fd = dev(x), dev(f)
    u = torch.empty_like(xd)
    for _ in range(3):
        ewald.ewald_apply(p.handle, xd.data_ptr(), fd.data_ptr(), u.data_ptr(), s)
    ua = host(u)
    xd.copy_(dev(x2))
    fd.copy_(dev(g))
    ewald.ewald_apply(p.handle, xd.data_ptr(), fd.data_ptr(), u.data_ptr(), s)
    ub = host(u)
    ref_a = host(plan(N, 1.0, 1e-6, F32).apply(dev(x), dev(f)))
    ref_b = host(plan(N, 1.0, 1e-6, F32).apply(dev(x2), dev(g)))
    assert errs(ua, ref_a)[1] < 5e-6
    assert errs(ub, ref_b)[1] < 5e-6
    x3d, f3d = dev(x), dev(f)  # new buffers: a new capture
    u3 = torch.empty_like(x3d)
    for _ in range(2):
        ewald.ewald_apply(p.handle, x3d.data_ptr(), f3d.data_ptr(), u3.data_ptr(), s)
    assert errs(host(u3), ref_a)[1] < 5e-6


def test_fp32_and_fp64_agree_to_tolerance():
    x, f = workloads.make("uniform", 20000, seed=117)
    a = host(plan(20000, 1.0, 1e-6, F32, M=64, P=10).apply(dev(x), dev(f)))
    b = host(plan(20000, 1.0, 1e-6, F64, M=64, P=10).apply(dev(x), dev(f)))
    l2, mx = errs(a, b)
    assert l2 < 1e-6 and mx < 1e-6


def test_stage_times_reported():
    x, f = workloads.make("uniform", 20000, seed=118)
    p = plan(20000, 1.0, 1e-6, F32)
    for mode in (1, 2):
        ewald.ewald_set_timing(p.handle, mode)
        p.apply(dev(x), dev(f))
        t = ewald.ewald_stage_times(p.handle)
        assert t["total_ms"] > 0 and t["p2p_ms"] > 0 and t["p2g_ms"] > 0 and t["g2p_ms"] > 0
    k, nfft = ewald.ewald_launch_counts(p.handle)
    assert 8 <= k <= 9 and nfft == 2  # bin 3, P2P, P2G, CNV, G2P, SUM (+ grid copy)


# ------------------------------------------------- double-single near field --

def test_near_field_double_single_matches_oracle():
    # FP32 bulk at tol <= 1e-7: pairs within the split radius in pairs of
    # FP32 values (~44 bits), the small terms beyond it in compensated FP32,
    # chosen so that their error stays near tol/10 of the near field -- the
    # near field's share of the eq. (ese) budget the planner allots
    tol = 1e-8
    x, f = workloads.make("uniform", 3000, seed=103)
    p = plan(3000, 1.0, tol, F32, M=32, P=8)
    assert p.params.near_ds == 1 and p.params.near_f64 == 1
    u = host(p.near_field(dev(x), dev(f)))
    ref = oracle.near_field(x, f, 1.0, p.params.xi, p.params.rc)
    l2, mx = errs(u, ref)
    assert l2 <= tol / 5 and mx <= tol, (l2, mx)


@pytest.mark.parametrize("kind,N,tol", [("uniform", 20000, 1e-8), ("clustered", 12000, 1e-9)])
def test_f32_bulk_double_single_full_apply(kind, N, tol):
    x, f = workloads.make(kind, N, seed=104)
    p = plan(N, 1.0, tol, F32)
    assert p.params.near_ds == 1
    u = host(p.apply(dev(x), dev(f)))
    idx = np.sort(np.random.default_rng(5).choice(N, 256, replace=False))
    ref = oracle.ewald(x, f, 1.0, targets=idx)
    l2, mx = errs(u[idx], ref)
    assert l2 <= tol and mx <= tol, (l2, mx)


# ------------------------------------------------- double-single grid ------

def _ds_plan(N, M, P):
    # FP32 bulk at tol <= 1e-7: P2G / G2P in double-single arithmetic too (8^3
    # tiles, P >= 8), with their extra kernels: window weights, grid copy
    p = plan(N, 1.0, 1e-8, F32, M=M, P=P)
    assert p.params.near_ds == 1 and p.params.tile == 8
    assert ewald.ewald_launch_counts(p.handle) == (10, 2)
    return p


@pytest.mark.parametrize("P,M", [(12, 32), (16, 40), (8, 24)])
def test_spread_double_single_matches_exact_window(P, M):
    x, f = workloads.make("uniform", 400, seed=108)
    p = _ds_plan(400, M, P)
    g = host(p.spread(dev(x), dev(f)))
    ref = spectral.spread(x, f, 1.0, M, P)
    _, werr = ewald.ewald_window_eval(P, p.params.poly_deg, np.zeros(1))
    bound = 3 * werr * np.abs(f).max() + 1e-13 * np.abs(ref).max()
    assert np.abs(g - ref).max() <= bound, (np.abs(g - ref).max(), bound)


@pytest.mark.parametrize("P,M", [(9, 32), (14, 48)])
def test_interp_double_single_matches_exact_window(P, M):
    rng = np.random.default_rng(109)
    x = workloads.uniform(rng, 300)
    v = rng.standard_normal((3, M, M, M))
    p = _ds_plan(300, M, P)
    u = host(p.interp(dev(x), dev(v)))
    ref = spectral.gather(x, v, 1.0, M, P)
    _, werr = ewald.ewald_window_eval(P, p.params.poly_deg, np.zeros(1))
    h3 = (1.0 / M) ** 3
    bound = 3 * werr * P ** 3 * h3 * np.abs(v).max() + 1e-12 * np.abs(ref).max()
    assert np.abs(u - ref).max() <= bound, (np.abs(u - ref).max(), bound)


def test_spread_interp_adjoint_double_single():
    rng = np.random.default_rng(110)
    M, P = 32, 13
    x = workloads.uniform(rng, 700)
    f = workloads.forces(rng, 700, zero_mean=False)
    v = rng.standard_normal((3, M, M, M))
    p = _ds_plan(700, M, P)
    g = host(p.spread(dev(x), dev(f)))
    u = host(p.interp(dev(x), dev(v)))
    h3 = (1.0 / M) ** 3
    lhs, rhs = h3 * np.sum(g * v), np.sum(f * u)
    assert abs(lhs - rhs) <= 1e-11 * abs(lhs)


def test_double_single_grid_matches_fp64_grid():
    # the same plan parameters with FP64 grid kernels (F64) and double-single
    # ones (F32 bulk): far fields agree to double-single rounding
    x, f = workloads.make("clustered", 6000, seed=111)
    p = _ds_plan(6000, 48, 14)
    q = plan(6000, 1.0, 1e-8, F64, M=48, P=14, xi=p.params.xi, rc=p.params.rc)
    a = host(p.far_field(dev(x), dev(f)))
    b = host(q.far_field(dev(x), dev(f)))
    l2, mx = errs(a, b)
    assert l2 <= 1e-11 and mx <= 1e-11, (l2, mx)


def test_fma_probe_reports_plausible_peaks():
    # FP32 FMA pipe of a GB300: 152 SMs x 128 lanes x 2 flops x ~2 GHz ~ 80
    # TFLOP/s; FP64 a small fraction of it
    p32, p64 = ewald.ewald_probe_fma_peaks(0)
    assert 5.0 < p32 < 500.0, p32
    assert 0.05 < p64 < p32 / 4, (p32, p64)
