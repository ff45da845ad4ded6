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


def test_double_layer_on_double_single_plans_is_unsupported():
    N = 500
    x, f, q, n = _case("uniform", N, 406)
    p = ewald.Plan(N, 1.0, 1e-8, F32)   # double-single grid kernels
    with pytest.raises(ewald.EwaldError) as e:
        p.apply_combined(dev(x), dev(f), dev(q), dev(n))
    assert e.value.status == ewald.EWALD_EUNSUPPORTED


def test_double_layer_nan_density_sets_status():
    N = 400
    x, f, q, n = _case("uniform", N, 407)
    q[7, 1] = np.nan
    p = ewald.Plan(N, 1.0, 1e-6, F64)
    p.apply_combined(dev(x), dev(f), dev(q), dev(n))
    assert p.sync_status() == ewald.EWALD_EINVAL
