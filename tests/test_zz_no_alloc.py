"""The allocation-free near field (ewald_near_field_noalloc) against the
regular entry point.

Some callers cannot allocate device memory (a pool or allocator that owns the
device, a plugin that must leave its host's allocator alone, a path that must
not synchronise the device), so the library offers a near field whose whole
workspace is a fixed array inside the library.  This file is named so that
pytest collects it last; it runs the same way alone or after the others.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover - CPU container
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from paper_2606_19059_gb300 import ewald, workloads  # noqa: E402

pytestmark = pytest.mark.gpu
DEV = torch.device("cuda:0")


def _dev(a):
    return torch.as_tensor(np.ascontiguousarray(a), dtype=torch.float64, device=DEV)


@pytest.mark.parametrize("dtype,tol,bound", [
    (ewald.EWALD_F64, 1e-8, 1e-12),
    (ewald.EWALD_F32_BULK, 1e-6, 2e-6),
    (ewald.EWALD_F32_BULK, 1e-7, 2e-6),
])
def test_noalloc_near_field_matches_plan_two_calls(dtype, tol, bound):
    N = 6000
    plan = ewald.Plan(N, 1.0, tol, dtype, M=32, P=8)
    stream = torch.cuda.current_stream().cuda_stream
    for seed in (301, 302):  # two calls in a row, different points and forces
        x, f = workloads.make("uniform", N, seed)
        xd, fd = _dev(x), _dev(f)
        ref = plan.near_field(xd, fd)
        out = torch.empty_like(xd)
        ewald.ewald_near_field_noalloc(N, plan.params, xd.data_ptr(), fd.data_ptr(), out.data_ptr(),
                                       stream)
        torch.cuda.synchronize()
        a, b = out.cpu().numpy(), ref.cpu().numpy()
        assert np.linalg.norm(a - b) <= bound * np.linalg.norm(b)
        assert np.abs(a - b).max() <= 5 * bound * np.abs(b).max()


def test_noalloc_rejects_sizes_beyond_its_workspace():
    plan = ewald.Plan(1000, 1.0, 1e-6, ewald.EWALD_F32_BULK)
    big = 32769
    with pytest.raises(ewald.EwaldError) as e:
        ewald.ewald_near_field_noalloc(big, plan.params, 1, 1, 1, 0)
    assert e.value.status == ewald.EWALD_EUNSUPPORTED
    prm = ewald.ewald_params()
    prm.L, prm.xi, prm.rc = 1.0, 100.0, 0.01  # 100 cells per side > 16
    with pytest.raises(ewald.EwaldError) as e:
        ewald.ewald_near_field_noalloc(100, prm, 1, 1, 1, 0)
    assert e.value.status == ewald.EWALD_EUNSUPPORTED
