"""The allocation-free near field (ewald_near_field_noalloc) against the
regular entry point and against the oracle's near field.

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

import oracle  # noqa: E402
from paper_2606_19059_gb300 import ewald, workloads  # noqa: E402

pytestmark = pytest.mark.gpu
DEV = torch.device("cuda:0")


def _dev(a):
    return torch.as_tensor(np.ascontiguousarray(a), dtype=torch.float64, device=DEV)


def _noalloc(N, prm, xd, fd):
    out = torch.empty_like(xd)
    ewald.ewald_near_field_noalloc(N, prm, xd.data_ptr(), fd.data_ptr(), out.data_ptr(),
                                   torch.cuda.current_stream().cuda_stream)
    torch.cuda.synchronize()
    return out.cpu().numpy()


# (dtype, tol, bound against the plan's near field, bound against the
# oracle's; relative to the result's size, rel_max bounds 5x): FP64 to
# rounding against the plan and to the kernels' rational erf(x)/x (6e-12
# evaluated) against the oracle, FP32 to its pair arithmetic, double-single
# (split near field: the small terms beyond the split radius in compensated
# FP32) to tol/5 against the oracle and to the FP32 pairs' summation order
# against the plan
CASES = [
    (ewald.EWALD_F64, 1e-8, 1e-12, 1e-11, False),
    (ewald.EWALD_F32_BULK, 1e-6, 2e-6, 2e-6, False),
    (ewald.EWALD_F32_BULK, 2e-7, 2e-6, 2e-6, False),
    (ewald.EWALD_F32_BULK, 1e-8, 5e-10, 2e-9, True),
]


@pytest.mark.parametrize("dtype,tol,bound,obound,ds", CASES)
def test_noalloc_near_field_matches_plan_and_oracle_two_calls(dtype, tol, bound, obound, ds):
    N = 6000
    plan = ewald.Plan(N, 1.0, tol, dtype, M=32, P=8)
    prm = plan.params
    assert prm.near_ds == (1 if ds else 0)
    for seed in (301, 302):  # two calls in a row, different points and forces
        x, f = workloads.make("uniform", N, seed)
        xd, fd = _dev(x), _dev(f)
        ref = plan.near_field(xd, fd).cpu().numpy()
        a = _noalloc(N, prm, xd, fd)
        assert np.linalg.norm(a - ref) <= bound * np.linalg.norm(ref)
        assert np.abs(a - ref).max() <= 5 * bound * np.abs(ref).max()
        o = oracle.near_field(x, f, 1.0, prm.xi, prm.rc)
        assert np.linalg.norm(a - o) <= obound * np.linalg.norm(o)
        assert np.abs(a - o).max() <= 5 * obound * np.abs(o).max()


def test_noalloc_nan_input_gives_nan_output():
    N = 500
    plan = ewald.Plan(N, 1.0, 1e-6, ewald.EWALD_F32_BULK, M=16, P=6)
    x, f = workloads.make("uniform", N, 303)
    x[17, 1] = np.nan
    a = _noalloc(N, plan.params, _dev(x), _dev(f))
    assert np.isnan(a).all()
    x[17, 1] = 0.5  # the flag is cleared by the next call
    a = _noalloc(N, plan.params, _dev(x), _dev(f))
    assert np.isfinite(a).all()


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
    prm.xi, prm.rc, prm.near_ds = 100.0, 0.07, 1  # xi rc = 7, past the double-single erfcx fit
    with pytest.raises(ewald.EwaldError) as e:
        ewald.ewald_near_field_noalloc(100, prm, 1, 1, 1, 0)
    assert e.value.status == ewald.EWALD_EUNSUPPORTED
