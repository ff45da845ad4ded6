"""Serving: the force-update generator and the request loop's host logic (no GPU).

The served requests perturb their forces between applies with normals from
Philox4x32-10; the input-generator side (workloads.py) is pinned here to the
generator's published known-answer vectors, and the device side is pinned to
this one by tests/test_gpu_serving.py.  The server's admission bookkeeping --
refusal of requests that can never fit, queue, cancellation, bounded waits --
runs on the host and is tested on a paused server that admits nothing.
"""
import ctypes
import os

import numpy as np

from paper_2606_19059_gb300 import ewald, workloads

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "philox4x32_10_kat.txt")


def test_philox_known_answers():
    rows = [ln.split() for ln in open(GOLDEN) if ln.strip() and not ln.startswith("#")]
    assert len(rows) == 3
    for r in rows:
        v = [int(h, 16) for h in r]
        out = workloads.philox4x32_10(*[np.array([c]) for c in v[:4]], v[4], v[5])
        assert [int(o[0]) for o in out] == v[6:10]


def test_perturbation_normals_are_standard_and_fresh():
    n = 200_000
    a = workloads.perturbation_normals(n, 1, 12345)
    assert a.shape == (n, 3)
    assert abs(a.mean()) < 0.01 and abs(a.std() - 1.0) < 0.01
    # kurtosis of a normal is 3; uniform-looking or clipped draws would not be
    k = ((a - a.mean()) ** 4).mean() / a.var() ** 2
    assert abs(k - 3.0) < 0.05
    b = workloads.perturbation_normals(n, 2, 12345)
    c = workloads.perturbation_normals(n, 1, 12346)
    for other in (b, c):
        assert abs(np.corrcoef(a.ravel(), other.ravel())[0, 1]) < 0.01
    assert np.array_equal(a, workloads.perturbation_normals(n, 1, 12345))


def test_served_forces_stay_centred():
    rng = np.random.default_rng(3)
    f0 = workloads.forces(rng, 5000)
    f = workloads.served_forces(f0, 20, 0.1, 77)
    assert abs(f.mean(axis=0)).max() < 1e-12
    d = f - f0
    # 19 updates of scale 0.1, each re-centred: per-component variance ~ 0.19
    assert 0.15 < d.var() < 0.23


def test_serving_stream_recipe():
    s = workloads.serving_stream(400, seed=5, rate_hz=20.0)
    t = np.array([r["t"] for r in s])
    N = np.array([r["N"] for r in s])
    assert np.all(np.diff(t) > 0) and 0.03 < np.mean(np.diff(t)) < 0.07
    assert N.min() >= 1000 and N.max() <= 4_000_000
    assert 0.35 < np.mean([r["kind"] == "uniform" for r in s]) < 0.65
    assert set(r["tol"] for r in s) <= set(workloads.BATCH_TOLS)
    x, f = workloads.served_box("clustered", 3000, 9)
    assert x.shape == (3000, 3) and (x >= 0).all() and (x < 1).all()


def _req(n, tol=1e-6):
    x = np.random.default_rng(n).random((n, 3))
    f = np.zeros((n, 3))
    u = np.zeros((n, 3))
    r = ewald.ewald_request(N=n, L=1.0, tol=tol, dtype=ewald.EWALD_F32_BULK, napplies=3, perturb=0.1, seed=1,
                            x_host=x.ctypes.data, f_host=f.ctypes.data, u_host=u.ctypes.data)
    return r, (x, f, u)


def test_server_queue_cancel_timeout_and_refusal():
    lib = ewald.load()
    h = ctypes.c_void_p()
    assert lib.ewald_server_create(0, 4, 1, ctypes.byref(h)) == ewald.EWALD_EINVAL
    assert lib.ewald_server_create(1 << 30, 0, 1, ctypes.byref(h)) == ewald.EWALD_EINVAL
    prm = ewald.ewald_choose_params(20000, 1.0, 1e-6, ewald.EWALD_F32_BULK)
    budget = int(1.5 * (prm.footprint_bytes + 8 * (9 * 20000 + 3)))
    assert lib.ewald_server_create(budget, 4, 1, ctypes.byref(h)) == ewald.EWALD_OK
    try:
        t = ctypes.c_int64(0)
        r1, keep1 = _req(20000)
        r2, keep2 = _req(20000)
        assert lib.ewald_server_submit(h, ctypes.byref(r1), ctypes.byref(t)) == ewald.EWALD_OK
        t1 = t.value
        assert lib.ewald_server_submit(h, ctypes.byref(r2), ctypes.byref(t)) == ewald.EWALD_OK
        t2 = t.value
        # a request that can never fit the budget is refused at the door
        big, keepb = _req(400000)
        assert lib.ewald_server_submit(h, ctypes.byref(big), ctypes.byref(t)) == ewald.EWALD_ENOMEM
        # bad requests
        bad, keepx = _req(100)
        bad.napplies = 0
        assert lib.ewald_server_submit(h, ctypes.byref(bad), ctypes.byref(t)) == ewald.EWALD_EINVAL
        bad.napplies, bad.tol = 3, 0.5
        assert lib.ewald_server_submit(h, ctypes.byref(bad), ctypes.byref(t)) == ewald.EWALD_EINVAL
        bad.tol, bad.u_host = 1e-6, None
        assert lib.ewald_server_submit(h, ctypes.byref(bad), ctypes.byref(t)) == ewald.EWALD_EINVAL
        st, lat = ctypes.c_int32(-1), ctypes.c_double(0)
        assert lib.ewald_server_poll(h, t1, ctypes.byref(st), ctypes.byref(lat)) == ewald.EWALD_OK
        assert st.value == ewald.EWALD_REQ_QUEUED and lat.value == -1.0
        # paused: nothing is admitted, a bounded wait runs out
        assert lib.ewald_server_wait(h, t1, ctypes.c_double(0.05)) == ewald.EWALD_ETIMEOUT
        assert lib.ewald_server_cancel(h, t2) == ewald.EWALD_OK
        assert lib.ewald_server_cancel(h, t2) == ewald.EWALD_EINVAL
        assert lib.ewald_server_wait(h, t2, ctypes.c_double(1.0)) == ewald.EWALD_OK
        assert lib.ewald_server_poll(h, t2, ctypes.byref(st), None) == ewald.EWALD_OK
        assert st.value == ewald.EWALD_REQ_CANCELLED
        assert lib.ewald_server_poll(h, 999, ctypes.byref(st), None) == ewald.EWALD_EINVAL
        s = ewald.ewald_server_summary()
        assert lib.ewald_server_stats(h, ctypes.byref(s)) == ewald.EWALD_OK
        assert (s.submitted, s.queued, s.cancelled, s.active, s.completed) == (2, 1, 1, 0, 0)
    finally:
        lib.ewald_server_destroy(h)  # drops the queued request without starting it
