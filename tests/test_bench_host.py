"""The benchmark's host-side assembly of its JSON line, on CPU: the GPU
measurement is replaced by a fixed result of the same shape, and the line
that main() prints is checked against the contract (keys, whole-job rate,
end-to-end rate, roofline and double-layer entries, launch count)."""
import json

import numpy as np
import pytest

import bench
from paper_2606_19059_gb300 import ewald, workloads


@pytest.fixture
def fake_result():
    kind, N, L, tol, M, P, seed = workloads.WORKLOADS[bench.WORKLOAD]
    x, _ = workloads.make(kind, N, seed, L)
    ov = ewald.ewald_params()
    ov.M, ov.P = M, P
    prm = ewald.ewald_choose_params(N, L, tol, ewald.EWALD_F32_BULK, override=ov).as_dict()
    st = {"bin_ms": 0.045, "p2p_ms": 0.297, "p2g_ms": 0.194, "fft_ms": 0.0435, "scale_ms": 0.0123,
          "ifft_ms": 0.041, "g2p_ms": 0.133, "sum_ms": 0.0061, "total_ms": 0.777}
    st_dl = dict(st, sum_ms=1.95, p2g_ms=0.588, total_ms=3.2)

    def run(args, rank, world):
        return {"ms32": [0.65] * args.steps, "wall32": 0.2, "ms64": [18.6] * 3, "stages": st,
                "e2e_s": [0.0007] * 5, "dl": {"ms": [3.15] * 5, "stages": st_dl},
                "clocks": {"sm_mhz": 2070.0, "sm_max_mhz": 2070.0, "reasons": [], "samples": 10},
                "kernels_per_step": 8, "ffts_per_step": 2, "params": prm,
                "N": N, "L": L, "tol": tol, "M": M, "P": P, "x": x}

    return run, N


def test_json_line_follows_the_contract(monkeypatch, capsys, fake_result):
    run, N = fake_result
    monkeypatch.setattr(bench, "run_gpu", run)
    monkeypatch.setattr("sys.argv", ["bench.py", "--no-batch", "--no-serve", "--no-cpu-baseline",
                                     "--no-clustered", "--steps", "10", "--warmup", "1"])
    monkeypatch.delenv("WORLD_SIZE", raising=False)
    bench.main()
    lines = [ln for ln in capsys.readouterr().out.splitlines() if ln.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    for k in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
              "scaling", "vs_baseline", "dtype", "data", "config", "roofline", "e2e", "gpu_launches", "clocks"):
        assert k in d, k
    assert d["n_gpus"] == 1 and d["steps"] == 10 and d["warmup"] >= 3
    assert d["value"] == pytest.approx(N / 0.65e-3)
    assert d["ms_per_step"] == pytest.approx(0.65)
    assert d["e2e"]["value"] == pytest.approx(N / 0.7e-3)
    assert d["e2e"]["h2d_bytes_per_step"] == 2 * N * 24 and d["e2e"]["d2h_bytes_per_step"] == N * 24
    assert d["gpu_launches"] == 8 * 10
    assert d["config"]["workload"] == bench.WORKLOAD
    roof = d["roofline"]
    assert roof["bound"] in ("alu", "hbm", "tensor")
    assert roof["frac"] == pytest.approx(roof["achieved"] / roof["peak"])
    assert d["double_layer"]["near_dl_ms"] == pytest.approx(1.95 - 0.0061, abs=1e-4)
    assert np.isfinite(d["double_layer"]["value"])
    # FP32 FFTs at tol 1e-6: the double layer's near field runs FP32 pairs
    assert d["double_layer"]["near_dl_kernel"].startswith("k_p2p_dl32")
    assert "clustered" not in d


def test_clustered_entry(monkeypatch, capsys, fake_result):
    run, N = fake_result
    kind, Nc, L, tol, M, P, seed = workloads.WORKLOADS[bench.CLUSTERED]
    ov = ewald.ewald_params()
    ov.M, ov.P = M, P
    prm = ewald.ewald_choose_params(Nc, L, tol, ewald.EWALD_F32_BULK, override=ov).as_dict()
    x = workloads.uniform(np.random.default_rng(3), 20000)  # a stand-in sample for the pair estimate
    st = {"bin_ms": 2.4, "p2p_ms": 420.0, "p2g_ms": 20.7, "fft_ms": 5.16, "scale_ms": 0.79,
          "ifft_ms": 5.2, "g2p_ms": 15.7, "sum_ms": 0.03, "total_ms": 470.0}

    def run_c(args, rank, world):
        return {"ms": 436.0, "value": Nc / 0.436, "ms64": 3300.0, "value64": Nc / 3.3, "stages": st,
                "params": prm, "N": 20000, "L": L, "tol": tol, "M": M, "P": P, "x": x, "steps": 3}

    monkeypatch.setattr(bench, "run_gpu", run)
    monkeypatch.setattr(bench, "run_clustered", run_c)
    monkeypatch.setattr("sys.argv", ["bench.py", "--no-batch", "--no-serve", "--no-cpu-baseline",
                                     "--steps", "10", "--warmup", "1"])
    monkeypatch.delenv("WORLD_SIZE", raising=False)
    bench.main()
    lines = [ln for ln in capsys.readouterr().out.splitlines() if ln.startswith("{")]
    d = json.loads(lines[0])
    c = d["clustered"]
    assert c["workload"] == bench.CLUSTERED and c["near"] == "double-single" and c["fft"] == "FP64"
    assert c["value"] == pytest.approx(Nc / 0.436) and c["fp64_plain"]["ms_per_step"] == 3300.0
    r = c["stage_roofline"]
    ncplx = M * M * (M // 2 + 1)
    assert r["fft"]["bytes_per_launch"] == 3 * M ** 3 * 8 + 3 * ncplx * 16
    assert r["fft"]["frac"] == pytest.approx(r["fft"]["achieved"] / r["fft"]["peak"])
    assert r["p2p"]["inrange_pairs_est"] > 0
    # M = 256 with FP64 spectra: the double-single y and z transform kernels
    assert M == 256 and "k_fgc_z64" in r["scale"]["kernel"] and "k_fft_y64" in r["fft"]["kernel"]
    # and the main line's FP32 spectra at M = 128: the FP32 z-transform kernel
    assert d["stage_roofline"]["scale"]["kernel"].startswith("k_fgc_z:")
