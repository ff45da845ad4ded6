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
                                     "--steps", "10", "--warmup", "1"])
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
