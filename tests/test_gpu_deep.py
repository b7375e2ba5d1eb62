"""Deep paths on the GPU: the deep-path benchmark module at a reduced image size runs every
schedule at depths 8 and 128 and the schedules agree on the gradient (they trace the same
paths; only the order of the floating-point gradient sums differs)."""
import pytest

pytestmark = pytest.mark.gpu


def test_deep_bench_schedules_agree():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2607_13265_gb300 import deep_bench
    rows = deep_bench.main(["--width", "64", "--height", "36", "--depths", "8", "128", "--reps", "1",
                            "--schedules", "grid", "persistent", "wavefront", "sweep"])
    assert len(rows) == 8
    by = {(r["schedule"], r["depth"]): r for r in rows}
    for d in (8, 128):
        assert by[("grid", d)]["vertices_per_path"] > 0.6 * d
        ref = by[("grid", d)]["grad_norm"]
        for s in ("persistent", "wavefront", "sweep"):
            for k, v in ref.items():
                assert by[(s, d)]["grad_norm"][k] == pytest.approx(v, rel=1e-4), (s, d, k)
    assert by[("grid", 128)]["local_bytes_per_thread"] >= 128 * 124
    assert by[("wavefront", 128)]["workspace_bytes"] > by[("wavefront", 8)]["workspace_bytes"]
