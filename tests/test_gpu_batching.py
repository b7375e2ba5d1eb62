"""Batched angles x views in one call, captured in a CUDA graph (reduced sizes): graph
replays reproduce the eager gradients, and the batched form beats the plain form."""
import pytest

pytestmark = pytest.mark.gpu


def test_batched_graph_and_plain_form():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2607_13265_gb300 import batch_bench
    out = batch_bench.main(["--replays", "3", "--angles", "6", "--views", "3", "--scale", "0.125", "--spp", "4",
                            "--depth", "4", "--no-tune"])
    assert out["batched"]["graph_vs_eager_grad_rel"] < 1e-4
    assert out["speedup_effective"] > 1.0
    assert len(out["per_view_gradients"]) == 3
    assert all(v["dtheta_l2"] > 0 for v in out["per_view_gradients"])
