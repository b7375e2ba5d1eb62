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
    assert out["batched_fused_l2"]["grad_rel_vs_image_form"] < 1e-4
    assert out["batched_fused_l2"]["peak_autograd_bytes"] < out["plain"]["peak_autograd_bytes"]
    assert len(out["per_view_gradients"]) == 3
    assert all(v["dtheta_l2"] > 0 for v in out["per_view_gradients"])


# (views, angles, spp, sizes, adjoint schedule): a few views and an unfiltered job on the
# default launch; 70 small views, more than one launch's 64 jobs, so that the L2 folds and the
# job tables run in two chunks, under the sweep schedule
FUSED_CASES = {"few_views": (3, 8, 4, (24, 40, 32), None), "70_views_sweep": (70, 3, 2, (8, 12, 9), 3)}


@pytest.mark.parametrize("case", list(FUSED_CASES))
def test_fused_l2_equals_image_form(case):
    """PolarizedL2 (loss folded into the camera filter) gives the loss and every gradient of
    PolarizedRender + ImageL2 on the same paths -- views with polarizer angles, plus
    an unfiltered job -- while keeping 12 floats per pixel instead of one image per angle."""
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import copy
    import numpy as np
    from paper_2607_13265_gb300 import api, build, scenegen as sg
    build.build()
    dctx = api.Context(0)
    nviews, nang, spp, sizes, adj_sched = FUSED_CASES[case]
    if adj_sched is not None:
        dctx.set_launch(0, 128, 0, adj_sched, 128, 0)
    scene, jobs = sg.cornell_views(nviews, nang, spp, 4, sizes)
    plain = copy.copy(jobs[0])
    plain.filter, plain.thetas, plain.stream = sg.FILTER_NONE, [], 7 + nviews
    jobs = jobs + [plain]
    gs = api.GpuScene(dctx, scene)
    batch = api.pack_jobs(jobs)
    adj = api.pack_jobs(api.adjoint_jobs(jobs))
    P = api.device_params(scene, batch)
    tp = scene.params()
    tp["tex"] = np.clip(tp["tex"] * 0.8 + 0.05, 0.0, 1.0)
    tp["theta"] = batch.theta + 0.1
    target = api.render_primal(dctx, gs, batch, api.device_params(scene, batch, tp)).clone()

    def grads(fused):
        leaf = {k: v.clone().requires_grad_(True) for k, v in P.items()}
        args = (leaf["tex"], leaf["ior"], leaf["le"], leaf["sheet"], leaf["theta"])
        torch.cuda.synchronize()
        torch.cuda.reset_peak_memory_stats()
        base = torch.cuda.memory_allocated()
        if fused:
            loss = api.PolarizedL2.apply(dctx, gs, batch, adj, target, *args)
        else:
            loss = api.ImageL2.apply(api.PolarizedRender.apply(dctx, gs, batch, adj, *args), target)
        loss.backward()
        torch.cuda.synchronize()
        dctx.sync_status()
        peak = torch.cuda.max_memory_allocated() - base
        return float(loss.detach()), {k: v.grad.double().cpu().numpy() for k, v in leaf.items()}, peak

    l_img, g_img, m_img = grads(False)
    l_fus, g_fus, m_fus = grads(True)
    assert l_fus == pytest.approx(l_img, rel=1e-5)
    for k in ("tex", "theta", "ior", "le"):
        n = np.linalg.norm(g_img[k])
        assert n > 0, k
        assert np.linalg.norm(g_fus[k] - g_img[k]) <= 1e-4 * n, (k, np.linalg.norm(g_fus[k] - g_img[k]) / n)
    assert m_fus < 0.5 * m_img, (m_fus, m_img)
