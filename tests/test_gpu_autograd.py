"""Differentiation through torch.autograd on the rocks workload (100,000 triangles of rough
dielectric rocks, 512x512, 32 spp, depth 16, a quarter-wave plate and a linear polarizer in
front of the camera, full Stokes output).  The loss is a seeded linear functional of an 8x8
crop of the image; its gradient w.r.t. the 512x512x3 albedo texture, the emitter Stokes
vector and the polarizer angle comes from PolarizedRender.backward (render_adjoint, cached
suffix replay) and is checked against
  * the taped FP64 oracle (conventional reverse AD) on the same crop and the same
    decorrelated adjoint paths: relative 1e-3 per parameter group;
  * central differences with h = 1e-3: of the GPU primal for the polarizer angle and the
    emitter Stokes components (their values do not steer any sampling decision, so the
    GPU's primal is itself the frozen-sampling estimator), and of the oracle's
    frozen-sampling estimator for albedo texels.  The GPU differences are taken in FP32:
    they are held to 1e-2 relative plus the rounding bound 8 ulp * sum|W I| / h."""
import copy

import numpy as np
import pytest

from paper_2607_13265_gb300 import scenegen as sg

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def setup(oracle_mod):
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2607_13265_gb300 import build, api
    build.build()
    dctx = api.Context(0)
    scene, job = sg.rocks_scene()
    gs = api.GpuScene(dctx, scene)
    batch = api.pack_jobs([job])
    adj = api.pack_jobs(api.adjoint_jobs([job]))
    P = api.device_params(scene, batch)
    # 8x8 crop and a seeded linear functional of its Stokes values; the comparison is made
    # for identical paths: crop pixels with a path whose FP32 and FP64 signatures differ
    # (a grazing ray that lands on the neighbouring triangle) are left out of the functional
    x0, y0 = 300, 220
    pix = np.array([(y0 + dy) * job.width + x0 + dx for dy in range(8) for dx in range(8)], np.int64)
    sig = torch.zeros(job.num_paths, dtype=torch.int32, device="cuda")
    aj = api.adjoint_jobs([job])
    api.render_primal(dctx, gs, api.pack_jobs(aj, path_sig=sig), P)
    sig_g = sig.cpu().numpy().view(np.uint32).reshape(-1, job.spp)[pix]
    _, _, sig_o = oracle_mod.OracleScene(scene).render(aj[0], scene.params(), pixels=pix, paths=True)
    same = (sig_g.ravel() == sig_o).reshape(-1, job.spp)
    assert same.mean() >= 0.95, same.mean()
    keep = same.all(1)
    w = np.random.default_rng(5).normal(size=(1, len(pix), 3, 4)) * keep[None, :, None, None]
    W = torch.zeros(batch.image_floats, dtype=torch.float32, device="cuda")
    W.view(1, -1, 3, 4)[:, torch.as_tensor(pix, device="cuda")] = torch.as_tensor(w, dtype=torch.float32, device="cuda")
    return torch, api, dctx, scene, job, gs, batch, adj, P, pix, w, W


def _autograd_grads(torch, api, dctx, gs, batch, adj, P, W):
    leaf = {k: v.clone().requires_grad_(True) for k, v in P.items()}
    img = api.PolarizedRender.apply(dctx, gs, batch, adj, leaf["tex"], leaf["ior"], leaf["le"], leaf["sheet"],
                                    leaf["theta"])
    (img * W).sum().backward()
    dctx.sync_status()
    return {k: v.grad.double().cpu().numpy() for k, v in leaf.items()}


def test_autograd_matches_taped_oracle(setup, oracle_mod):
    torch, api, dctx, scene, job, gs, batch, adj, P, pix, w, W = setup
    g = _autograd_grads(torch, api, dctx, gs, batch, adj, P, W)
    aj = copy.copy(job)
    aj.pass_id = 1
    ref = oracle_mod.OracleScene(scene).gradient(aj, scene.params(), w, pixels=pix, mode="tape")
    off, tw, th, ch = scene.tex_desc[0]
    o, gg = ref["tex"][off:off + tw * th * ch], g["tex"][off:off + tw * th * ch]
    assert np.linalg.norm(o) > 0
    assert np.linalg.norm(gg - o) <= 1e-3 * np.linalg.norm(o)
    for k in ("le", "theta"):
        o, gg = ref[k], g[k][:ref[k].size]
        assert np.linalg.norm(o) > 0, k
        assert np.linalg.norm(gg - o) <= 1e-3 * np.linalg.norm(o), (k, gg, o)


def test_autograd_matches_central_differences(setup, oracle_mod):
    torch, api, dctx, scene, job, gs, batch, adj, P, pix, w, W = setup
    g = _autograd_grads(torch, api, dctx, gs, batch, adj, P, W)
    h = 1e-3

    def gpu_loss(name, idx, delta):
        Q = {k: v.clone() for k, v in P.items()}
        Q[name][idx] += delta
        # the adjoint's paths (pass 1): the gradient estimates exactly this estimator
        img = api.render_primal(dctx, gs, adj, Q)
        return float((img.double() * W.double()).sum())

    # rounding of the FP32 image enters the difference quotient as ~ulp * sum|W I| / h
    img = api.render_primal(dctx, gs, adj, P)
    noise = 8 * 2.0**-24 * float((img.double() * W.double()).abs().sum()) / h
    for name, idx in [("theta", 0), ("le", 0), ("le", 1), ("le", 6), ("le", 11)]:
        fd = (gpu_loss(name, idx, h) - gpu_loss(name, idx, -h)) / (2 * h)
        an = g[name][idx]
        assert abs(an - fd) <= 1e-2 * abs(fd) + noise, (name, idx, an, fd, noise)

    # albedo texels: the oracle's frozen-sampling estimator (the rocks' lobe choice depends on albedo)
    O = oracle_mod.OracleScene(scene)
    aj = copy.copy(job)
    aj.pass_id = 1
    base = scene.params()
    off = int(scene.tex_desc[0][0])
    texg = g["tex"][off:]
    for rank in (0, 3):
        t = int(off + np.argsort(-np.abs(texg))[rank])

        def J(delta):
            live = {k: np.array(v, dtype=np.float64, copy=True) for k, v in base.items()}
            live["tex"][t] += delta
            return float((w * O.render(aj, base, pixels=pix, params_live=live)).sum())

        fd = (J(h) - J(-h)) / (2 * h)
        assert abs(g["tex"][t] - fd) <= 1e-3 * max(abs(fd), 1e-12), (t, g["tex"][t], fd)
