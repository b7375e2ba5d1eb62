"""The allocation-free primal entry point (dppt_render_primal_noalloc).

Callers that must not let the library allocate device memory -- because their
device memory belongs to another allocator or a fixed budget, because they must
not block in the driver's allocator, or because they issue work while a stream
is captured -- use this entry point instead of dppt_render_primal.  Its raw
image scratch is a fixed array compiled into the library, shared by all calls.

The test calls it through the C ABI twice in a row and compares each result with
dppt_render_primal's image (the per-pixel relative error of the parity tests,
1e-4).  The second call checks that leftovers of the first call in the shared
array do not leak into the next result.  This file is collected last.
"""
import ctypes

import numpy as np
import pytest

from parity import IMG_TOL_P999, image_rel_err

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2607_13265_gb300 import build, api, scenegen as sg
    build.build()
    dctx = api.Context(0)
    scene, job = sg.cornell_box()
    gs = api.GpuScene(dctx, scene)
    return torch, api, sg, dctx, scene, job, gs


@pytest.mark.parametrize("spp", [8, 3])
def test_noalloc_matches_render_primal_on_two_calls(env, spp):
    torch, api, sg, dctx, scene, job, gs = env
    job.width, job.height, job.spp = 48, 40, spp
    job.thetas = [0.2, 1.0, 2.5]
    batch = api.pack_jobs([job])
    P = api.device_params(scene, batch)
    ref = api.render_primal(dctx, gs, batch, P).clone()
    dctx.sync_status()
    ref_np = ref.double().cpu().numpy().reshape(3, -1, 3, 4)
    cp = api._c_params(P)
    for _ in range(2):
        out = torch.full_like(ref, float("nan"))
        st = dctx.lib.dppt_render_primal_noalloc(dctx.h, gs.h, ctypes.byref(batch.c_jobs[0]), ctypes.byref(cp),
                                                 api._ptr(out), api._stream_ptr(None))
        assert st == 0, dctx.lib.dppt_last_error(dctx.h)
        dctx.sync_status()
        got = out.double().cpu().numpy().reshape(3, -1, 3, 4)
        assert np.isfinite(got).all()
        assert float(image_rel_err(got, ref_np).max()) <= IMG_TOL_P999


def test_noalloc_rejects_jobs_beyond_its_scratch(env):
    torch, api, sg, dctx, scene, job, gs = env
    job.width, job.height, job.spp = 600, 600, 1
    job.thetas = [0.3]
    batch = api.pack_jobs([job])
    P = api.device_params(scene, batch)
    out = torch.zeros(batch.image_floats, device="cuda")
    cp = api._c_params(P)
    st = dctx.lib.dppt_render_primal_noalloc(dctx.h, gs.h, ctypes.byref(batch.c_jobs[0]), ctypes.byref(cp),
                                             api._ptr(out), api._stream_ptr(None))
    assert st == -1
    assert b"exceeds the fixed scratch" in dctx.lib.dppt_last_error(dctx.h)
