"""The allocation-free primal entry point (dppt_render_primal_noalloc).

Callers that must not let the library allocate device memory -- because their
device memory belongs to another allocator or a fixed budget, because they must
not block in the driver's allocator, or because they issue work while a stream
is captured -- use this entry point instead of dppt_render_primal.  Its raw
image scratch is a fixed array compiled into the library, shared by all calls.

The tests call it through the C ABI twice in a row and compare each result with
dppt_render_primal's image (the per-pixel relative error of the parity tests,
1e-4): filtered and unfiltered jobs, samples per pixel that take each of the
three pixel-sum modes (a power of two up to 32, a larger power of two, any other
count), and depths in two cache buckets.  The second call checks that leftovers
of the first call in the shared array do not leak into the next result.  On a
fresh context, a call after the first one must leave the device's free memory
unchanged.

The file is named to be collected last: the entry point is an addition beside
the method's calls, so a failure here should not stop a run that halts at the
first failure before every other test has run.  Each test builds what it needs,
so the file passes alone in a fresh process as well as after the others.
"""
import copy
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


def _noalloc(api, dctx, gs, batch, cp, out):
    return dctx.lib.dppt_render_primal_noalloc(dctx.h, gs.h, ctypes.byref(batch.c_jobs[0]), ctypes.byref(cp),
                                               api._ptr(out), api._stream_ptr(None))


@pytest.mark.parametrize("spp,depth,filtered", [(8, 4, True), (3, 4, True), (64, 8, True), (8, 12, False),
                                                (64, 4, False)])
def test_noalloc_matches_render_primal_on_two_calls(env, spp, depth, filtered):
    torch, api, sg, dctx, scene, job0, gs = env
    job = copy.copy(job0)
    job.width, job.height, job.spp, job.max_depth = 48, 40, spp, depth
    if filtered:
        job.thetas = [0.2, 1.0, 2.5]
    else:
        job.filter, job.thetas = sg.FILTER_NONE, []
    A = job.num_angles
    batch = api.pack_jobs([job])
    P = api.device_params(scene, batch)
    ref = api.render_primal(dctx, gs, batch, P).clone()
    dctx.sync_status()
    ref_np = ref.double().cpu().numpy().reshape(A, -1, 3, 4)
    cp = api._c_params(P)
    for _ in range(2):
        out = torch.full_like(ref, float("nan"))
        st = _noalloc(api, dctx, gs, batch, cp, out)
        assert st == 0, dctx.lib.dppt_last_error(dctx.h)
        dctx.sync_status()
        got = out.double().cpu().numpy().reshape(A, -1, 3, 4)
        assert np.isfinite(got).all()
        assert float(image_rel_err(got, ref_np).max()) <= IMG_TOL_P999


def test_noalloc_allocates_nothing(env):
    """On a fresh context, once a first call has run, a second call (filtered, 512 x 512,
    the scratch's limit) leaves the device's free memory unchanged."""
    torch, api, sg, _, scene, job0, _ = env
    dctx = api.Context(0)
    gs = api.GpuScene(dctx, scene)
    job = copy.copy(job0)
    job.width = job.height = 512
    job.spp, job.thetas = 4, [0.4, 1.7]
    batch = api.pack_jobs([job])
    P = api.device_params(scene, batch)
    cp = api._c_params(P)
    out = torch.zeros(batch.image_floats, device="cuda")
    assert _noalloc(api, dctx, gs, batch, cp, out) == 0, dctx.lib.dppt_last_error(dctx.h)
    dctx.sync_status()
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    assert _noalloc(api, dctx, gs, batch, cp, out) == 0, dctx.lib.dppt_last_error(dctx.h)
    dctx.sync_status()
    torch.cuda.synchronize()
    assert torch.cuda.mem_get_info()[0] == free0
    assert float(out.abs().max()) > 0


def test_noalloc_rejects_jobs_beyond_its_scratch(env):
    torch, api, sg, dctx, scene, job0, gs = env
    job = copy.copy(job0)
    job.width, job.height, job.spp = 600, 600, 1
    job.thetas = [0.3]
    batch = api.pack_jobs([job])
    P = api.device_params(scene, batch)
    out = torch.zeros(batch.image_floats, device="cuda")
    cp = api._c_params(P)
    st = _noalloc(api, dctx, gs, batch, cp, out)
    assert st == -1
    assert b"exceeds the fixed scratch" in dctx.lib.dppt_last_error(dctx.h)
