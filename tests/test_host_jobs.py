"""The binding's job packing, on CPU: the offsets the C ABI reads.  Images are float32
[angle][height][width][3][4] per job, laid back to back in job order; a job without a camera
filter has one image and takes no entry of the angle vector; a filtered job's angles follow
those of the filtered jobs before it.  Expected values are computed here from that layout."""
import math

import numpy as np
import pytest
import torch

from paper_2607_13265_gb300 import api, scenegen as sg

F_NONE, F_POL, F_QWP = sg.FILTER_NONE, sg.FILTER_POLARIZER, sg.FILTER_QWP_POLARIZER


def _jobs():
    return [
        sg.Job(camera=0, width=5, height=3, spp=2, max_depth=3, seed=7, stream=1),
        sg.Job(camera=1, width=4, height=4, spp=3, max_depth=5, seed=8, filter=F_POL, thetas=[0.1, 0.7, 2.0]),
        sg.Job(camera=0, width=2, height=7, spp=1, max_depth=2, filter=F_QWP, thetas=[math.pi / 4]),
        sg.Job(camera=2, width=1, height=1, spp=4, max_depth=8, pass_id=1),
        sg.Job(camera=0, width=3, height=2, spp=5, max_depth=4, filter=F_POL, thetas=[-0.3, 1.1]),
    ]


def test_image_and_angle_offsets():
    jobs = _jobs()
    b = api.pack_jobs(jobs)
    sizes = [a * w * h * 12 for a, w, h in [(1, 5, 3), (3, 4, 4), (1, 2, 7), (1, 1, 1), (2, 3, 2)]]
    starts = np.concatenate([[0], np.cumsum(sizes)[:-1]])
    assert b.offsets == starts.tolist() and b.image_floats == sum(sizes)
    assert all(o % 4 == 0 for o in b.offsets)                 # the ABI wants whole float4s
    assert [b.c_jobs[i].num_angles for i in range(5)] == [1, 3, 1, 1, 2]
    assert [b.c_jobs[i].theta_offset for i in range(5)] == [0, 0, 3, 0, 4]
    assert np.array_equal(b.theta, [0.1, 0.7, 2.0, math.pi / 4, -0.3, 1.1])
    for i, j in enumerate(jobs):
        c = b.c_jobs[i]
        assert (c.camera, c.width, c.height, c.spp, c.max_depth, c.filter) == \
            (j.camera, j.width, j.height, j.spp, j.max_depth, j.filter)
        assert (c.seed, c.stream, c.pass_, c.out_offset) == (j.seed, j.stream, j.pass_id, b.offsets[i])
        # a filtered job's slice of the angle vector is its own angles, in order
        if j.filter != F_NONE:
            th = b.theta[c.theta_offset:c.theta_offset + c.num_angles]
            assert np.array_equal(th, j.thetas)


def test_blocks_tile_the_image_without_overlap():
    b = api.pack_jobs(_jobs())
    cover = np.zeros(b.image_floats, np.int32)
    for i, j in enumerate(b.jobs):
        cover[b.offsets[i]:b.offsets[i] + j.num_angles * j.num_pixels * 12] += 1
    assert np.all(cover == 1)


def test_path_signature_offsets():
    jobs = _jobs()
    sig = torch.zeros(sum(j.num_paths for j in jobs), dtype=torch.int32)
    b = api.pack_jobs(jobs, path_sig=sig)
    start = 0
    for i, j in enumerate(jobs):
        assert b.c_jobs[i].path_sig == sig.data_ptr() + 4 * start
        start += j.num_paths


def test_no_filtered_job_keeps_a_placeholder_angle():
    b = api.pack_jobs([sg.Job(camera=0, width=2, height=2, spp=1, max_depth=1)])
    assert b.theta.shape == (1,) and b.c_jobs[0].theta_offset == 0


def test_filtered_job_without_angles_is_rejected():
    jobs = _jobs()
    jobs[2].thetas = []
    with pytest.raises(ValueError, match="job 2"):
        api.pack_jobs(jobs)


def test_adjoint_jobs_change_only_the_pass():
    jobs = _jobs()
    adj = api.adjoint_jobs(jobs)
    for j, a in zip(jobs, adj):
        assert a.pass_id == 1 and a is not j
        assert (a.camera, a.width, a.height, a.spp, a.max_depth, a.seed, a.stream, a.filter, a.thetas) == \
            (j.camera, j.width, j.height, j.spp, j.max_depth, j.seed, j.stream, j.filter, j.thetas)
    assert [j.pass_id for j in jobs] == [0, 0, 0, 1, 0]


def test_raw_batch_drops_the_filters_and_keeps_the_paths():
    """The fused L2 loss reads each job's raw image [H][W][3][4] at its raw offset: the raw
    batch has the same jobs without their filters, one image each, back to back."""
    jobs = _jobs()
    rb = api.raw_batch(api.pack_jobs(jobs))
    sizes = [j.num_pixels * 12 for j in jobs]
    assert rb.offsets == np.concatenate([[0], np.cumsum(sizes)[:-1]]).tolist()
    assert rb.image_floats == sum(sizes)
    for i, j in enumerate(jobs):
        c = rb.c_jobs[i]
        assert c.filter == F_NONE and c.num_angles == 1
        assert (c.camera, c.width, c.height, c.spp, c.max_depth, c.seed, c.stream, c.pass_) == \
            (j.camera, j.width, j.height, j.spp, j.max_depth, j.seed, j.stream, j.pass_id)
    assert jobs[1].filter == F_POL and len(jobs[1].thetas) == 3      # the caller's jobs are untouched
