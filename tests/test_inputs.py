"""The seeded synthetic workloads, on CPU: each generator yields the sizes its recipe states
(triangle counts per material, image sizes, samples, depth, angles, textures) and the same
arrays on every call."""
import math

import numpy as np
import pytest

from paper_2607_13265_gb300 import scenegen as sg


def _tris_by_type(s):
    types = np.array([m.type for m in s.materials])
    counts = {}
    for mat, n in enumerate(np.bincount(np.asarray(s.tri_mat), minlength=len(s.materials))):
        counts[int(types[mat])] = counts.get(int(types[mat]), 0) + int(n)
    return counts


def test_views_by_angles_workload():
    s, jobs = sg.cornell_views()
    assert len(s.tris) == 12 and len(s.spheres) == 2 and len(s.lights) == 1
    assert [j.width for j in jobs] == [128, 183, 238, 293, 347, 402, 457, 512]
    assert all(j.width == j.height and j.spp == 16 and j.max_depth == 8 for j in jobs)
    assert sum(j.num_pixels for j in jobs) == 945_372
    for j in jobs:
        assert j.filter == sg.FILTER_POLARIZER and len(j.thetas) == 64
        assert np.allclose(j.thetas, np.arange(64) * math.pi / 64)      # 64 angles in [0, 180 deg)
    assert len({j.camera for j in jobs}) == 8


def test_icosphere_workload():
    s, job = sg.icosphere_scene()
    assert _tris_by_type(s) == {sg.MAT_CONDUCTOR_GGX: 50_000, sg.MAT_PLASTIC_GGX: 2, sg.MAT_EMITTER: 2}
    assert (job.width, job.height, job.spp, job.max_depth) == (256, 256, 64, 8)
    assert [tuple(d[1:]) for d in s.tex_desc] == [(128, 128, 3), (128, 128, 1)]


def test_rocks_workload():
    s, job = sg.rocks_scene()
    # 8 rocks of 12,500 triangles (rough dielectric), a diffuse ground quad and the light
    assert _tris_by_type(s) == {sg.MAT_PLASTIC_GGX: 100_000, sg.MAT_DIFFUSE: 2, sg.MAT_EMITTER: 2}
    assert (job.width, job.height, job.spp, job.max_depth) == (512, 512, 32, 16)
    assert job.filter == sg.FILTER_QWP_POLARIZER and job.thetas == pytest.approx([math.pi / 4])


def test_large_workload():
    s, job = sg.large_scene()
    assert len(s.tris) == 500_018 and len(s.lights) == 4
    assert (job.width, job.height, job.spp, job.max_depth, len(job.thetas)) == (1024, 1024, 128, 12, 16)
    sizes = sorted(tuple(d[1:]) for d in s.tex_desc)
    assert (1024, 1024, 3) in sizes and (1024, 1024, 1) in sizes
    types = {m.type for m in s.materials}
    assert {sg.MAT_DIFFUSE, sg.MAT_CONDUCTOR_GGX, sg.MAT_PLASTIC_GGX, sg.MAT_POLARIZER_SHEET,
            sg.MAT_RETARDER_SHEET} <= types


def test_deep_stack_workload():
    s, job = sg.deep_stack_scene()
    counts = _tris_by_type(s)
    assert counts[sg.MAT_POLARIZER_SHEET] == 2 * 85 and len(s.sheet) == 85
    assert counts[sg.MAT_CONDUCTOR_GGX] == 8_000
    assert np.degrees(s.sheet[0]) == pytest.approx(0.0) and np.degrees(s.sheet[-1]) == pytest.approx(90.0)
    assert (job.width, job.height, job.spp) == (1280, 720, 1)


@pytest.mark.parametrize("make", [sg.icosphere_scene, sg.rocks_scene, sg.cornell_views, sg.mixed_scene,
                                  lambda: sg.normal_map_scene()])
def test_generators_are_deterministic(make):
    a, b = make()[0], make()[0]
    for name in ("verts", "tris", "uvs", "tri_mat", "spheres", "lights"):
        assert np.array_equal(np.asarray(getattr(a, name)), np.asarray(getattr(b, name))), name
    assert np.array_equal(np.asarray(a.params()["tex"]), np.asarray(b.params()["tex"]))
