"""Pins of the oracle's normal-mapped shading (tangent-space maps, n_t = 2 c - 1; shading
normal normalize(n_t.x T + n_t.y B + n_t.z N) with T = dP/du of the triangle made normal to
N and B = N x T) and of its texel derivatives.

* A flat map (n_t = (0, 0, 1) everywhere) reproduces the renderer without normal maps,
  path by path (paths that part by a rounding-level near-edge hit are excluded).
* The cached suffix replay equals the tape on the normal maps' texel gradients.
* The texel gradients equal central differences of the frozen-sampling estimator, and so
  do the normal-mapped materials' own albedo, roughness and index-of-refraction
  gradients."""
import copy

import numpy as np
import pytest

from paper_2607_13265_gb300 import scenegen as sg


def test_flat_normal_map_is_the_geometric_normal(oracle_mod):
    sf, job = sg.normal_map_scene(flat=True)
    s0, _ = sg.normal_map_scene(flat=True)
    for m in s0.materials:
        m.normal_tex = -1
    _, pf, sig_f = oracle_mod.OracleScene(sf).render(job, sf.params(), paths=True)
    _, p0, sig_0 = oracle_mod.OracleScene(s0).render(job, s0.params(), paths=True)
    same = sig_f == sig_0
    assert same.mean() >= 0.99
    assert np.abs(pf[same] - p0[same]).max() <= 1e-12 * max(1.0, np.abs(p0).max())


def _setup(oracle_mod):
    s, job = sg.normal_map_scene()
    o = oracle_mod.OracleScene(s)
    P = s.params()
    aj = copy.copy(job)
    aj.pass_id = 1
    img = o.render(aj, P)
    dI = np.random.default_rng(1).normal(size=img.shape)
    return s, o, P, aj, dI


def test_bumps_change_the_image(oracle_mod):
    s, o, P, aj, dI = _setup(oracle_mod)
    s0, _ = sg.normal_map_scene(flat=True)
    img = o.render(aj, P)
    img0 = oracle_mod.OracleScene(s0).render(aj, s0.params())
    assert np.abs(img - img0).max() > 0.05 * np.abs(img0).max()


def test_normal_map_gradient_replay_equals_tape(oracle_mod):
    s, o, P, aj, dI = _setup(oracle_mod)
    gt = o.gradient(aj, P, dI, mode="tape")["tex"]
    gr = o.gradient(aj, P, dI, mode="replay")["tex"]
    maps = slice(0, 3 * 16 * 16 * 3)           # the three normal maps come first
    assert np.linalg.norm(gt[maps]) > 0
    assert np.linalg.norm(gr - gt) <= 1e-12 * np.linalg.norm(gt)


def test_normal_map_gradient_matches_central_differences(oracle_mod):
    s, o, P, aj, dI = _setup(oracle_mod)
    g = o.gradient(aj, P, dI, mode="tape")["tex"]
    h = 1e-5
    for t in np.argsort(-np.abs(g[:3 * 16 * 16 * 3]))[:4]:
        def J(d):
            live = {k: np.array(v, dtype=np.float64, copy=True) for k, v in P.items()}
            live["tex"][t] += d
            return float((dI * o.render(aj, P, params_live=live)).sum())
        fd = (J(h) - J(-h)) / (2 * h)
        assert abs(g[t] - fd) <= 1e-6 * abs(fd), (t, g[t], fd)


def test_normal_mapped_material_parameters_match_central_differences(oracle_mod):
    """On normal-mapped materials the albedo and roughness texels and the index of refraction
    are differentiated too: both routes against central differences."""
    s, o, P, aj, dI = _setup(oracle_mod)
    gt = o.gradient(aj, P, dI, mode="tape")
    gr = o.gradient(aj, P, dI, mode="replay")
    (r_off, rw, rh, _), (a_off, aw, ah, ac) = s.tex_desc[3], s.tex_desc[4]
    checks = [("ior", 0)]
    for off, n in ((r_off, rw * rh), (a_off, aw * ah * ac)):
        block = np.abs(gt["tex"][off:off + n])
        checks += [("tex", int(off + k)) for k in np.argsort(-block)[:3]]
    h = 1e-5
    for name, t in checks:
        def J(d):
            live = {k: np.array(v, dtype=np.float64, copy=True) for k, v in P.items()}
            live[name].reshape(-1)[t] += d
            return float((dI * o.render(aj, P, params_live=live)).sum())
        fd = (J(h) - J(-h)) / (2 * h)
        assert gt[name][t] != 0.0, (name, t)
        assert abs(gt[name][t] - fd) <= 1e-6 * max(1.0, abs(fd)), (name, t, gt[name][t], fd)
        assert gr[name][t] == pytest.approx(gt[name][t], rel=1e-10, abs=1e-12)
