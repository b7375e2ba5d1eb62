"""Pins of the oracle's hybrid cached replay (Sec. 4.4, Eq. hybrid_decision) against the
taped reverse AD (conventional AD, the exact derivative of the same estimator).

* k = 1 caches every suffix: it is the cached suffix replay, exact.
* gamma = 0, eps = +inf recomputes every missing suffix: exact for every k.
* gamma = 0, eps = 0 inverts wherever det != 0: exact up to rounding on these scenes.
* the scalar route drops the suffix's polarization: exact on an ideal depolarizer (the
  diffuse furnace), biased where a polarization-sensitive vertex follows a nearly
  depolarizing block -- the bias vanishes as gamma -> 0.
* route counts: k = 1 uses only checkpoints; with k > 1 a fraction ~1/k of the
  channel-vertices is served from checkpoints."""
import numpy as np
import pytest

from paper_2607_13265_gb300 import scenegen as sg

INF = float("inf")


def _rel(g, o):
    n = np.linalg.norm(o)
    return float(np.linalg.norm(g - o) / n) if n > 0 else float(np.linalg.norm(g))


def _case(oracle_mod, name):
    if name == "deep":
        s, job = sg.deep_stack_scene(num_sheets=20, width=8, height=6, spp=2, depth=40, freq=6, tex_res=16)
    elif name == "mixed":
        s, job = sg.mixed_scene(width=12, spp=2, depth=6)
    else:
        s, job = sg.cornell_box()
        job.width = job.height = 12
    o = oracle_mod.OracleScene(s)
    P = s.params()
    dI = np.random.default_rng(1).normal(size=o.render(job, P).shape)
    tape = o.gradient(job, P, dI, mode="tape")
    keys = [k for k in ("tex", "ior", "le", "sheet", "theta") if tape[k].size and np.linalg.norm(tape[k]) > 0]
    return o, job, P, dI, tape, keys


@pytest.mark.parametrize("name", ["deep", "mixed", "cornell"])
def test_exact_configurations(oracle_mod, name):
    o, job, P, dI, tape, keys = _case(oracle_mod, name)
    for k, gamma, eps in [(1, 0.3, 1e-6), (4, 0.0, INF), (8, 0.0, INF), (16, 0.0, INF), (4, 0.0, 0.0)]:
        g, routes = o.gradient_hybrid(job, P, dI, k, gamma, eps)
        for key in keys:
            assert _rel(g[key], tape[key]) < 1e-9, (name, k, gamma, eps, key, _rel(g[key], tape[key]))
        if k == 1:
            assert routes["scalar"] == routes["inverse"] == routes["recompute"] == 0
        else:
            total = sum(routes.values())
            assert routes["cached"] < total and routes["scalar"] == 0
            if eps == INF:
                assert routes["inverse"] == 0 and routes["recompute"] > 0


def test_scalar_route_exact_on_depolarizer(oracle_mod):
    s, job = sg.furnace_scene(0.5, 1.0)
    job.max_depth = 12
    o = oracle_mod.OracleScene(s)
    P = s.params()
    dI = np.random.default_rng(2).normal(size=o.render(job, P).shape)
    tape = o.gradient(job, P, dI, mode="tape")["tex"]
    g, routes = o.gradient_hybrid(job, P, dI, 4, 0.5, 1e-6)
    assert routes["scalar"] > 0 and routes["inverse"] == routes["recompute"] == 0
    assert _rel(g["tex"], tape) < 1e-12


def test_scalar_route_bias_vanishes_with_gamma(oracle_mod):
    """Behind a diffuse bounce the block throughput is rank one; with a glass vertex after it
    DI stays small, the scalar route drops the polarization the IOR derivative needs."""
    o, job, P, dI, tape, keys = _case(oracle_mod, "cornell")
    big, r_big = o.gradient_hybrid(job, P, dI, 4, 0.2, 1e-6)
    small, r_small = o.gradient_hybrid(job, P, dI, 4, 1e-4, 1e-6)
    assert r_big["scalar"] > r_small["scalar"]
    assert _rel(big["ior"], tape["ior"]) > 1e-4
    assert _rel(small["ior"], tape["ior"]) < 1e-9
    assert _rel(big["tex"], tape["tex"]) < 1e-9      # the diffuse albedo needs only s0


def test_invalid_interval(oracle_mod):
    o, job, P, dI, tape, keys = _case(oracle_mod, "mixed")
    with pytest.raises(AssertionError):
        o.gradient_hybrid(job, P, dI, 0, 0.0, INF)
