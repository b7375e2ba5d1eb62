"""Closed-form pins of the oracle's light transport: next-event estimation with multiple
importance sampling, smooth-dielectric transmission with its radiance scaling, and the
frame rotations of the Fresnel and GGX pBRDF operators.

Each check compares the FP64 oracle with a result that radiometry and optics fix, not
with the oracle's own formulas:
  * a Lambertian floor lit by two one-sided parallelogram lights: the pixel equals
    (albedo / pi) * sum_l L_l * Phi_l, where Phi_l is the cosine-weighted solid angle of
    light l from Lambert's polygon formula (itself checked against quadrature).  The
    estimator of Eq. 2 with NEE + power-heuristic MIS and the BSDF-sampling-only estimator
    (the same quads as emitting surfaces) must both reach it within a Monte Carlo bound;
  * one smooth interface seen from either side: every transmitted path carries exactly
    L (eta_cam / eta_light)^2 (radiance scales with the squared index of the medium it
    enters) and the s/p split of the textbook transmittances T_s = 1 - |r_s|^2,
    T_p = 1 - |r_p|^2; a glass slab carries the product of two such transmissions;
  * specular reflection of polarized light: every reflected path of a smooth dielectric
    carries M(r_s, r_p) Le / F exactly, and rough GGX lobes (conductor, and a rough
    dielectric at Brewster's angle) approach the same Mueller matrix as the roughness
    goes to 0.01 -- with the light's Stokes vector given in a frame that shares its x
    axis with the s axis, so that every frame rotation on the way must cancel.

The building blocks are held the same way: Philox against numpy's, the Fresnel
coefficients at Brewster's angle, the GGX normalization and Smith masking identities,
the polarizer as a projector, Malus's law, the white furnace, cached suffix replay and
the hybrid's exact configurations against taped AD, basic polarized PRB's O(sigma)
convergence behind depolarizers (Sec. 4.1), and a flat normal map against the geometric
normal.
test_planted_mistake_is_caught builds copies of oracle.cpp with one line changed (a
dropped term, a swapped operand, an inverted rotation or factor, a wrong sign or index)
and requires the check named for each to fail on it.
"""
import concurrent.futures
import math
import os
import subprocess

import numpy as np
import pytest

from paper_2607_13265_gb300 import scenegen as sg

ORACLE_CPP = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "oracle", "oracle.cpp")


# ---------------------------------------------------------------- textbook optics
def polygon_phi(x, n, corners) -> float:
    """Cosine-weighted solid angle int cos(theta) dw of a planar polygon seen from x with
    normal n (Lambert's formula: half the sum over edges of the edge's angle times the
    normal's component along the edge plane's normal); the polygon must lie above x's
    horizon.  Irradiance from a uniform Lambertian emitter of radiance L is L * Phi."""
    u = [(np.asarray(c, float) - x) / np.linalg.norm(np.asarray(c, float) - x) for c in corners]
    tot = 0.0
    for i in range(len(u)):
        a, b = u[i], u[(i + 1) % len(u)]
        cr = np.cross(a, b)
        tot += math.acos(float(np.clip(a @ b, -1.0, 1.0))) * float(n @ cr) / float(np.linalg.norm(cr))
    return abs(tot) / 2.0


def fresnel_rs_rp(cos_i: float, n1: float, n2: complex):
    """Fresnel amplitude coefficients (Born & Wolf) from index n1 into n2 (complex for a
    conductor), principal root for the refracted cosine."""
    cos_t = np.sqrt(1.0 - (n1 / n2) ** 2 * (1.0 - cos_i * cos_i) + 0j)
    rs = (n1 * cos_i - n2 * cos_t) / (n1 * cos_i + n2 * cos_t)
    rp = (n2 * cos_i - n1 * cos_t) / (n2 * cos_i + n1 * cos_t)
    return complex(rs), complex(rp)


def reflection_mueller(rs: complex, rp: complex) -> np.ndarray:
    """Mueller matrix of a reflection in the s/p frames: A, B from |r_s|^2, |r_p|^2 and
    C + iS = r_s conj(r_p), in the block form the method's frames are stated with."""
    A = (abs(rs) ** 2 + abs(rp) ** 2) / 2
    B = (abs(rs) ** 2 - abs(rp) ** 2) / 2
    z = rs * np.conj(rp)
    return np.array([[A, B, 0, 0], [B, A, 0, 0], [0, 0, z.real, z.imag], [0, 0, -z.imag, z.real]])


def test_lambert_polygon_formula_matches_quadrature():
    """The closed form used below against a midpoint quadrature of cos cos / r^2 dA."""
    x, n = np.zeros(3), np.array([0.0, 1.0, 0.0])
    for o, e1, e2 in sg.LIGHT_QUADS:
        o, e1, e2 = (np.asarray(v, float) for v in (o, e1, e2))
        N = 400
        s = (np.arange(N) + 0.5) / N
        area = np.linalg.norm(np.cross(e1, e2))
        nl = np.cross(e1, e2) / area
        P = o + s[:, None, None] * e1 + s[None, :, None] * e2
        d = x - P
        r2 = (d * d).sum(-1)
        quad = float(((d @ nl) * (-(d @ n)) / r2 ** 2).mean() * area)
        assert polygon_phi(x, n, [o, o + e1, o + e1 + e2, o + e2]) == pytest.approx(quad, rel=1e-6)


# ---------------------------------------------------------------- checks (raise AssertionError)
def check_nee_mis(make, surface_emission=False):
    """Direct light on a Lambertian floor from two one-sided parallelogram lights: NEE with
    the power heuristic (or, with surface_emission, BSDF sampling alone) against
    (a / pi) sum_l L_l Phi_l, 5 standard errors of the path mean (10^6 paths) plus 0.02% for
    the camera's footprint."""
    albedo, le = np.array([0.6, 0.5, 0.4]), (5.0, 3.0)
    s, job = sg.polygon_light_scene(tuple(albedo), le, surface_emission=surface_emission,
                                    spp=262144)
    _, paths, _ = make(s).render(job, s.params(), paths=True)
    x, n = np.zeros(3), np.array([0.0, 1.0, 0.0])
    E = 0.0
    for (o, e1, e2), L in zip(sg.LIGHT_QUADS, le):
        o, e1, e2 = (np.asarray(v, float) for v in (o, e1, e2))
        E += L * polygon_phi(x, n, [o, o + e1, o + e1 + e2, o + e2])
    expect = albedo / math.pi * E
    s0 = paths[:, :, 0]
    mean, sem = s0.mean(0), s0.std(0) / math.sqrt(s0.shape[0])
    assert np.all(np.abs(mean - expect) <= 5 * sem + 2e-4 * expect), (mean, expect, sem)
    assert np.all(paths[:, :, 1:] == 0.0)


def check_transmission(make, camera_inside, theta=35.0, ior=1.5, L=1.3):
    """One smooth interface between the camera and an unpolarized light: every transmitted
    path carries s0 = L (eta_cam / eta_light)^2 and s1 / s0 = (T_s - T_p) / (T_s + T_p) with
    x along s (s2 = s3 = 0); the transmitted fraction is the unpolarized transmittance."""
    s, job = sg.glass_interface_scene(ior, theta, camera_inside=camera_inside, le=L, spp=4096)
    _, paths, _ = make(s).render(job, s.params(), paths=True)
    n_cam, n_light = (ior, 1.0) if camera_inside else (1.0, ior)
    rs, rp = fresnel_rs_rp(math.cos(math.radians(theta)), n_cam, n_light)
    Ts, Tp = 1 - abs(rs) ** 2, 1 - abs(rp) ** 2
    v = paths[:, 0]
    hit = v[:, 0] != 0.0
    assert np.allclose(v[hit, 0], L * (n_cam / n_light) ** 2, rtol=1e-9)
    # the 0.01 deg field of view spreads the incidence angle by ~1e-4 rad
    assert np.allclose(v[hit, 1] / v[hit, 0], (Ts - Tp) / (Ts + Tp), atol=1e-4)
    assert np.allclose(v[hit, 2:], 0.0, atol=1e-4 * L)
    T = (Ts + Tp) / 2
    assert abs(hit.mean() - T) <= 5 * math.sqrt(T * (1 - T) / hit.size)


def check_slab(make, theta=40.0, ior=1.5, L=1.0):
    """A glass slab (two parallel interfaces) in front of an unpolarized light: the
    (eta)^2 factors of entering and leaving cancel, and each path transmitted twice
    carries the product of the two transmissions over the two unpolarized sampling
    probabilities: s0 = L (1 + b^2), s1 = 2 L b with b = (T_s - T_p) / (T_s + T_p)."""
    s, job = sg.glass_interface_scene(ior, theta, slab=0.2, le=L, spp=4096)
    _, paths, _ = make(s).render(job, s.params(), paths=True)
    rs, rp = fresnel_rs_rp(math.cos(math.radians(theta)), 1.0, ior)
    Ts, Tp = 1 - abs(rs) ** 2, 1 - abs(rp) ** 2
    b = (Ts - Tp) / (Ts + Tp)
    v = paths[:, 0]
    hit = v[:, 0] != 0.0
    assert np.allclose(v[hit, 0], L * (1 + b * b), atol=1e-5 * L)
    assert np.allclose(v[hit, 1], 2 * L * b, atol=1e-4 * L)
    T = (Ts + Tp) / 2
    assert abs(hit.mean() - T * T) <= 5 * math.sqrt(T * T * (1 - T * T) / hit.size)


LE_POL = np.array([1.0, 0.3, 0.5, 0.2])


def check_smooth_reflection(make, theta=40.0, ior=1.5):
    """Polarized light reflected by a smooth dielectric: every reflected path carries
    M(r_s, r_p) Le / F with F = (|r_s|^2 + |r_p|^2) / 2, the light's x axis being the s axis."""
    s, job = sg.specular_limit_scene("smooth", theta, ior=ior, le=LE_POL, spp=2048)
    _, paths, _ = make(s).render(job, s.params(), paths=True)
    M = reflection_mueller(*fresnel_rs_rp(math.cos(math.radians(theta)), 1.0, ior))
    v = paths[:, 0]
    hit = v[:, 0] != 0.0
    assert hit.sum() > 20
    assert np.allclose(v[hit], (M @ LE_POL) / M[0, 0], atol=1e-3)


def check_rough_limit(make, kind, theta, light_size=8.0, s0_tol=0.05):
    """A GGX lobe of roughness 0.01 reflects polarized light as its smooth limit does: the
    pixel's Stokes ratios s_k / s0 match (M Le)_k / (M Le)_0 to 0.02 (M the reflection
    Mueller matrix at the mirror angle), and with a light covering the lobe s0 matches
    (M Le)_0 to s0_tol.  A small light (light_size 0.4 at distance 10) leaves a large part
    of the estimate to next-event estimation."""
    s, job = sg.specular_limit_scene(kind, theta, roughness=0.01, le=LE_POL, spp=16384, light_size=light_size)
    img = make(s).render(job, s.params())[0]
    n2 = complex(0.2, 3.0) if kind == "conductor" else 1.5
    ref = reflection_mueller(*fresnel_rs_rp(math.cos(math.radians(theta)), 1.0, n2)) @ LE_POL
    px = img[:, 0, :].mean(0)
    assert px[0] > 0
    assert np.allclose(px / px[0], ref / ref[0], atol=0.02), (px / px[0], ref / ref[0])
    if s0_tol is not None:
        assert px[0] == pytest.approx(ref[0], rel=s0_tol), (px[0], ref[0])


class Oracle:
    """The oracle a check runs on: the oracle's own library, or a copy built from oracle.cpp
    with one line changed.  Called with a scene it returns that library's OracleScene."""

    def __init__(self, mod, library=None):
        self.mod, self.library = mod, library

    def __call__(self, s):
        return self.mod.OracleScene(s, library=self.library)


def _real(oracle_mod):
    return Oracle(oracle_mod)


# ---------------------------------------------------------------- building blocks
# The checks below hold the oracle's building blocks and its replay algebra; each expected
# value comes from a published definition, a textbook closed form or the other derivative
# route, so that the planted mistakes further down have something to fail against.
def check_philox(make):
    """Philox4x64-10 (Salmon et al. 2011) against numpy.random.Philox, which advances its
    counter before producing a block."""
    rng = np.random.default_rng(5)
    for _ in range(8):
        key = rng.integers(0, 2**63, 2, dtype=np.uint64)
        ctr = rng.integers(0, 2**63, 4, dtype=np.uint64)
        ref = np.random.Philox(key=key, counter=ctr).random_raw(4)
        nxt = ctr.copy()
        nxt[0] += np.uint64(1)
        assert np.array_equal(make.mod.philox4x64(nxt, key, library=make.library), ref)


def check_uniforms(make):
    """The uniforms of (path, vertex): u = (w >> 8) 2^-24 for the low then the high 32-bit
    half of each Philox output word, key (seed ^ pass * 0x9E3779B97F4A7C15, stream)."""
    seed, pas, stream, path, vertex = 91, 1, 2, 987654321, 3
    k0 = np.uint64(seed) ^ np.uint64((pas * 0x9E3779B97F4A7C15) % 2**64)
    ref = np.random.Philox(key=[k0, np.uint64(stream)], counter=[path - 1, vertex, 0, 0]).random_raw(4)
    words = []
    for x in ref:
        words += [int(x) & 0xFFFFFFFF, int(x) >> 32]
    expect = np.array([(w >> 8) / 2**24 for w in words])
    assert np.array_equal(make.mod.uniforms(seed, pas, stream, path, vertex, library=make.library), expect)


def check_brewster(make, n=1.5):
    """At Brewster's angle (tan theta = n) r_p = 0 and r_s = (1 - n^2) / (1 + n^2): the
    reflection is A = B = r_s^2 / 2, C = S = 0."""
    A, B, C, S = make.mod.fresnel_reflect(math.cos(math.atan(n)), 1.0, n, library=make.library)
    rs = (1 - n * n) / (1 + n * n)
    assert A == pytest.approx(rs * rs / 2, rel=1e-12) and B == pytest.approx(rs * rs / 2, rel=1e-12)
    assert abs(C) < 1e-15 and abs(S) < 1e-15


def _ggx_knots(alpha):
    return [0.0, max(0.0, 1.0 - 4.0 * alpha * alpha), 1.0]


def check_ggx_area(make, alpha=0.3):
    """The GGX microfacet normals cover the macro-surface once: 2 pi int_0^1 D(mu) mu dmu = 1."""
    integrate = pytest.importorskip("scipy.integrate")
    D = lambda mu: make.mod.ggx(mu, 1.0, 1.0, alpha, library=make.library)[0]
    k = _ggx_knots(alpha)
    area = sum(integrate.quad(lambda m: D(m) * m, a, b, epsabs=1e-13, epsrel=1e-11, limit=400)[0]
               for a, b in zip(k[:-1], k[1:]) if b > a)
    assert 2.0 * math.pi * area == pytest.approx(1.0, rel=1e-8)


def check_ggx_masking(make, alpha=0.5, theta_o=1.0):
    """Smith masking normalizes the visible projected area (Heitz 2014):
    G1(o) int max(0, o.h) D(h) dw_h = cos(theta_o).  It ties G1's alpha to D's."""
    integrate = pytest.importorskip("scipy.integrate")
    D = lambda mu: make.mod.ggx(mu, 1.0, 1.0, alpha, library=make.library)[0]
    so, co = math.sin(theta_o), math.cos(theta_o)

    def inner(mu):
        s = math.sqrt(max(0.0, 1.0 - mu * mu))
        return integrate.quad(lambda ph: max(0.0, so * s * math.cos(ph) + co * mu), 0.0, math.pi,
                              epsabs=1e-12, limit=200)[0] * D(mu)

    k = _ggx_knots(alpha)
    proj = 2.0 * sum(integrate.quad(inner, a, b, epsabs=1e-10, epsrel=1e-8, limit=200)[0]
                     for a, b in zip(k[:-1], k[1:]) if b > a)
    g1 = make.mod.ggx(1.0, co, 1.0, alpha, library=make.library)[1]
    assert g1 * proj == pytest.approx(co, rel=1e-6)


def check_polarizer(make):
    """The camera's ideal linear polarizer at theta, with its transmission axis along the
    sensor's x axis at theta = 0: a rank-1 projector that sends unpolarized light to
    (1, cos 2 theta, sin 2 theta, 0) / 2."""
    for th in (0.4, 1.3):
        P = make.mod.camera_filter(sg.FILTER_POLARIZER, th, library=make.library)
        assert np.allclose(P @ P, P, atol=1e-15)
        assert np.allclose(P @ [1, 0, 0, 0], [0.5, 0.5 * math.cos(2 * th), 0.5 * math.sin(2 * th), 0], atol=1e-15)


def check_malus(make, alpha=0.3, theta=1.1, L=2.0):
    """Unpolarized light through a sheet polarizer at alpha, then the camera polarizer at
    theta: Malus's law, I = (L / 2) cos^2(theta - alpha)."""
    s, job = sg.malus_scene(alpha, le=L)
    job.thetas = [theta]
    img = make(s).render(job, s.params())
    assert np.allclose(img[0, :, :, 0], 0.5 * L * math.cos(theta - alpha) ** 2, rtol=1e-6, atol=1e-9)


def check_furnace(make, a=0.6, e=1.5, depth=3):
    """A closed diffuse box that emits e everywhere: every path carries e sum_{k<depth} a^k,
    whatever its directions (cosine sampling weight a per bounce)."""
    s, job = sg.furnace_scene(a, e)
    job.max_depth = depth
    img = make(s).render(job, s.params())
    assert np.allclose(img[0, :, :, 0], e * sum(a**k for k in range(depth)), rtol=1e-12)


def check_tape_equals_replay(make):
    """Cached suffix replay (Sec. 4.3) against conventional taped AD over the whole path, on a
    small scene with every material: a wrong suffix index, a transposed adjoint-row update
    or a dropped term of the fold L_v = E_v + W_v L_{v+1} changes only the replay."""
    s, job = sg.mixed_scene(width=10, spp=2, depth=5)
    o = make(s)
    img = o.render(job, s.params())
    dI = np.random.default_rng(2).normal(size=img.shape)
    g1 = o.gradient(job, s.params(), dI, mode="tape")
    g2 = o.gradient(job, s.params(), dI, mode="replay")
    for k in g1:
        if len(g1[k]) == 0:
            continue
        assert np.linalg.norm(g1[k]) > 0, k
        assert np.allclose(g1[k], g2[k], rtol=1e-9, atol=1e-10 * np.abs(g1[k]).max()), k


def test_nee_mis_matches_polygon_irradiance(oracle_mod):
    check_nee_mis(_real(oracle_mod))


def test_bsdf_sampling_matches_polygon_irradiance(oracle_mod):
    check_nee_mis(_real(oracle_mod), surface_emission=True)


@pytest.mark.parametrize("inside", [False, True])
def test_transmission_radiance_and_polarization(oracle_mod, inside):
    check_transmission(_real(oracle_mod), inside)


def test_glass_slab(oracle_mod):
    check_slab(_real(oracle_mod))


def test_smooth_reflection_of_polarized_light(oracle_mod):
    check_smooth_reflection(_real(oracle_mod))


@pytest.mark.parametrize("kind,theta,size", [("conductor", 50.0, 8.0), ("conductor", 50.0, 0.4),
                                             ("plastic", math.degrees(math.atan(1.5)), 8.0)])
def test_rough_lobe_specular_limit(oracle_mod, kind, theta, size):
    check_rough_limit(_real(oracle_mod), kind, theta, light_size=size, s0_tol=0.05 if size > 1 else None)


def test_rough_dielectric_at_brewster_is_s_polarized(oracle_mod):
    """Brewster's angle with the specular lobe alone: whatever the light's polarization,
    the reflected light is polarized along s (s1 = s0), as for a smooth interface."""
    s, job = sg.specular_limit_scene("plastic", math.degrees(math.atan(1.5)), roughness=0.01, le=LE_POL,
                                     spp=16384)
    px = oracle_mod.OracleScene(s).render(job, s.params())[0][:, 0, :].mean(0)
    assert px[1] / px[0] == pytest.approx(1.0, abs=2e-3)
    assert abs(px[2]) < 2e-3 * px[0] and abs(px[3]) < 2e-3 * px[0]


def check_hybrid_exact(make, k, gamma, eps):
    """Hybrid cached replay (Sec. 4.4) in a configuration that recovers every missing suffix
    exactly (gamma = 0 with eps = 0: inversion wherever det != 0, else recomputation; eps =
    inf: recomputation only) equals taped AD on a small scene with every material."""
    s, job = sg.mixed_scene(width=12, spp=2, depth=6)
    o = make(s)
    P = s.params()
    dI = np.random.default_rng(1).normal(size=o.render(job, P).shape)
    tape = o.gradient(job, P, dI, mode="tape")
    g, routes = o.gradient_hybrid(job, P, dI, k, gamma, eps)
    assert routes["inverse" if eps == 0.0 else "recompute"] > 0
    for key in ("tex", "ior", "le", "sheet", "theta"):
        if tape[key].size and np.linalg.norm(tape[key]) > 0:
            assert np.linalg.norm(g[key] - tape[key]) < 1e-9 * np.linalg.norm(tape[key]), key


def check_hybrid_scalar_furnace(make):
    """The hybrid's scalar route is exact behind ideal depolarizers (the diffuse furnace)."""
    s, job = sg.furnace_scene(0.5, 1.0)
    job.max_depth = 12
    o = make(s)
    P = s.params()
    dI = np.random.default_rng(2).normal(size=o.render(job, P).shape)
    tape = o.gradient(job, P, dI, mode="tape")["tex"]
    g, routes = o.gradient_hybrid(job, P, dI, 4, 0.5, 1e-6)
    assert routes["scalar"] > 0
    assert np.linalg.norm(g["tex"] - tape) < 1e-12 * np.linalg.norm(tape)


def check_flat_normal_map(make):
    """A flat tangent-space normal map (texel (0.5, 0.5, 1), n = 2c - 1 = (0, 0, 1)) shades
    with the geometric normal: every path the map leaves unchanged carries the same value."""
    sf, job = sg.normal_map_scene(flat=True)
    s0, _ = sg.normal_map_scene(flat=True)
    for m in s0.materials:
        m.normal_tex = -1
    _, pf, sig_f = make(sf).render(job, sf.params(), paths=True)
    _, p0, sig_0 = make(s0).render(job, s0.params(), paths=True)
    same = sig_f == sig_0
    assert same.mean() >= 0.99
    assert np.abs(pf[same] - p0[same]).max() <= 1e-12 * max(1.0, np.abs(p0).max())


def check_pprb_furnace(make, sigma=1e-3):
    """Basic polarized PRB behind ideal depolarizers (Sec. 4.1, case 2): the diffuse furnace's
    albedo derivative is recovered with an error of the noise's order, below sigma / 2."""
    s, job = sg.furnace_scene(0.5, 1.0)
    job.max_depth = 4
    o = make(s)
    P = s.params()
    dI = np.random.default_rng(1).normal(size=o.render(job, P).shape)
    tape = o.gradient(job, P, dI, mode="tape")["tex"]
    g = o.gradient(job, P, dI, mode="pprb", sigma=sigma)["tex"]
    assert np.linalg.norm(g - tape) < 0.5 * sigma * np.linalg.norm(tape)


def check_camera(make, W=24, H=16, vfov=40.0, dist=5.0):
    """The pinhole camera: pixel (0, 0) is the top-left; the vertical field of view is vfov; a
    world point at (x, y) in the plane dist in front of a camera looking down -z with up +y
    lands at pixel column W/2 (1 + x / (dist t a)) and row H/2 (1 - y / (dist t)),
    t = tan(vfov / 2), a = W / H.  Emitting squares half a pixel wide, centred on chosen pixel
    centres, must light exactly those pixels."""
    s = sg.Scene()
    t, a = math.tan(math.radians(vfov) / 2), W / H
    side = 0.5 * 2 * t / H * dist                   # half a pixel, in world units
    targets = [(3, 2), (20, 13), (12, 4), (1, 12)]
    for px, py in targets:
        x = ((px + 0.5) / W * 2 - 1) * dist * t * a
        y = (1 - (py + 0.5) / H * 2) * dist * t
        s.add_light((x - side / 2, y - side / 2, 0.0), (side, 0, 0), (0, side, 0), 1.0)
    s.add_camera((0, 0, dist), (0, 0, 0), (0, 1, 0), vfov)
    job = sg.Job(camera=0, width=W, height=H, spp=64, max_depth=1)
    img = make(s).render(job, s.params())[0, :, 0, 0].reshape(H, W)
    lit = {(int(c), int(r)) for r, c in zip(*np.nonzero(img > 0))}
    assert lit == set(targets), sorted(lit)


def check_intersections(make):
    """Closest hits against analytic distances: the triangle (0,0,0), (1,0,0), (0,1,0) in
    z = 0 and a sphere of radius 0.5 at (3, 0, 0); rays just inside and outside the triangle
    (both faces), the sphere's near root from outside, its exit from inside, a chord at
    height 0.4 (t = 2 - sqrt(0.25 - 0.16)), a miss, and an oblique ray whose hit is the smaller
    root of |o + t d - c|^2 = r^2.  The tree and the brute-force loop must both give them."""
    s = sg.Scene()
    m = s.add_material(sg.Material(sg.MAT_DIFFUSE))
    s.add_mesh(np.array([[0, 0, 0], [1, 0, 0], [0, 1, 0]], float), np.array([[0, 1, 2]]), m, np.zeros((3, 2)))
    s.add_sphere((3, 0, 0), 0.5, m)
    s.add_light((10, 10, 10), (1, 0, 0), (0, 1, 0), 1.0)
    s.add_camera((0, 0, 5), (0, 0, 0), (0, 1, 0), 40.0)
    sph = len(s.tris)                              # spheres are numbered after the triangles
    d_ob = np.array([0.3, 0.1, -1.0]) / math.sqrt(1.1)
    o_ob = np.array([2.8, -0.1, 2.0])
    lc = o_ob - np.array([3.0, 0.0, 0.0])
    b = float(lc @ d_ob)
    t_ob = -b - math.sqrt(b * b - (float(lc @ lc) - 0.25))
    d_tri = np.array([0.1, 0.0, -1.0]) / math.sqrt(1.01)
    rays = [((0.2, 0.2, 1), (0, 0, -1), 0, 1.0), ((0.2, 0.2, -1), (0, 0, 1), 0, 1.0),
            ((0.25, 0.25, 1), d_tri, 0, math.sqrt(1.01)),
            ((0.6, 0.6, 1), (0, 0, -1), -1, None), ((-0.2, 0.3, 1), (0, 0, -1), -1, None),
            ((3, 0, 2), (0, 0, -1), sph, 1.5), ((3, 0, 0), (1, 0, 0), sph, 0.5),
            ((3, 0.4, 2), (0, 0, -1), sph, 2.0 - math.sqrt(0.25 - 0.16)), ((3, 0.6, 2), (0, 0, -1), -1, None),
            (o_ob, d_ob, sph, t_ob)]
    o = make(s)
    for org, d, prim, t_hit in rays:
        for brute in (False, True):
            p, th = o.closest(org, d, brute=brute)
            assert p == prim, (org, d, brute, p)
            if prim >= 0:
                assert th == pytest.approx(t_hit, rel=1e-12), (org, d, brute, th, t_hit)


def check_texture(make):
    """Bilinear filtering of texels [h][w][ch] with texel centres at ((i + 1/2) / w,
    (j + 1/2) / h) and wrap-around addressing: a texel centre returns that texel, a midpoint
    between two centres their mean, the centre of four texels their mean, and the seam at
    u = 0 (or v = 0) mixes the last and first columns (rows); u + 1 reads what u reads."""
    w, h, ch = 5, 4, 2
    tex = np.random.default_rng(9).uniform(0.1, 0.9, (h, w, ch))
    look = lambda c, u, v: make.mod.tex_lookup(tex, c, u, v, library=make.library)
    for c in range(ch):
        for j in range(h):
            for i in range(w):
                assert look(c, (i + 0.5) / w, (j + 0.5) / h) == pytest.approx(tex[j, i, c], abs=1e-15)
                i1, j1 = (i + 1) % w, (j + 1) % h
                assert look(c, (i + 1.0) / w, (j + 0.5) / h) == pytest.approx((tex[j, i, c] + tex[j, i1, c]) / 2,
                                                                              abs=1e-15)
                assert look(c, (i + 0.5) / w, (j + 1.0) / h) == pytest.approx((tex[j, i, c] + tex[j1, i, c]) / 2,
                                                                              abs=1e-15)
                quad = (tex[j, i, c] + tex[j, i1, c] + tex[j1, i, c] + tex[j1, i1, c]) / 4
                assert look(c, (i + 1.0) / w, (j + 1.0) / h) == pytest.approx(quad, abs=1e-15)
        assert look(c, 0.0, 0.5 / h) == pytest.approx((tex[0, 0, c] + tex[0, w - 1, c]) / 2, abs=1e-15)
        assert look(c, 0.5 / w, 0.0) == pytest.approx((tex[0, 0, c] + tex[h - 1, 0, c]) / 2, abs=1e-15)
        assert look(c, 1.37, 0.61) == pytest.approx(look(c, 0.37, 0.61), abs=1e-14)
        assert look(c, -0.21, 0.3) == pytest.approx(look(c, 0.79, 0.3), abs=1e-14)


def check_depolarization_index(make):
    """The depolarization index of Gil and Bernabeu, sqrt(sum m_ij^2 - m00^2) / (sqrt(3) m00),
    which the hybrid replay (Sec. 4.4) compares with gamma: 1 for every non-depolarizing
    operator (identity, a frame rotation, an ideal polarizer, a Fresnel reflection), 0 for the
    ideal depolarizer that keeps only M00 (Sec. 4.1), a for the partial depolarizer
    diag(1, a, a, a), and independent of the operator's scale."""
    di = lambda m: make.mod.depol_index(np.asarray(m, float), library=make.library)
    c, s = math.cos(0.8), math.sin(0.8)
    rot = [[1, 0, 0, 0], [0, c, s, 0], [0, -s, c, 0], [0, 0, 0, 1]]
    A, B, C, S = make.mod.fresnel_reflect(0.6, 1.0, complex(0.2, 3.0))
    fres = [[A, B, 0, 0], [B, A, 0, 0], [0, 0, C, S], [0, 0, -S, C]]
    pol = make.mod.camera_filter(sg.FILTER_POLARIZER, 0.4)
    for m in (np.eye(4), rot, fres, pol, 3.5 * np.asarray(pol)):
        assert di(m) == pytest.approx(1.0, abs=1e-12)
    assert di(np.diag([0.7, 0, 0, 0])) == 0.0
    for a in (0.1, 0.5, 0.9):
        assert di(np.diag([2.0, 2 * a, 2 * a, 2 * a])) == pytest.approx(a, abs=1e-14)


# ---------------------------------------------------------------- planted mistakes
# (name, text in oracle.cpp, replacement, which occurrence, the check that must catch it)
_NEE = lambda m: check_nee_mis(m)
MUTANTS = [
    ("emit_pdf_drops_light_count", "double pl = dist2 / (cl * L.area * nL);", "double pl = dist2 / (cl * L.area);", 0, _NEE),
    ("nee_pdf_drops_light_count", "double pl = dist2 / (cl * L.area * nL);", "double pl = dist2 / (cl * L.area);", 1, _NEE),
    ("nee_pdf_cosine_at_receiver", "double pl = dist2 / (cl * L.area * nL);", "double pl = dist2 / (cx * L.area * nL);", 1, _NEE),
    ("nee_mis_weight_swapped", "double wmis = pl * pl / (pl * pl + pb * pb);", "double wmis = pb * pb / (pl * pl + pb * pb);", 0, _NEE),
    ("emit_mis_weight_swapped", "vt.w_emit = prev_pdf * prev_pdf / (prev_pdf * prev_pdf + pl * pl);",
     "vt.w_emit = pl * pl / (prev_pdf * prev_pdf + pl * pl);", 0, _NEE),
    ("nee_cosine_dropped", "vt.nee_w = cx / pl * wmis;", "vt.nee_w = 1.0 / pl * wmis;", 0, _NEE),
    ("transmit_radiance_inverted", "T sc = (eo / et) * (eo / et);", "T sc = (et / eo) * (et / eo);", 0,
     lambda m: check_transmission(m, False)),
    ("transmit_radiance_dropped", "T sc = (eo / et) * (eo / et);", "T sc = T(1.0);", 0,
     lambda m: check_transmission(m, True)),
    ("transmit_split_sign", "fac * (ts * ts - tp * tp) * 0.5", "fac * (tp * tp - ts * ts) * 0.5", 0,
     lambda m: check_transmission(m, False)),
    ("transmit_cosine_ratio_inverted", "T fac = (eta_t * cos_t) / (eta_i * cos_i);",
     "T fac = (eta_i * cos_i) / (eta_t * cos_t);", 0, lambda m: check_transmission(m, False)),
    ("fresnel_phase_conjugated", "Cx<T> rsp = cmul(rs, Cx<T>{rp.re, -rp.im});",
     "Cx<T> rsp = cmul(Cx<T>{rs.re, -rs.im}, rp);", 0, lambda m: check_rough_limit(m, "conductor", 50.0)),
    ("ggx_rin_inverted", "M4<double> Rin = rot_fixed(-wi, onb_t1(-wi), sax);",
     "M4<double> Rin = rot_fixed(-wi, sax, onb_t1(-wi));", 0, lambda m: check_rough_limit(m, "conductor", 50.0)),
    ("ggx_rin_reversed_propagation", "M4<double> Rin = rot_fixed(-wi, onb_t1(-wi), sax);",
     "M4<double> Rin = rot_fixed(wi, onb_t1(wi), sax);", 0, lambda m: check_rough_limit(m, "conductor", 50.0)),
    ("ggx_rout_inverted", "M4<double> Rout = rot_fixed(vt.wo, sax, onb_t1(vt.wo));",
     "M4<double> Rout = rot_fixed(vt.wo, onb_t1(vt.wo), sax);", 0,
     lambda m: check_rough_limit(m, "plastic", math.degrees(math.atan(1.5)))),
    ("smooth_rin_inverted", "M4<double> Rin = rot_fixed(-wi, onb_t1(-wi), sax);",
     "M4<double> Rin = rot_fixed(-wi, sax, onb_t1(-wi));", 1, lambda m: check_smooth_reflection(m)),
    ("smooth_rout_inverted", "M4<double> Rout = rot_fixed(vt.wo, sax, onb_t1(vt.wo));",
     "M4<double> Rout = rot_fixed(vt.wo, onb_t1(vt.wo), sax);", 1, lambda m: check_smooth_reflection(m)),
    ("emitter_frame_reversed_for_hits", "M4<double> R = emitter_rot(L, vt.wo);", "M4<double> R = emitter_rot(L, -vt.wo);",
     0, lambda m: check_smooth_reflection(m)),
    ("emitter_frame_reversed_for_nee", "M4<double> R = emitter_rot(L, -vt.wl);", "M4<double> R = emitter_rot(L, vt.wl);",
     0, lambda m: check_rough_limit(m, "conductor", 50.0, light_size=0.4, s0_tol=None)),
    # building blocks: the counter-based generator, Fresnel, GGX, the elements, the depolarizer
    ("philox_round_reads_wrong_word", "unsigned __int128 p1 = (unsigned __int128)M1 * c2;",
     "unsigned __int128 p1 = (unsigned __int128)M1 * c1;", 0, check_philox),
    ("philox_key_bumped_before_first_round", "if (r > 0) { k0 += W0; k1 += W1; }", "{ k0 += W0; k1 += W1; }", 0,
     check_philox),
    ("uniform_from_wrong_half", "r.u[2 * k] = (double)(lo >> 8) * (1.0 / 16777216.0);",
     "r.u[2 * k] = (double)(hi >> 8) * (1.0 / 16777216.0);", 0, check_uniforms),
    ("fresnel_rs_cosines_swapped", "Cx<T> a = cmul(ei, ci), b = cmul(eta_t, cos_t);",
     "Cx<T> a = cmul(ei, cos_t), b = cmul(eta_t, ci);", 0, check_brewster),
    ("fresnel_rp_negated", "Cx<T> rp = cdiv(csub(c, d), cadd(c, d));", "Cx<T> rp = cdiv(csub(d, c), cadd(c, d));", 0,
     check_smooth_reflection),
    ("ggx_D_drops_pi", "return a2 / (k * k * M_PI);", "return a2 / (k * k);", 0, check_ggx_area),
    ("ggx_D_alpha_unsquared", "T a2 = alpha * alpha;", "T a2 = alpha;", 0, check_ggx_masking),
    ("ggx_G1_alpha_unsquared", "sqrt(alpha * alpha * t2 + 1.0)", "sqrt(alpha * t2 + 1.0)", 0, check_ggx_masking),
    ("polarizer_axis_along_y", "r.m[0][1] = T(0.5); r.m[1][0] = T(0.5);", "r.m[0][1] = T(-0.5); r.m[1][0] = T(-0.5);",
     0, check_polarizer),
    ("element_rotated_backwards", "return mmul(mmul(rot_cs<T>(c, -s), m), rot_cs<T>(c, s));",
     "return mmul(mmul(rot_cs<T>(c, s), m), rot_cs<T>(c, -s));", 0, check_malus),
    ("diffuse_drops_one_over_pi", "f[c].m[0][0] = alb[c] * (1.0 / M_PI);", "f[c].m[0][0] = alb[c];", 0, check_furnace),
    # the cached suffix replay's algebra
    ("replay_reads_own_suffix", "S4<Var> wl = mvec(e.W[c], Lc[v + 1][c]);", "S4<Var> wl = mvec(e.W[c], Lc[v][c]);", 0,
     check_tape_equals_replay),
    ("replay_adjoint_row_transposed", "sacc += arow[c][k] * ev[v].W[c].m[k][j];",
     "sacc += arow[c][k] * ev[v].W[c].m[j][k];", 0, check_tape_equals_replay),
    ("replay_fold_drops_emission", "for (int k = 0; k < 4; ++k) Lc[v][c].s[k] = ev[v].E[c].s[k] + wl.s[k];",
     "for (int k = 0; k < 4; ++k) Lc[v][c].s[k] = wl.s[k];", 0, check_tape_equals_replay),
    # the hybrid cached replay's recovery of the suffixes between checkpoints
    ("hybrid_block_emission_after_throughput", "S4<double> be = mvec(bt[c], ev.E[c]);",
     "S4<double> be = mvec(mmul(bt[c], ev.W[c]), ev.E[c]);", 0, lambda m: check_hybrid_exact(m, 4, 0.0, 0.0)),
    ("hybrid_block_throughput_reversed", "bt[c] = mmul(bt[c], ev.W[c]);", "bt[c] = mmul(ev.W[c], bt[c]);", 0,
     lambda m: check_hybrid_exact(m, 4, 0.0, 0.0)),
    ("hybrid_recompute_skips_a_vertex", "for (int j = v + 1; j < std::min(next, n); ++j) {",
     "for (int j = v + 2; j < std::min(next, n); ++j) {", 0, lambda m: check_hybrid_exact(m, 4, 0.0, float("inf"))),
    ("hybrid_scalar_route_undivided", "Ln[c].s[0] = r.s[0] / bt[c].m[0][0];", "Ln[c].s[0] = r.s[0];", 0,
     check_hybrid_scalar_furnace),
    # the normal map's decoding and basic polarized PRB's inversion
    ("normal_map_x_not_decoded", "T a = tex_lookup<T>(s, P, m.normal_tex, 0, vt.tu, vt.tv) * 2.0 - 1.0;",
     "T a = tex_lookup<T>(s, P, m.normal_tex, 0, vt.tu, vt.tv);", 0, check_flat_normal_map),
    ("pprb_emission_not_removed", "m[k][4] = L[c][k] - (T)ev[v].E[c].s[k];", "m[k][4] = L[c][k];", 0,
     check_pprb_furnace),
    # sampling: the GGX half-vector pdf without the Jacobian 1 / (4 cos theta_oh) biases the lobe
    ("ggx_pdf_drops_half_vector_jacobian", "return ggx_D<double>(ch, alpha) * ch / (4.0 * oh);",
     "return ggx_D<double>(ch, alpha) * ch;", 0, lambda m: check_rough_limit(m, "conductor", 50.0)),
    # the pinhole camera
    ("camera_rows_flipped", "double sy = (1.0 - 2.0 * (py + jv) / H) * c.tanh;",
     "double sy = (2.0 * (py + jv) / H - 1.0) * c.tanh;", 0, check_camera),
    ("camera_right_reversed", "cm.right = normalize(cross(cm.fwd, ld3(c + 6)));",
     "cm.right = normalize(cross(ld3(c + 6), cm.fwd));", 0, check_camera),
    ("camera_aspect_dropped", "double sx = (2.0 * (px + ju) / W - 1.0) * c.tanh * aspect;",
     "double sx = (2.0 * (px + ju) / W - 1.0) * c.tanh;", 0, check_camera),
    ("camera_full_field_angle", "cm.tanh = std::tan(0.5 * c[9] * M_PI / 180.0);",
     "cm.tanh = std::tan(c[9] * M_PI / 180.0);", 0, check_camera),
    # ray intersection
    ("triangle_u_lower_bound_dropped", "if (u < 0.0 || u > 1.0) return -1.0;", "if (u > 1.0) return -1.0;", 0,
     check_intersections),
    ("triangle_tests_w_not_u_plus_w", "if (w < 0.0 || u + w > 1.0) return -1.0;", "if (w < 0.0 || w > 1.0) return -1.0;",
     0, check_intersections),
    ("sphere_radius_unsquared", "double disc = rad * rad - dot(f, f);", "double disc = rad - dot(f, f);", 0,
     check_intersections),
    ("sphere_far_root_first", "if (t0 > 0.0 && t0 < tmax) return t0;", "if (t1 > 0.0 && t1 < tmax) return t1;", 0,
     check_intersections),
    # texture filtering
    ("texture_half_texel_offset_dropped", "double x = u * (double)t.w - 0.5, y = v * (double)t.h - 0.5;",
     "double x = u * (double)t.w, y = v * (double)t.h - 0.5;", 0, check_texture),
    ("texture_tap_column_swapped", "tp.idx[1] = t.off + (ya * t.w + xb) * t.ch;",
     "tp.idx[1] = t.off + (ya * t.w + xa) * t.ch;", 0, check_texture),
    ("texture_clamped_not_wrapped", "auto wrap = [](int64_t a, int64_t n) { int64_t m = a % n; return m < 0 ? m + n : m; };",
     "auto wrap = [](int64_t a, int64_t n) { int64_t m = a % n; return m < 0 ? 0 : m; };", 0, check_texture),
    ("texture_tap_index_transposed", "tp.idx[0] = t.off + (ya * t.w + xa) * t.ch;",
     "tp.idx[0] = t.off + (xa * t.h + ya) * t.ch;", 0, check_texture),
    # the hybrid's depolarization index
    ("depol_index_three_for_root_three",
     "return std::sqrt(std::max(0.0, s2 - m.m[0][0] * m.m[0][0])) / (std::sqrt(3.0) * m.m[0][0]);",
     "return std::sqrt(std::max(0.0, s2 - m.m[0][0] * m.m[0][0])) / (3.0 * m.m[0][0]);", 0,
     check_depolarization_index),
    ("depol_index_keeps_m00",
     "return std::sqrt(std::max(0.0, s2 - m.m[0][0] * m.m[0][0])) / (std::sqrt(3.0) * m.m[0][0]);",
     "return std::sqrt(std::max(0.0, s2)) / (std::sqrt(3.0) * m.m[0][0]);", 0, check_depolarization_index),
]


def _replace_nth(text: str, old: str, new: str, k: int) -> str:
    pos = -1
    for _ in range(k + 1):
        pos = text.index(old, pos + 1)
    return text[:pos] + new + text[pos + len(old):]


@pytest.fixture(scope="module")
def mutant_libs(tmp_path_factory, oracle_mod):
    src = open(ORACLE_CPP).read()
    out = tmp_path_factory.mktemp("oracle_mutants")
    jobs = {}
    for name, old, new, k, _ in MUTANTS:
        assert src.count(old) > k, f"{name}: the oracle no longer contains {old!r}"
        cpp = out / f"{name}.cpp"
        cpp.write_text(_replace_nth(src, old, new, k))
        jobs[name] = (cpp, out / f"{name}.so")

    def compile_one(item):
        cpp, so = item
        subprocess.check_call(["g++", "-std=c++17", "-O1", "-shared", "-fPIC", "-o", str(so), str(cpp)])
        return str(so)

    with concurrent.futures.ThreadPoolExecutor(max_workers=os.cpu_count() or 4) as ex:
        built = dict(zip(jobs, ex.map(compile_one, jobs.values())))
    return {name: oracle_mod.load(path) for name, path in built.items()}


@pytest.mark.parametrize("name", [m[0] for m in MUTANTS])
def test_planted_mistake_is_caught(oracle_mod, mutant_libs, name):
    check = {m[0]: m[4] for m in MUTANTS}[name]
    check(_real(oracle_mod))                      # the unmodified oracle passes the check
    library = mutant_libs[name]
    with pytest.raises(AssertionError):
        check(Oracle(oracle_mod, library))


def test_pinhole_camera(oracle_mod):
    check_camera(_real(oracle_mod))


def test_ray_intersections(oracle_mod):
    check_intersections(_real(oracle_mod))


def test_texture_filtering(oracle_mod):
    check_texture(_real(oracle_mod))


def test_depolarization_index(oracle_mod):
    check_depolarization_index(_real(oracle_mod))
