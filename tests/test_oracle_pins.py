"""Pins for the FP64 oracle against facts fixed by optics and mathematics, not by the oracle.

Each test names the fact it checks.  Together they are chosen so that a dropped term, a
wrong sign or index, or a transposed operand in the oracle fails at least one of them:
Malus's law and its derivative (polarizer, frame rotations, camera filter), the GGX
normalization and Smith masking identities (pBRDF lobes), the quarter-wave
conversion to circular light (retarder block), Brewster's angle (Fresnel s/p split and the
s/p frame), energy conservation and textbook closed forms of the Fresnel coefficients,
exact depolarization after a diffuse bounce (Sec. 4.1 case 2), the white furnace (sampling
weights and the depth convention), Euler homogeneity in the emitter Stokes vector,
agreement of the two derivative routes (taped AD vs cached suffix replay, Sec. 4.3), and
central finite differences of the frozen-sampling estimator.
"""
import math

import numpy as np
import pytest

from paper_2607_13265_gb300 import scenegen as sg


# ---------------------------------------------------------------- counter-based RNG
def test_philox_matches_numpy(oracle_mod):
    """Philox4x64-10 blocks equal numpy.random.Philox (which pre-increments its counter)."""
    rng = np.random.default_rng(123)
    for _ in range(20):
        key = rng.integers(0, 2**63, 2, dtype=np.uint64)
        ctr = rng.integers(0, 2**63, 4, dtype=np.uint64)
        ref = np.random.Philox(key=key, counter=ctr).random_raw(4)
        nxt = ctr.copy()
        nxt[0] += np.uint64(1)
        assert np.array_equal(oracle_mod.philox4x64(nxt, key), ref)


def test_uniform_layout(oracle_mod):
    """u_k = (word_k >> 8) * 2^-24 with word 2i/2i+1 = low/high half of output i;
    key = (seed ^ pass*0x9E3779B97F4A7C15, stream), counter = (path, vertex, 0, 0)."""
    seed, pas, stream, path, vertex = 77, 1, 3, 123456789, 5
    k0 = np.uint64(seed) ^ np.uint64((pas * 0x9E3779B97F4A7C15) % 2**64)
    ref = np.random.Philox(key=[k0, np.uint64(stream)], counter=[path - 1, vertex, 0, 0]).random_raw(4)
    words = []
    for x in ref:
        words += [int(x) & 0xFFFFFFFF, int(x) >> 32]
    expect = np.array([(w >> 8) / 2**24 for w in words])
    assert np.array_equal(oracle_mod.uniforms(seed, pas, stream, path, vertex), expect)


def test_csqrt_principal_branch(oracle_mod):
    for z in [complex(-4, 0), complex(-4, 1e-30), complex(3, 4), complex(-3, -4), complex(0.2, 3.0),
              complex(1e-9, -2), complex(0, 0)]:
        assert abs(oracle_mod.csqrt(z) - np.sqrt(z)) <= 1e-15 * max(1, abs(z))
    assert oracle_mod.csqrt(complex(-4.0, 0.0)) == complex(0.0, 2.0)


# ---------------------------------------------------------------- Fresnel
def test_fresnel_normal_incidence_and_energy(oracle_mod):
    for n in [1.33, 1.5, 2.4]:
        R0 = ((n - 1) / (n + 1)) ** 2
        A, B, C, S = oracle_mod.fresnel_reflect(1.0, 1.0, n)
        assert A == pytest.approx(R0, rel=1e-13) and abs(B) < 1e-15
        assert C == pytest.approx(-R0, rel=1e-13) and S == 0.0   # r_p = -r_s at normal incidence
        for ci in np.linspace(0.05, 1.0, 12):
            R = oracle_mod.fresnel_reflect(ci, 1.0, n)
            sin_t = math.sqrt(1 - ci * ci) / n
            T = oracle_mod.fresnel_transmit(ci, 1.0, n)
            # energy: (Rs+Rp)/2 + (Ts+Tp)/2 = 1 and the s/p split is conserved: B_R + B_T = 0
            assert R[0] + T[0] == pytest.approx(1.0, abs=1e-14)
            assert R[1] + T[1] == pytest.approx(0.0, abs=1e-14)
            # Stokes reciprocity: reflectance from inside at the refracted angle is the same
            ct = math.sqrt(1 - sin_t**2)
            assert oracle_mod.fresnel_reflect(ct, n, 1.0)[0] == pytest.approx(R[0], rel=1e-12)
            # a non-depolarizing Mueller matrix: A^2 = B^2 + C^2 + S^2
            assert R[0] ** 2 == pytest.approx(R[1] ** 2 + R[2] ** 2 + R[3] ** 2, rel=1e-12)


def test_fresnel_brewster(oracle_mod):
    n = 1.5
    tb = math.atan(n)
    A, B, C, S = oracle_mod.fresnel_reflect(math.cos(tb), 1.0, n)
    # at Brewster's angle r_p = 0 and r_s = (1 - n^2) / (1 + n^2)
    rs = (1 - n * n) / (1 + n * n)
    assert A == pytest.approx(rs * rs / 2, rel=1e-12)
    assert B == pytest.approx(rs * rs / 2, rel=1e-12)
    assert abs(C) < 1e-15 and abs(S) < 1e-15
    assert rs * rs == pytest.approx(0.1479, abs=1e-4)


def test_fresnel_total_internal_reflection_is_a_retarder(oracle_mod):
    n = 1.5
    crit = math.sqrt(1 - 1 / n**2)
    for ci in [0.05, 0.3, 0.6, crit * 0.999]:
        A, B, C, S = oracle_mod.fresnel_reflect(ci, n, 1.0)
        assert A == pytest.approx(1.0, abs=1e-14) and abs(B) < 1e-14
        assert C * C + S * S == pytest.approx(1.0, abs=1e-13)
        # phase difference of s and p (Born & Wolf): tan(d/2) = cos_i sqrt(sin^2 - 1/n^2) / sin^2
        s2 = 1 - ci * ci
        d = 2 * math.atan(ci * math.sqrt(s2 - 1 / n**2) / s2)
        assert abs(math.cos(d)) == pytest.approx(abs(C), abs=1e-12)


@pytest.mark.parametrize("alpha", [0.05, 0.2, 0.5, 1.0])
def test_ggx_projected_area_and_masking_identities(oracle_mod, alpha):
    """Two identities of the GGX microfacet model (Walter et al. 2007; Heitz 2014, "Understanding
    the masking-shadowing function"), fixed by geometry rather than by the oracle:
    the microfacet normals cover the macro-surface exactly once,
        int D(h) cos(theta_h) dw_h = 2 pi int_0^1 D(mu) mu dmu = 1,
    and the Smith masking G1 normalizes the visible projected area for every direction o,
        G1(o) int max(0, o.h) D(h) dw_h = cos(theta_o).
    A missing 1/pi, a squared or unsquared alpha, or a wrong exponent in D or G1 breaks one."""
    integrate = pytest.importorskip("scipy.integrate")
    D = lambda mu: oracle_mod.ggx(mu, 1.0, 1.0, alpha)[0]
    # D peaks within ~alpha of mu = 1: split the range there for the quadrature
    knots = [0.0, max(0.0, 1.0 - 4.0 * alpha * alpha), 1.0]
    area = sum(integrate.quad(lambda m: D(m) * m, a, b, epsabs=1e-13, epsrel=1e-11, limit=400)[0]
               for a, b in zip(knots[:-1], knots[1:]) if b > a)
    assert 2.0 * math.pi * area == pytest.approx(1.0, rel=1e-8)
    for theta_o in (0.0, 0.5, 1.0, 1.3):
        o = np.array([math.sin(theta_o), 0.0, math.cos(theta_o)])

        def visible(phi, mu):
            s = math.sqrt(max(0.0, 1.0 - mu * mu))
            return max(0.0, o[0] * s * math.cos(phi) + o[2] * mu) * D(mu)

        # the phi integrand is even: integrate over [0, pi] and double
        inner = lambda mu: integrate.quad(lambda ph: visible(ph, mu), 0.0, math.pi, epsabs=1e-12, limit=200)[0]
        proj = 2.0 * sum(integrate.quad(inner, a, b, epsabs=1e-10, epsrel=1e-8, limit=200)[0]
                         for a, b in zip(knots[:-1], knots[1:]) if b > a)
        g1 = oracle_mod.ggx(1.0, math.cos(theta_o), 1.0, alpha)[1]
        assert g1 * proj == pytest.approx(math.cos(theta_o), rel=1e-6), (alpha, theta_o)


def test_conductor_normal_incidence(oracle_mod):
    eta = complex(0.2, 3.0)
    A, B, C, S = oracle_mod.fresnel_reflect(1.0, 1.0, eta)
    assert A == pytest.approx(((0.2 - 1) ** 2 + 9) / ((0.2 + 1) ** 2 + 9), rel=1e-13)
    assert abs(B) < 1e-15


# ---------------------------------------------------------------- optical elements
def test_camera_filters(oracle_mod):
    for th in [0.0, 0.4, 1.3, -0.7]:
        P = oracle_mod.camera_filter(sg.FILTER_POLARIZER, th)
        assert np.allclose(P @ P, P, atol=1e-15)                      # ideal polarizer is a projector
        assert np.allclose(P @ [1, 0, 0, 0], [0.5, 0.5 * math.cos(2 * th), 0.5 * math.sin(2 * th), 0], atol=1e-15)
        assert np.allclose(P[:, 3], 0) and np.allclose(P[3, :], 0)    # loses s3 (Sec. 4.1)
        assert np.linalg.matrix_rank(P) == 1
    # quarter-wave plate turns circular light into linear at 45 deg, then P(45) passes it all
    C45 = oracle_mod.camera_filter(sg.FILTER_QWP_POLARIZER, math.pi / 4)
    Cm45 = oracle_mod.camera_filter(sg.FILTER_QWP_POLARIZER, -math.pi / 4)
    circ = np.array([1, 0, 0, 1.0])
    assert (C45 @ circ)[0] + (Cm45 @ circ)[0] == pytest.approx(1.0, abs=1e-15)
    assert max((C45 @ circ)[0], (Cm45 @ circ)[0]) == pytest.approx(1.0, abs=1e-15)


@pytest.mark.parametrize("alpha,theta", [(0.3, 1.1), (0.0, 0.0), (1.0, -0.4), (2.0, 0.5)])
def test_malus_law_and_derivative(oracle_mod, alpha, theta):
    """Unpolarized L through a sheet polarizer at alpha, then the camera polarizer at theta:
    I = (L/2) cos^2(theta - alpha); dI/dtheta = -(L/2) sin 2(theta - alpha) = -dI/dalpha."""
    L = 2.0
    s, job = sg.malus_scene(alpha, le=L)
    job.thetas = [theta]
    o = oracle_mod.OracleScene(s)
    img = o.render(job, s.params())
    expect = 0.5 * L * math.cos(theta - alpha) ** 2
    # off-axis rays see the sheet axis projected at an angle O(fov^2) ~ 1e-8 away
    assert np.allclose(img[0, :, :, 0], expect, rtol=1e-6, atol=1e-9)
    dI = np.zeros_like(img)
    dI[0, :, 0, 0] = 1.0
    dI_dth = -0.5 * L * math.sin(2 * (theta - alpha)) * job.num_pixels
    for mode in ("tape", "replay"):
        g = o.gradient(job, s.params(), dI, mode=mode)
        assert g["theta"][0] == pytest.approx(dI_dth, rel=1e-6, abs=1e-6)
        assert g["sheet"][0] == pytest.approx(-dI_dth, rel=1e-6, abs=1e-6)
        # Euler: I is homogeneous of degree 1 in the emitter Stokes vector
        le = s.params()["le"].ravel()
        assert np.dot(le, g["le"]) == pytest.approx(float(img[0, :, 0, 0].sum()), rel=1e-10)


def test_unfiltered_polarizer_sheet(oracle_mod):
    s, job = sg.malus_scene(0.6, le=2.0)
    job.filter, job.thetas = sg.FILTER_NONE, []
    img = oracle_mod.OracleScene(s).render(job, s.params())
    assert np.allclose(img[0, :, 0], [1.0, math.cos(1.2), math.sin(1.2), 0.0], atol=1e-8)


@pytest.mark.parametrize("alpha,phi", [(0.0, math.pi / 4), (0.5, 0.5 - math.pi / 4), (0.3, 0.1)])
def test_quarter_wave_sheet(oracle_mod, alpha, phi):
    """Linear light at alpha through a quarter-wave plate with fast axis phi:
    s0 is kept and |s3| = s0 |sin 2(alpha - phi)| (circular at 45 deg)."""
    s, job = sg.retarder_scene(alpha, phi, le=2.0)
    img = oracle_mod.OracleScene(s).render(job, s.params())[0, :, 0]
    assert np.allclose(img[:, 0], 1.0, atol=1e-9)
    assert np.allclose(np.abs(img[:, 3]), abs(math.sin(2 * (alpha - phi))), atol=1e-7)
    dop = np.sqrt((img[:, 1:] ** 2).sum(1)) / img[:, 0]
    assert np.allclose(dop, 1.0, atol=1e-7)


def test_brewster_reflection_is_s_polarized(oracle_mod):
    """Every reflected path at Brewster's angle is fully polarized along s (the sensor x
    axis here) with no s2/s3; the mean s0 tends to R_s/2 * L; a polarizer along p blocks it."""
    s, job = sg.brewster_scene(1.5, le=1.0)
    job.spp = 512
    o = oracle_mod.OracleScene(s)
    img, paths, _ = o.render(job, s.params(), paths=True)
    refl = paths[:, 0, 0] > 0
    assert refl.any() and (~refl).any()
    v = paths[refl, 0]
    assert np.allclose(v[:, 1] / v[:, 0], 1.0, atol=1e-6)      # s1 = s0: polarized along s
    assert np.allclose(v[:, 2:] / v[:, :1], 0.0, atol=2e-3)     # tiny fov: only off-axis frame tilt
    rs2 = ((1 - 2.25) / (1 + 2.25)) ** 2
    frac = refl.mean()
    assert abs(frac - rs2 / 2) < 4 * math.sqrt(rs2 / 2 * (1 - rs2 / 2) / refl.size)
    job.filter, job.thetas = sg.FILTER_POLARIZER, [math.pi / 2]
    blocked = o.render(job, s.params())
    assert np.abs(blocked[0, :, 0, 0]).max() < 1e-6 * img[0, :, 0, 0].max() + 1e-12


# ---------------------------------------------------------------- transport invariants
def test_diffuse_depolarizes(oracle_mod):
    """Without any polarizing element before the camera and only diffuse surfaces, every pixel
    has s1 = s2 = s3 = 0 exactly (an ideal depolarizer keeps only M00, Sec. 4.1)."""
    s, job = sg.cornell_box()
    s.spheres = s.spheres[:1]
    s.sph_mat = s.sph_mat[:1]
    job.width = job.height = 12
    job.spp, job.filter, job.thetas = 4, sg.FILTER_NONE, []
    img = oracle_mod.OracleScene(s).render(job, s.params())
    assert img[..., 0].max() > 0
    assert np.all(img[..., 1:] == 0.0)


def test_white_furnace(oracle_mod):
    """Closed diffuse emitting box: every path is exactly e * sum_{k<d} a^k and its albedo
    derivative is e * sum_{k<d} k a^(k-1), whatever the sampled directions."""
    a, e = 0.6, 1.5
    s, job = sg.furnace_scene(a, e)
    o = oracle_mod.OracleScene(s)
    for depth in (1, 2, 5):
        job.max_depth = depth
        img = o.render(job, s.params())
        assert np.allclose(img[0, :, :, 0], e * sum(a**k for k in range(depth)), rtol=1e-12)
        assert np.all(img[0, :, :, 1:] == 0)
        dI = np.zeros_like(img)
        dI[0, :, 1, 0] = 1.0
        for mode in ("tape", "replay"):
            g = o.gradient(job, s.params(), dI, mode=mode)["tex"]
            expect = e * sum(k * a ** (k - 1) for k in range(1, depth)) * job.num_pixels
            assert g[1] == pytest.approx(expect, rel=1e-12, abs=1e-12)
            assert g[0] == 0.0 and g[2] == 0.0


def test_dop_bound_and_mixed_scene(oracle_mod):
    s, job = sg.mixed_scene(width=16, spp=4)
    job.filter, job.thetas = sg.FILTER_NONE, []
    img, paths, _ = oracle_mod.OracleScene(s).render(job, s.params(), paths=True)
    for arr in (img[0], paths):
        s0 = arr[..., 0]
        pol = np.sqrt((arr[..., 1:] ** 2).sum(-1))
        assert np.all(pol <= s0 * (1 + 1e-9) + 1e-12)
    assert np.abs(paths[..., 3]).max() > 1e-3          # the scene does produce circular light


def test_bvh_matches_brute_force(oracle_mod):
    s, _ = sg.mixed_scene()
    o = oracle_mod.OracleScene(s)
    rng = np.random.default_rng(5)
    for _ in range(300):
        org = rng.uniform(-2, 2, 3)
        d = rng.normal(size=3)
        d /= np.linalg.norm(d)
        p1, t1 = o.closest(org, d)
        p2, t2 = o.closest(org, d, brute=True)
        assert p1 == p2 and (p1 < 0 or t1 == t2)


# ---------------------------------------------------------------- derivatives
@pytest.fixture(scope="module")
def mixed(oracle_mod):
    s, job = sg.mixed_scene(width=10, spp=2, depth=5)
    return s, job, oracle_mod.OracleScene(s)


def test_tape_equals_cached_replay(mixed):
    """Conventional AD over the whole path and cached suffix replay (Sec. 4.3) compute the
    same derivative; any slip in the fold, the suffix index or the adjoint row breaks this."""
    s, job, o = mixed
    img = o.render(job, s.params())
    dI = np.random.default_rng(1).normal(size=img.shape)
    g1 = o.gradient(job, s.params(), dI, mode="tape")
    g2 = o.gradient(job, s.params(), dI, mode="replay")
    for k in g1:
        if len(g1[k]) == 0:
            continue
        assert np.linalg.norm(g1[k]) > 0, k
        assert np.allclose(g1[k], g2[k], rtol=1e-11, atol=1e-12 * np.abs(g1[k]).max()), k


def test_emitter_euler_identity(mixed):
    s, job, o = mixed
    P = s.params()
    img = o.render(job, P)
    dI = np.random.default_rng(2).normal(size=img.shape)
    g = o.gradient(job, P, dI, mode="replay")
    assert np.dot(P["le"].ravel(), g["le"]) == pytest.approx(float((dI * img).sum()), rel=1e-10)


def _fd(o, job, P, dI, name, idx, h=1e-4):
    def J(delta):
        Pl = {k: np.array(v, dtype=np.float64, copy=True) for k, v in P.items()}
        Pl[name].reshape(-1)[idx] += delta
        return float((dI * o.render(job, P, params_live=Pl)).sum())
    return (J(h) - J(-h)) / (2 * h)


def test_central_differences(mixed):
    """Both derivative routes match central differences of the frozen-sampling estimator for
    every kind of parameter: camera polarizer angles, sheet angles, indices of refraction,
    albedo and roughness texels, emitter Stokes components.  h = 1e-4 keeps the O(h^2)
    truncation below the tolerance even for paths near the critical angle of the glass."""
    s, job, o = mixed
    P = dict(s.params())
    P["theta"] = np.array(job.thetas)
    img = o.render(job, P)
    dI = np.random.default_rng(3).normal(size=img.shape)
    g = o.gradient(job, P, dI, mode="replay")
    (a_off, _, _, _), (r_off, rw, rh, _) = s.tex_desc[0], s.tex_desc[1]
    ga, gr = g["tex"][a_off:r_off], g["tex"][r_off:r_off + rw * rh]
    checks = [("theta", 0), ("theta", 1), ("sheet", 0), ("sheet", 1), ("ior", 0), ("ior", 1),
              ("le", 0), ("le", 14), ("le", 15), ("le", 23),
              ("tex", int(a_off + np.argmax(np.abs(ga)))), ("tex", int(a_off + np.argsort(np.abs(ga))[-7])),
              ("tex", int(r_off + np.argmax(np.abs(gr)))), ("tex", int(r_off + np.argsort(np.abs(gr))[-5]))]
    for name, idx in checks:
        fd = _fd(o, job, P, dI, name, idx)
        an = g[name][idx]
        assert an != 0.0, (name, idx)
        assert abs(an - fd) <= 1e-6 * max(1.0, abs(fd)), (name, idx, an, fd)


def test_conventional_ad_tape_model(oracle_mod):
    """The memory model of conventional reverse AD (oracle/tape_memory.py) on a small sample of
    the deep-stack workload: the tape holds a fixed number of nodes per vertex, so it grows in
    proportion to the path's vertices, while the replay's cache holds 124 B per vertex."""
    from oracle import tape_memory
    rows = tape_memory.main(["--depths", "4", "16", "--width", "8", "--height", "5"])
    assert [r["depth"] for r in rows] == [4, 16]
    for r in rows:
        assert r["tape_nodes_per_path"] > 0 and r["vertices_per_path"] > 1
        assert r["conv_ad_bytes_16B"] == pytest.approx(4 * r["conv_ad_bytes_4B_lower_bound"])
        assert r["cache_bytes_full"] == pytest.approx(r["vertices_per_path"] * 1280 * 720 * 124)
    shallow, deep = rows
    assert deep["vertices_per_path"] > 2 * shallow["vertices_per_path"]
    assert deep["tape_nodes_per_vertex"] == pytest.approx(shallow["tape_nodes_per_vertex"], rel=0.05)
    assert deep["conv_ad_bytes_16B"] > 10 * deep["cache_bytes_full"]
