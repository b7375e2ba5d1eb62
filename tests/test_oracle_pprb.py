"""The case analysis of Sec. 4.1 on the oracle's three derivative routes.

Basic polarized PRB (P-PRB) recovers each suffix by inverting the sampled transport factor,
regularized with noise u*I (u ~ N(0, sigma), the same u in the primal and the adjoint,
Sec. 4.2).  Sec. 4.1 predicts that this works for invertible elements (retarders) and for
ideal depolarizers (diffuse), and fails for non-invertible polarization-aware elements
(linear polarizers), for every choice of sigma.  Cached suffix replay needs no inversion and
stays exact everywhere.  The tape (conventional reverse AD) is the reference; the relative
error is the L2 norm of the difference over the L2 norm of the reference.

The sigma sweep covers 1e-1 .. 1e-7.  With the noise in both phases the P-PRB gradient is
that of a noised estimator (error ~ sigma); small sigma makes the inversions of a chain of
rank-deficient factors ill-conditioned (error ~ eps / sigma^k).  Single precision (the
precision of a GPU renderer) leaves no sigma at which both are small."""
import numpy as np
import pytest

from paper_2607_13265_gb300 import scenegen as sg

SIGMAS = (1e-1, 1e-2, 1e-3, 1e-4, 1e-5, 1e-6, 1e-7)


def _rel(g, o):
    return float(np.linalg.norm(g - o) / np.linalg.norm(o))


def _setup(oracle_mod, scene, job, seed=1):
    o = oracle_mod.OracleScene(scene)
    P = scene.params()
    img = o.render(job, P)
    dI = np.random.default_rng(seed).normal(size=img.shape)
    return o, P, dI


def test_polarizer_stack_breaks_pprb_for_every_sigma(oracle_mod):
    """Five linear polarizers: the sheet-angle gradients need the polarization state behind
    each sheet, which a rank-deficient factor does not carry."""
    s, job = sg.polarizer_stack_scene([0.0, 0.4, 0.9, 1.3, 1.9])
    o, P, dI = _setup(oracle_mod, s, job)
    tape = o.gradient(job, P, dI, mode="tape")["sheet"]
    assert np.all(np.abs(tape) > 1e-3)
    assert _rel(o.gradient(job, P, dI, mode="replay")["sheet"], tape) < 1e-12
    single = [_rel(o.gradient(job, P, dI, mode="pprb", sigma=sg_, single=True)["sheet"], tape) for sg_ in SIGMAS]
    assert min(single) > 0.05, single
    double = [_rel(o.gradient(job, P, dI, mode="pprb", sigma=sg_)["sheet"], tape) for sg_ in SIGMAS]
    assert min(double) > 1e-3, double
    assert double[-1] > 1.0, double          # ill-conditioned at small sigma even in FP64


def test_pprb_without_primal_noise_loses_the_null_space(oracle_mod):
    """Regularizing only the inversion (a plain primal) recovers the suffix's projection onto
    the polarizer's range: the error grows like 1/sigma."""
    s, job = sg.polarizer_stack_scene([0.0, 0.5, 1.1])
    o, P, dI = _setup(oracle_mod, s, job)
    tape = o.gradient(job, P, dI, mode="tape")["sheet"]
    errs = [_rel(o.gradient(job, P, dI, mode="pprb", sigma=x, primal_noise=False)["sheet"], tape)
            for x in (1e-1, 1e-3)]
    assert errs[0] > 1.0 and errs[1] > 50 * errs[0], errs


def test_camera_filter_angle_survives_pprb(oracle_mod):
    """The camera filter acts on the path's total, which P-PRB has exactly: its angle's
    gradient needs no recovered suffix."""
    s, job = sg.polarizer_stack_scene([0.0, 0.5, 1.1])
    job.thetas = [0.3]
    o, P, dI = _setup(oracle_mod, s, job)
    P["theta"] = np.array([0.3])
    tape = o.gradient(job, P, dI, mode="tape")["theta"]
    g = o.gradient(job, P, dI, mode="pprb", sigma=1e-7, primal_noise=False)["theta"]
    assert abs(tape[0]) > 1e-3
    assert _rel(g, tape) < 1e-12


@pytest.mark.parametrize("single", [False, True])
def test_retarders_are_invertible_so_pprb_converges(oracle_mod, single):
    """Case 1 of Sec. 4.1: with invertible factors the P-PRB error is the noise's, O(sigma)."""
    s, job = sg.retarder_pair_scene()
    o, P, dI = _setup(oracle_mod, s, job)
    tape = o.gradient(job, P, dI, mode="tape")["sheet"]
    assert _rel(o.gradient(job, P, dI, mode="replay")["sheet"], tape) < 1e-12
    errs = [_rel(o.gradient(job, P, dI, mode="pprb", sigma=x, single=single)["sheet"], tape) for x in SIGMAS]
    for x, e in zip(SIGMAS, errs):
        assert e < 0.5 * x + (1e-6 if single else 1e-12), (x, e)


@pytest.mark.parametrize("single", [False, True])
def test_depolarizer_albedo_gradient_converges_under_pprb(oracle_mod, single):
    """Case 2 of Sec. 4.1: in a diffuse furnace the albedo derivative needs only s0 of the
    suffix, which the regularized inversion recovers; the error is O(sigma)."""
    s, job = sg.furnace_scene(0.5, 1.0)
    job.max_depth = 4
    o, P, dI = _setup(oracle_mod, s, job)
    tape = o.gradient(job, P, dI, mode="tape")["tex"]
    assert _rel(o.gradient(job, P, dI, mode="replay")["tex"], tape) < 1e-12
    errs = [_rel(o.gradient(job, P, dI, mode="pprb", sigma=x, single=single)["tex"], tape) for x in SIGMAS]
    for x, e in zip(SIGMAS, errs):
        assert e < 0.5 * x + (1e-6 if single else 1e-12), (x, e)
