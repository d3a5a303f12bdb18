"""The oracle's Monte Carlo error bar sigma(C_D) (§III.B: the statistical
scatter of C_D), pinned by calibration over independent Philox streams.

sigma is the standard error of the mean of the per-particle drag
contributions.  If it is right, then over many independent runs
  * z = (C_D - exact) / sigma has mean 0 and variance 1 on convex bodies,
    where the panel sum is the exact expectation (plate and icosphere), and
  * the scatter of C_D between runs equals the mean of sigma^2 on a concave
    body, where no exact value exists (the hemispherical shell, two hits per
    entering particle on average).
A sigma off by sqrt(2), or taken per hit instead of per particle (which
matters only where particles hit more than once), moves the variance ratio to
about 2 or 1/2; with 256 runs the ratio's own standard error is 0.09, and the
windows below are about four of those wide.
"""
import math

import numpy as np

from tpmc_inputs import meshes as M
from tpmc_inputs import workloads as W


def _runs(orc, xyz, tri, params, N, n_runs):
    mesh = orc.Mesh(xyz, tri)
    cd, sig = np.zeros(n_runs), np.zeros(n_runs)
    for k in range(n_runs):
        r, _, _ = orc.trace(mesh, orc.make_params(**params, stream=k), N)
        cd[k], sig[k] = r["CD"], r["CD_sigma"]
    return cd, sig


def _check_z(z, n_runs):
    # mean: standard error 1/sqrt(n); variance: standard error sqrt(2/(n-1))
    assert abs(z.mean()) < 4.0 / math.sqrt(n_runs), z.mean()
    v = z.var(ddof=1)
    assert abs(v - 1.0) < 4.0 * math.sqrt(2.0 / (n_runs - 1)), v


def test_sigma_calibrated_on_the_plate(orc):
    xyz, tri = M.plate()
    c, rb = M.bounding_sphere(xyz)
    S, alpha = 5.0, math.radians(30.0)
    Vhat = W.plate_alpha_dir(alpha)
    params = dict(**W.base_state(S=S), dir=Vhat, eps_diffuse=1.0, A_ref=1.0, r_cv=1.05 * rb, center=tuple(c),
                  seed=2024, max_bounces=8)
    n_runs = 256
    cd, sig = _runs(orc, xyz, tri, params, 20_000, n_runs)
    F = orc.panel_sum(xyz, tri, Vhat, S, 1.0, math.sqrt(0.3), two_sided=True)
    ref = F @ np.asarray(Vhat) / (0.5 * S * S)
    _check_z((cd - ref) / sig, n_runs)
    # sigma itself is nearly constant between runs of equal size
    assert sig.std() < 0.05 * sig.mean()


def test_sigma_calibrated_on_the_icosphere(orc):
    case = W.icosphere_case(N=1)
    params = dict(case["params"], seed=77)
    n_runs = 256
    cd, sig = _runs(orc, case["xyz"], case["tri"], params, 4_000, n_runs)
    F = orc.panel_sum(case["xyz"], case["tri"], (0, 0, 1), 7.5, 1.0, math.sqrt(0.3))
    ref = F[2] / (0.5 * 7.5 ** 2 * math.pi)
    _check_z((cd - ref) / sig, n_runs)


def test_sigma_matches_the_scatter_on_a_concave_shell(orc):
    """Multiple reflections: each entering particle hits the shell about twice,
    so a per-hit error estimate would differ from the per-particle one."""
    case = W.hemisphere_case(N=1, n_lat=8, n_lon=24)
    params = dict(case["params"], max_bounces=64)
    n_runs = 256
    cd, sig = _runs(orc, case["xyz"], case["tri"], params, 4_000, n_runs)
    ratio = cd.var(ddof=1) / np.mean(sig ** 2)
    assert abs(ratio - 1.0) < 4.0 * math.sqrt(2.0 / (n_runs - 1)), ratio
