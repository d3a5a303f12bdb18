"""Pins of the oracle's moments about a reference point (CPU only).

§III.D.1 computes the aerodynamic moment about the quarter chord and divides
it by q_inf and the chord.  The torque sum is pinned on a flat plate, where the
flux and hence the load are uniform over the sheet, so the expected torque
about any point is (centroid - ref) x F with F the plate's exact force (the
panel sum, itself pinned to Sentman's Eq. 3); and on the sphere, whose torque
about its centre vanishes by its axial symmetry about the flow.  The
statistical error comes from independent seeds (batch means).  The exact
reference-shift identity and the coefficient definitions close the set.
"""
import math

import numpy as np
import pytest

from tpmc_inputs import meshes as M
from tpmc_inputs import workloads as W


def _batch(orc, mesh, params, N, seeds):
    T, F = [], []
    for s in seeds:
        r, _, _ = orc.trace(mesh, orc.make_params(**dict(params, seed=s)), N)
        T.append(r["torque"])
        F.append(r["force"])
    T = np.array(T)
    return T.mean(axis=0), T.std(axis=0, ddof=1) / math.sqrt(len(seeds)), np.array(F).mean(axis=0)


@pytest.mark.parametrize("ref", [(0.0, 0.0, 0.0), (0.3, -0.2, -0.5)])
def test_plate_torque_is_lever_arm_cross_exact_force(orc, ref):
    xyz, tri = M.plate(1.0)
    mesh = orc.Mesh(xyz, tri)
    S, alpha = 5.0, math.radians(40.0)
    Vhat = W.plate_alpha_dir(alpha)
    params = dict(**W.base_state(S=S), dir=Vhat, eps_diffuse=1.0, A_ref=1.0, ref_point=ref, r_cv=0.75)
    T, se, _ = _batch(orc, mesh, params, 40_000, range(1, 13))
    F_exact_nd = orc.panel_sum(xyz, tri, Vhat, S, 1.0, math.sqrt(0.3), two_sided=True)  # units n m c^2 per area
    st = W.base_state(S=S)
    c = math.sqrt(2 * W.K_B * st["T_inf"] / st["m"])
    F_exact = F_exact_nd * st["n"] * st["m"] * c * c  # plate area 1 m^2
    expect = np.cross(-np.asarray(ref), F_exact)  # centroid at the origin
    scale = np.linalg.norm(F_exact) * 0.5
    assert np.all(np.abs(T - expect) <= 4.5 * se + 1e-4 * scale), (T, expect, se)


def test_sphere_torque_about_its_centre_vanishes(orc):
    xyz, tri = M.icosphere(3)
    mesh = orc.Mesh(xyz, tri)
    Vhat = np.array([0.3, -0.5, 0.81])
    params = dict(**W.base_state(S=3.0), dir=tuple(Vhat), eps_diffuse=1.0, A_ref=math.pi, r_cv=1.2)
    T, se, F = _batch(orc, mesh, params, 20_000, range(21, 33))
    assert np.all(np.abs(T) <= 4.5 * se + 1e-6 * np.linalg.norm(F)), (T, se)
    # an off-centre reference point picks up exactly (centre - ref) x F on average
    ref = np.array([0.0, 0.7, -0.2])
    T2, se2, F2 = _batch(orc, mesh, dict(params, ref_point=tuple(ref)), 20_000, range(21, 33))
    np.testing.assert_allclose(T2, np.cross(-ref, F2), rtol=0, atol=4.5 * float(se2.max()) + 1e-6 * np.linalg.norm(F))


def test_reference_shift_identity_and_coefficients(orc):
    case = W.satellite_moment_case(N=20_000)
    mesh = orc.Mesh(case["xyz"], case["tri"])
    V, _, _ = W.alpha_beta_dirs([35.0], [60.0])
    p1 = dict(case["params"], dir=tuple(V[0]))
    r1, _, _ = orc.trace(mesh, orc.make_params(**p1), case["N"])
    ref2 = (0.4, -1.0, 0.2)
    r2, _, _ = orc.trace(mesh, orc.make_params(**dict(p1, ref_point=ref2)), case["N"])
    d = np.asarray(p1["ref_point"]) - np.asarray(ref2)
    np.testing.assert_allclose(r2["torque"], np.asarray(r1["torque"]) + np.cross(d, r1["force"]),
                               rtol=1e-9, atol=1e-9 * np.linalg.norm(r1["torque"]))
    q, A, l = r1["q_inf"], p1["A_ref"], p1["l_ref"]
    np.testing.assert_allclose(r1["CM"], np.asarray(r1["torque"]) / (q * A * l), rtol=1e-14)
    np.testing.assert_allclose(r1["CF"], np.asarray(r1["force"]) / (q * A), rtol=1e-14)
    assert abs(np.dot(r1["CF"], V[0]) - r1["CD"]) < 1e-12 * abs(r1["CD"])


def test_alpha_beta_convention(orc):
    """The pitch axis is perpendicular to the roll axis and the flow, and a
    positive rotation about it carries the roll axis toward the arriving flow."""
    V, E, grid = W.alpha_beta_dirs([0.0, 20.0, 70.0, -45.0], [0.0, 90.0, 200.0])
    for v, e, (a, b) in zip(V, E, grid):
        d = -v
        assert abs(np.linalg.norm(v) - 1) < 1e-15 and abs(e @ [0, 0, 1]) < 1e-15
        assert abs(d @ e) < 1e-15
        assert abs(math.degrees(math.acos(np.clip(d[2], -1, 1))) - abs(a)) < 1e-9
        # a small rotation about e moves z by e x z; that step reduces the angle to d when a > 0
        step = np.cross(e, [0.0, 0.0, 1.0])
        if abs(a) > 1e-9:
            assert (step @ d) * np.sign(a) > 0
