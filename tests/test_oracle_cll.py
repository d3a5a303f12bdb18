"""Pins of the oracle's Cercignani-Lampis-Lord (CLL) surface model (CPU only).

CLL is an alternative to the paper's Maxwell diffuse/specular mix (§II.A),
built as an extension.  Its pins are the model's defining properties:
- at alpha_n = alpha_t = 1 it is the diffuse law, the same uniforms giving
  the same re-emitted velocity as the (separately pinned) Maxwell sampler;
- at 0 it is specular reflection;
- alpha_n is the normal-energy accommodation and sigma_t = 1 - sqrt(1 - alpha_t)
  the tangential-momentum accommodation of a fixed incident velocity;
- reciprocity: molecules arriving with the wall-temperature flux distribution
  leave with the same distribution, whatever the coefficients.
"""
import math

import numpy as np
import pytest
from scipy import stats

from tpmc_inputs import meshes as M
from tpmc_inputs import workloads as W

NRM = np.array([0.3, -0.2, 0.93])
NRM = NRM / np.linalg.norm(NRM)
T1 = np.cross(NRM, [1.0, 0.0, 0.0])
T1 = T1 / np.linalg.norm(T1)
T2 = np.cross(NRM, T1)
CW = 0.6  # wall thermal speed over the free-stream c_mp


def test_cll_limits_are_the_diffuse_law_and_specular_reflection(orc):
    rng = np.random.default_rng(3)
    for _ in range(200):
        v = rng.normal(size=3) * 2.0
        if v @ NRM > 0:
            v = -v
        u = (rng.integers(0, 2**23, size=4) + 0.5) * 2.0**-23
        # diffuse: the Maxwell sampler takes (choice, normal, tangential speed, angle)
        d_cll = orc.cll(v, NRM, T1, u, 1.0, 1.0, CW)
        d_max = orc.gsi(v, NRM, T1, [0.0, u[0], u[2], u[3]], 1.0, CW)
        np.testing.assert_allclose(d_cll, d_max, rtol=1e-13, atol=1e-13)
        s_cll = orc.cll(v, NRM, T1, u, 0.0, 0.0, CW)
        np.testing.assert_allclose(s_cll, v - 2 * (v @ NRM) * NRM, rtol=1e-13, atol=1e-13)
        # the outgoing velocity always leaves the surface
        for an, at in ((0.3, 0.5), (0.9, 0.2)):
            assert orc.cll(v, NRM, T1, u, an, at, CW) @ NRM >= 0.0


def _many(orc, v, alpha_n, alpha_t, n, seed):
    rng = np.random.default_rng(seed)
    U = (rng.integers(0, 2**23, size=(n, 4)) + 0.5) * 2.0**-23
    return np.array([orc.cll(v, NRM, T1, u, alpha_n, alpha_t, CW) for u in U])


@pytest.mark.parametrize("alpha_n,sigma_t", [(0.3, 0.2), (0.8, 0.6)])
def test_cll_coefficients_are_the_accommodation_coefficients(orc, alpha_n, sigma_t):
    alpha_t = sigma_t * (2.0 - sigma_t)
    vn_in, vt_in = 1.4, np.array([0.9, -0.5])  # c_W units
    v = CW * (-vn_in * NRM + vt_in[0] * T1 + vt_in[1] * T2)
    out = _many(orc, v, alpha_n, alpha_t, 40_000, 7) / CW
    vn = out @ NRM
    vt = np.stack([out @ T1, out @ T2], axis=1)
    # normal energy: E[vn'^2] = alpha_n E_wall + (1 - alpha_n) vn^2, E_wall[vn^2] = 1 for the flux law
    e_n = (vn_in ** 2 - np.mean(vn ** 2)) / (vn_in ** 2 - 1.0)
    se_n = np.std(vn ** 2) / math.sqrt(len(vn)) / abs(vn_in ** 2 - 1.0)
    assert abs(e_n - alpha_n) < 4.5 * se_n, (e_n, alpha_n, se_n)
    # tangential momentum: E[vt'] = (1 - sigma_t) vt
    for k in range(2):
        s_t = 1.0 - np.mean(vt[:, k]) / vt_in[k]
        se = np.std(vt[:, k]) / math.sqrt(len(vt)) / abs(vt_in[k])
        assert abs(s_t - sigma_t) < 4.5 * se, (k, s_t, sigma_t, se)


@pytest.mark.parametrize("alpha_n,sigma_t", [(0.25, 0.4), (0.7, 0.9), (1.0, 0.1)])
def test_cll_reciprocity_keeps_the_wall_flux_distribution(orc, alpha_n, sigma_t):
    alpha_t = sigma_t * (2.0 - sigma_t)
    rng = np.random.default_rng(11)
    n = 12_000
    # incident: the wall-temperature flux law, drawn independently (Rayleigh normal, Gaussian tangential)
    vn = stats.rayleigh(scale=1 / math.sqrt(2)).rvs(n, random_state=rng)
    vt = rng.normal(scale=1 / math.sqrt(2), size=(n, 2))
    U = (rng.integers(0, 2**23, size=(n, 4)) + 0.5) * 2.0**-23
    out = np.array([orc.cll(CW * (-vn[i] * NRM + vt[i, 0] * T1 + vt[i, 1] * T2), NRM, T1, U[i], alpha_n, alpha_t, CW)
                    for i in range(n)]) / CW
    assert stats.kstest(out @ NRM, stats.rayleigh(scale=1 / math.sqrt(2)).cdf).pvalue > 1e-3
    for t in (T1, T2):
        assert stats.kstest(out @ t, stats.norm(scale=1 / math.sqrt(2)).cdf).pvalue > 1e-3


def test_cll_runs_reduce_to_the_maxwell_runs(orc):
    xyz, tri = M.icosphere(2)
    mesh = orc.Mesh(xyz, tri)
    base = dict(**W.base_state(S=4.0), dir=(0.2, 0.5, -0.84), A_ref=math.pi, r_cv=1.3, seed=21, max_bounces=8)
    # specular: no draws are used, so the runs are identical
    r_spec, _, _ = orc.trace(mesh, orc.make_params(**base, eps_diffuse=0.0), 50_000)
    r_cll0, _, _ = orc.trace(mesh, orc.make_params(**base, eps_diffuse=0.0, gsi_model=orc.GSI_CLL, alpha_n=0.0,
                                                  sigma_t=0.0), 50_000)
    np.testing.assert_allclose(r_cll0["sum_dv"], r_spec["sum_dv"], rtol=1e-12)
    # diffuse: same law, other draws: the exact (panel-sum) drag within the error
    r_cll1, _, _ = orc.trace(mesh, orc.make_params(**base, eps_diffuse=0.0, gsi_model=orc.GSI_CLL, alpha_n=1.0,
                                                  sigma_t=1.0), 200_000)
    Vhat = np.asarray(base["dir"]) / np.linalg.norm(base["dir"])
    F = orc.panel_sum(xyz, tri, Vhat, 4.0, 1.0, math.sqrt(0.3))
    ref = F @ Vhat / (0.5 * 16.0 * math.pi)
    assert abs(r_cll1["CD"] - ref) <= 1e-4 * ref + 3.5 * r_cll1["CD_sigma"]
