"""Pins of the oracle's random numbers, flux and seeding laws (CPU only).

Each check compares the oracle with something other than itself: published
known-answer vectors, numerical quadrature of the paper's densities, the
textbook mean speed of a drifting Maxwellian (disk-projection identity) and an
independent flux sampler written here with numpy.
"""
import math
import os

import numpy as np
import pytest
from scipy import integrate, special, stats

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _kat_rows():
    rows = []
    with open(os.path.join(GOLDEN, "philox4x32_10_kat.txt")) as f:
        for line in f:
            if line.strip() and not line.startswith("#"):
                rows.append([int(x, 16) for x in line.split()])
    return rows


def test_philox_known_answers(orc):
    rows = _kat_rows()
    assert len(rows) == 3
    for r in rows:
        out = orc.philox4x32_10(r[0:4], r[4:6])
        assert out.tolist() == r[6:10]


def test_uniform_mapping(orc):
    assert orc.uniform(0) == 2.0 ** -24
    assert orc.uniform(0xFFFFFFFF) == 1.0 - 2.0 ** -24
    assert orc.uniform(0x200) == 1.5 * 2.0 ** -23
    assert orc.uniform(0x1FF) == 2.0 ** -24  # low 9 bits are dropped
    # every value is exactly representable in float32
    rng = np.random.default_rng(0)
    for w in list(rng.integers(0, 2 ** 32, 2000)) + [0, 2 ** 31, 2 ** 32 - 1]:
        u = orc.uniform(int(w))
        assert float(np.float32(u)) == u


def test_seeding_uniforms_layout_and_independence(orc):
    """The five seeding uniforms come from one Philox block: the top 23 bits of
    its four words, and a fifth from bits 0-8 of words 0 and 1 and 0-4 of word
    2, rebuilt here from the published generator's output."""
    seed, stream = 0x0123456789ABCDEF, 77
    for pid in (0, 1, 12345, 2 ** 33 + 5):
        w = orc.philox4x32_10([pid & 0xFFFFFFFF, pid >> 32, stream, 0], [seed & 0xFFFFFFFF, seed >> 32])
        low = (int(w[0]) & 0x1FF) | ((int(w[1]) & 0x1FF) << 9) | ((int(w[2]) & 0x1F) << 18)
        want = [((int(x) >> 9) + 0.5) * 2.0 ** -23 for x in w] + [(low + 0.5) * 2.0 ** -23]
        assert list(orc.seed_uniforms(seed, stream, pid)) == want
    # over many particles: each uniform is uniform, and the fifth is uncorrelated with the others
    U = np.array([orc.seed_uniforms(seed, stream, pid) for pid in range(20_000)])
    for k in range(5):
        assert stats.kstest(U[:, k], "uniform").pvalue > 1e-3
    C = np.corrcoef(U.T)
    assert np.max(np.abs(C - np.eye(5))) < 4.0 / math.sqrt(len(U))


# ------------------------------------------------------------------ Gamma
def _mean_speed_quadrature(S):
    """<|v|> (units of c) of a drifting Maxwellian with mean speed ratio S, by 2-D quadrature."""
    # f(v) d^3v = pi^{-3/2} exp(-(v^2 - 2 v S mu + S^2)) 2 pi v^2 dv dmu
    def inner(v):
        # integral over mu of exp(2 v S mu) on [-1, 1]
        a = 2.0 * v * S
        ang = 2.0 * math.sinh(a) / a if a > 1e-12 else 2.0
        return v ** 3 * 2.0 * math.pi * math.exp(-(v - S) ** 2) * (ang * math.exp(-2 * v * S)) / math.pi ** 1.5
    val, _ = integrate.quad(inner, 0.0, S + 12.0, limit=400, epsabs=0, epsrel=1e-13)
    return val


@pytest.mark.parametrize("S", [0.05, 0.3, 1.0, 2.0, 7.5, 12.0])
def test_gamma_equals_disk_projection(orc, S):
    # Every stream line crosses the sphere's cross-section pi r^2, so the
    # number flux into the sphere is pi r^2 n <|v|>.
    lhs = orc.gamma_coefficient(S)
    rhs = math.pi * _mean_speed_quadrature(S)
    assert abs(lhs - rhs) <= 1e-11 * rhs


@pytest.mark.parametrize("S", [0.3, 2.0, 7.5])
def test_gamma_equals_flux_integral_over_sphere(orc, S):
    # Eq. 7-8: integrate the per-area number flux G(S sin phi) over the unit sphere.
    val, _ = integrate.quad(lambda ph: orc.flux_G(S * math.sin(ph)) * 2 * math.pi * math.cos(ph), -math.pi / 2,
                            math.pi / 2, epsabs=0, epsrel=1e-13, limit=200)
    assert abs(val - orc.gamma_coefficient(S)) <= 1e-11 * val


def test_flux_G_is_the_half_range_number_flux(orc):
    # G(s) = int_0^inf x e^{-(x-s)^2} dx / sqrt(pi)  (one velocity component, units of c)
    for s in [-3.0, -0.5, 0.0, 0.7, 4.0]:
        hi = max(s, 0.0) + 15.0
        val, _ = integrate.quad(lambda x: x * math.exp(-(x - s) ** 2) / math.sqrt(math.pi), 0, hi, epsabs=0,
                                epsrel=1e-13, limit=200)
        assert abs(orc.flux_G(s) - val) < 1e-12 * max(val, 1e-300)
        valp, _ = integrate.quad(lambda x: x * x * math.exp(-(x - s) ** 2) / math.sqrt(math.pi), 0, hi,
                                 epsabs=0, epsrel=1e-13, limit=200)
        assert abs(orc.flux_P(s) - valp) < 1e-12 * valp


# ---------------------------------------------------------- position law
@pytest.mark.parametrize("S", [0.01, 0.5, 2.0, 7.5, 12.0])
def test_g_integrates_to_one(orc, S):
    val, _ = integrate.quad(lambda ph: orc.g_phi(ph, S), -math.pi / 2, math.pi / 2, epsabs=0, epsrel=1e-12,
                            limit=200)
    assert abs(val - 1.0) < 1e-10


def test_g_limits(orc):
    # Eq. 12: S -> 0 gives cos(phi)/2;  Eq. 13: S -> inf gives sin(2 phi) for phi >= 0, else 0.
    for ph in np.linspace(-1.5, 1.5, 13):
        assert abs(orc.g_phi(ph, 1e-6) - 0.5 * math.cos(ph)) < 1e-5
        big = orc.g_phi(ph, 400.0)
        want = math.sin(2 * ph) if ph >= 0 else 0.0
        assert abs(big - want) < 5e-3


@pytest.mark.parametrize("S", [0.2, 2.0, 7.5, 12.0])
def test_position_cdf_matches_quadrature_and_inverts(orc, S):
    assert abs(orc.position_cdf(-1.0, S)) < 1e-15
    assert abs(orc.position_cdf(1.0, S) - 1.0) < 1e-13
    for x in [-0.9, -0.3, 0.0, 0.2, 0.6, 0.95]:
        val, _ = integrate.quad(lambda y: orc.h_x(y, S), -1.0, x, epsabs=1e-15, epsrel=1e-12, limit=200)
        assert abs(orc.position_cdf(x, S) - val) < 1e-12
    for u in [2.0 ** -24, 1e-4, 0.004, 0.3, 0.5, 0.9, 1 - 2.0 ** -24]:
        x = orc.position_inverse(u, S)
        assert -1.0 <= x <= 1.0
        assert abs(orc.position_cdf(x, S) - u) < 1e-14


# ------------------------------------------------------- normal speed law
@pytest.mark.parametrize("s", [-6.0, -2.5, -0.4, 0.0, 0.5, 3.0, 10.0])
def test_normal_speed_normaliser_and_cdf(orc, s):
    # Z(s) = int_0^inf 2 x exp(-(x-s)^2) dx (Eq. 14a with the numerator read as 2 v_n / c)
    Z, _ = integrate.quad(lambda x: 2 * x * math.exp(-(x - s) ** 2), 0, max(s, 0) + 15, epsabs=0, epsrel=1e-13,
                          limit=400, points=[max(s, 0.0)])
    assert abs(orc.normal_speed_norm(s) - Z) < 1e-10 * Z
    tot, _ = integrate.quad(lambda x: orc.normal_speed_pdf(x, s), 0, max(s, 0) + 15, epsrel=1e-12, limit=400,
                            points=[max(s, 0.0)])
    assert abs(tot - 1.0) < 1e-9
    for x in [0.05, 0.5, 1.0, max(s, 0) + 0.3, max(s, 0) + 2.0]:
        val, _ = integrate.quad(lambda y: orc.normal_speed_pdf(y, s), 0, x, epsabs=1e-15, epsrel=1e-12, limit=400)
        assert abs(orc.normal_speed_cdf(x, s) - val) < 1e-9
    for u in [2.0 ** -24, 0.01, 0.5, 0.99, 1 - 2.0 ** -24]:
        x = orc.normal_speed_inverse(u, s)
        assert x > 0
        assert abs(orc.normal_speed_cdf(x, s) - u) < 1e-12
    # upper tail: the root is resolved to double precision (complement of F, by quadrature)
    x = orc.normal_speed_inverse(1 - 2.0 ** -24, s)
    surv, _ = integrate.quad(lambda y: 2 * y * math.exp(-(y - s) ** 2), x, x + 12, epsabs=0, epsrel=1e-13, limit=200)
    assert abs(surv / orc.normal_speed_norm(s) - 2.0 ** -24) < 1e-9 * 2.0 ** -24


# --------------------------------------- joint seeding law (independent sampler)
def _independent_flux_sampler(rng, n, S, Vhat, r):
    """Particles entering a sphere of radius r, by disk projection (no use of Eq. 11 or 14).

    A molecule with velocity v enters the sphere at a point uniform on the
    disk of radius r perpendicular to v, at a rate proportional to |v|; so
    draw v from the drifting Maxwellian, keep it with probability |v| / v_max,
    drop a point uniformly on the disk and move it back to the sphere.
    """
    Vhat = np.asarray(Vhat, float) / np.linalg.norm(Vhat)
    vmax = S + 9.0
    out_v = []
    while sum(len(a) for a in out_v) < n:
        v = S * Vhat + rng.normal(scale=math.sqrt(0.5), size=(2 * n, 3))
        sp = np.linalg.norm(v, axis=1)
        keep = rng.uniform(size=2 * n) * vmax < sp
        out_v.append(v[keep])
    v = np.concatenate(out_v)[:n]
    vh = v / np.linalg.norm(v, axis=1, keepdims=True)
    a = np.where(np.abs(vh[:, :1]) < 0.9, np.array([[1.0, 0, 0]]), np.array([[0, 1.0, 0]]))
    e1 = np.cross(vh, a)
    e1 /= np.linalg.norm(e1, axis=1, keepdims=True)
    e2 = np.cross(vh, e1)
    rho = r * np.sqrt(rng.uniform(size=n))
    ang = 2 * math.pi * rng.uniform(size=n)
    p = rho[:, None] * (np.cos(ang)[:, None] * e1 + np.sin(ang)[:, None] * e2)
    p = p - np.sqrt(r * r - rho * rho)[:, None] * vh
    return p, v


def _local_components(p, v, Vhat, r):
    Vhat = np.asarray(Vhat, float) / np.linalg.norm(Vhat)
    nin = -p / r
    x = nin @ Vhat
    t1 = Vhat[None, :] - x[:, None] * nin
    t1 /= np.linalg.norm(t1, axis=1, keepdims=True)
    t2 = np.cross(t1, nin)
    return x, (v * nin).sum(1), (v * t1).sum(1), (v * t2).sum(1)


@pytest.mark.parametrize("S,Vhat", [(7.5, (0.0, 0.0, 1.0)), (2.0, (0.3, -0.5, 0.8)), (0.7, (0.0, 0.0, -1.0))])
def test_seeding_joint_law_matches_independent_sampler(orc, S, Vhat):
    from tpmc_inputs import workloads as W

    n = 60_000
    r = 1.5
    mesh = orc.Mesh(np.zeros((3, 3)), np.zeros((0, 3), np.uint32))
    st = W.base_state(S=S)
    p = orc.make_params(**st, dir=Vhat, eps_diffuse=1.0, A_ref=1.0, r_cv=r, seed=99, max_bounces=1)
    res, _, rec = orc.trace(mesh, p, n, records=True)
    assert res["n_hits"] == 0 and res["force"] == [0.0, 0.0, 0.0]
    np.testing.assert_allclose(np.linalg.norm(rec["pos"], axis=1), r, rtol=1e-14)
    xo, vno, t1o, t2o = _local_components(rec["pos"], rec["vel"], Vhat, r)
    ps, vs = _independent_flux_sampler(np.random.default_rng(5), n, S, Vhat, r)
    xs, vns, t1s, t2s = _local_components(ps, vs, Vhat, r)
    assert (vno > 0).all()
    for a, b in [(xo, xs), (vno, vns), (t1o, t1s), (t2o, t2s)]:
        assert stats.ks_2samp(a, b).pvalue > 1e-4
    # joint: (x, v_n) on a 6 x 6 grid of the independent sampler's quantiles
    qx = np.quantile(xs, np.linspace(0, 1, 7)[1:-1])
    qv = np.quantile(vns, np.linspace(0, 1, 7)[1:-1])
    ho = np.histogram2d(np.digitize(xo, qx), np.digitize(vno, qv), bins=[np.arange(7) - 0.5] * 2)[0]
    hs = np.histogram2d(np.digitize(xs, qx), np.digitize(vns, qv), bins=[np.arange(7) - 0.5] * 2)[0]
    m = (ho + hs) > 0
    chi2 = (((ho - hs) ** 2)[m] / (ho + hs)[m]).sum()
    dof = m.sum() - 1
    assert stats.chi2.sf(chi2, dof) > 1e-4


def test_seeding_mean_normal_speed_closed_form(orc):
    # E[x] for p(x) = 2 x e^{-(x-s)^2}/Z is (s e^{-s^2} + sqrt(pi)(1/2 + s^2)(1+erf s)) / Z = 2 sqrt(pi) P(s) / Z
    for s in [-2.0, 0.0, 1.5, 6.0]:
        Z = math.exp(-s * s) + math.sqrt(math.pi) * s * (1 + math.erf(s))
        want = (s * math.exp(-s * s) + math.sqrt(math.pi) * (0.5 + s * s) * (1 + math.erf(s))) / Z
        us = (np.arange(20000) + 0.5) / 20000
        got = np.mean([orc.normal_speed_inverse(u, s) for u in us])
        assert abs(got - want) < 2e-4 * want
