"""Seeded synthetic TPMC workloads: free-stream states, attitudes and seeds.

The paper's verification runs (§III.C) use T_inf = 922 K, T_W = 300 K and
1e7 particles per case; the workloads below follow the benchmark
configurations (atomic oxygen, T_inf = 1000 K) and also keep the paper's
922 K case.  Nothing here computes any part of the method: these are the
inputs both the oracle and the CUDA library receive.
"""
from __future__ import annotations

import math

import numpy as np

from . import meshes

AMU = 1.66053906660e-27  # kg
K_B = 1.380649e-23       # J/K
M_OXYGEN = 16.0 * AMU


def stream_speed(S: float, T_inf: float, m: float = M_OXYGEN) -> float:
    """Bulk speed V that gives the speed ratio S = V / sqrt(2 k T / m) (Nomenclature)."""
    return S * math.sqrt(2.0 * K_B * T_inf / m)


def base_state(S=7.5, T_inf=1000.0, T_W=300.0, n=1.0e15, m=M_OXYGEN):
    return dict(n=n, T_inf=T_inf, m=m, V=stream_speed(S, T_inf, m), T_W=T_W)


def icosphere_case(N=100_000, seed=20131213):
    """Sphere R = 1 m as a 1,280-triangle icosphere in a CV of radius 1.5 m; S = 7.5; diffuse; FP64."""
    xyz, tri = meshes.icosphere(3, 1.0)
    st = base_state(S=7.5)
    return dict(name="icosphere-1280-S7.5-fp64", xyz=xyz, tri=tri, N=N,
                params=dict(**st, dir=(0.0, 0.0, 1.0), eps_diffuse=1.0, A_ref=math.pi, ref_point=(0, 0, 0),
                            r_cv=1.5, center=(0, 0, 0), max_bounces=64, seed=seed),
                precision="fp64")


def plate_alpha_dir(alpha_rad: float):
    """Flow direction making angle alpha with the plate normal (+z), in the x-z plane."""
    return (math.sin(alpha_rad), 0.0, -math.cos(alpha_rad))


def cylinder_alpha_dir(alpha_rad: float):
    """Flow direction making angle alpha with the cylinder axis (+z), in the x-z plane."""
    return (math.sin(alpha_rad), 0.0, -math.cos(alpha_rad))


def sweep_cases(shape: str, N_each=10_000_000, n_alpha=32, S_values=(2.0, 5.0, 10.0), eps_values=(0.0, 1.0)):
    """Plate (2 triangles) or closed cylinder (4,096 triangles) over alpha in [0, 90] deg x S x GSI.

    Returns (xyz, tri, list of case dicts).  Seeds: 1000 + case index.
    """
    if shape == "plate":
        xyz, tri = meshes.plate(1.0)
        A_ref = 1.0
        dir_fn = plate_alpha_dir
    elif shape == "cylinder":
        xyz, tri = meshes.cylinder(0.5, 2.0, 128, 15)
        A_ref = 2.0 * 0.5 * 2.0
        dir_fn = cylinder_alpha_dir
    else:
        raise ValueError(shape)
    c, rb = meshes.bounding_sphere(xyz)
    cases = []
    k = 0
    for eps in eps_values:
        for S in S_values:
            for i in range(n_alpha):
                alpha = math.radians(90.0 * i / (n_alpha - 1))
                st = base_state(S=S)
                cases.append(dict(alpha=alpha, S=S, eps=eps, N=N_each,
                                  params=dict(**st, dir=dir_fn(alpha), eps_diffuse=eps, A_ref=A_ref,
                                              ref_point=(0, 0, 0), r_cv=1.05 * rb, center=tuple(c),
                                              max_bounces=64, seed=1000 + k)))
                k += 1
    return xyz, tri, cases


def satellite_case(N=100_000_000, target_triangles=60_000, seed=7):
    """Concave synthetic satellite, flow -x into the dish, Maxwell 0.9 diffuse, S = 7."""
    xyz, tri = meshes.satellite(target_triangles)
    c, rb = meshes.bounding_sphere(xyz)
    st = base_state(S=7.0)
    return dict(name=f"satellite-{tri.shape[0]}-S7", xyz=xyz, tri=tri, N=N,
                params=dict(**st, dir=(-1.0, 0.0, 0.0), eps_diffuse=0.9, A_ref=2.0, ref_point=(0, 0, 0),
                            r_cv=1.05 * rb, center=tuple(c), max_bounces=64, seed=seed),
                precision="fp32")


def hemisphere_case(N=1_000_000, n_lat=32, n_lon=96, S=40.0, S_W=math.sqrt(2.5), seed=5):
    """Concave hemispherical shell (6,048 triangles) facing an axial flow.

    The flow (+z) enters the open side; full diffuse accommodation.  A large
    S (40, T_inf = 1 K) makes the free stream hyperthermal (the incoming part
    of C_D is 2 + 1/S^2), and the wall temperature is set from S_W (640 K for
    the default S_W = 1.58) so that the re-emission term of C_D is large
    against the statistical error.  A_ref is
    the area of the faceted opening (a regular n_lon-gon inscribed in the
    unit circle).
    """
    xyz, tri = meshes.hemisphere_shell(1.0, n_lat, n_lon)
    T_inf = 1.0
    V = stream_speed(S, T_inf)
    T_W = M_OXYGEN * (V / S_W) ** 2 / (2.0 * K_B)
    A_ref = 0.5 * n_lon * math.sin(2.0 * math.pi / n_lon)
    return dict(name=f"hemisphere-{tri.shape[0]}-S{S:g}-SW{S_W:.3g}", xyz=xyz, tri=tri, N=N, S=S, S_W=S_W,
                params=dict(n=1.0e15, T_inf=T_inf, m=M_OXYGEN, V=V, T_W=T_W, dir=(0.0, 0.0, 1.0), eps_diffuse=1.0,
                            A_ref=A_ref, ref_point=(0, 0, 0), r_cv=1.2, center=(0, 0, 0), max_bounces=200,
                            seed=seed),
                precision="fp32")


def table1_state():
    """Flight conditions of §III.D.1, Table 1 (225 km circular orbit): T_inf 809.2 K,
    T_W 300 K, V 7770 m/s, rho 9.06e-14 kg/m^3, read as atomic oxygen (n = rho / m)."""
    return dict(n=9.06e-14 / M_OXYGEN, T_inf=809.2, m=M_OXYGEN, V=7770.0, T_W=300.0)


def alpha_beta_dirs(alphas_deg, betas_deg):
    """Attitudes of the restoring-moment sweep (§III.D.1) about the roll axis +z.

    The flow arrives from d = (sin a cos b, sin a sin b, cos a): a is the angle of
    incidence from the roll axis (a = 0: head-on onto the +z end), b the roll
    angle.  Returns (Vhat, e_p, grid) with Vhat = -d the flow direction, e_p =
    (-sin b, cos b, 0) the pitch axis (a positive moment about e_p turns +z
    toward d, decreasing |a| for a > 0), and grid the (a, b) pairs, a fastest.
    """
    grid = [(a, b) for b in betas_deg for a in alphas_deg]
    V, E = [], []
    for a, b in grid:
        ar, br = math.radians(a), math.radians(b)
        V.append((-math.sin(ar) * math.cos(br), -math.sin(ar) * math.sin(br), -math.cos(ar)))
        E.append((-math.sin(br), math.cos(br), 0.0))
    return np.array(V), np.array(E), grid


def satellite_moment_case(N=100_000, target_triangles=60_000, seed=11):
    """Synthetic satellite at the Table 1 conditions, moments about the quarter
    chord: chord c = 2 m (bus length along the roll axis z), reference point
    c/4 behind the +z end (z = 0.5 m), A_ref = 1 m^2 so that CM = M / (q_inf c)
    is the paper's area-scaled pitching-moment coefficient.  Diffuse walls."""
    xyz, tri = meshes.satellite(target_triangles)
    c, rb = meshes.bounding_sphere(xyz)
    return dict(name=f"satellite-{tri.shape[0]}-table1", xyz=xyz, tri=tri, N=N, chord=2.0,
                params=dict(**table1_state(), dir=(0.0, 0.0, -1.0), eps_diffuse=1.0, A_ref=1.0,
                            ref_point=(0.0, 0.0, 0.5), l_ref=2.0, r_cv=1.05 * rb, center=tuple(c),
                            max_bounces=64, seed=seed),
                precision="fp32")


def attitude_grid(n_yaw=32, n_pitch=32):
    """Yaw, pitch over a 32 x 32 grid of [-90, 90) deg; flow into the body along -(cos p cos y, cos p sin y, sin p)."""
    dirs = []
    for i in range(n_yaw):
        yaw = math.radians(-90.0 + 180.0 * i / n_yaw)
        for j in range(n_pitch):
            pitch = math.radians(-90.0 + 180.0 * j / n_pitch)
            dirs.append((-math.cos(pitch) * math.cos(yaw), -math.cos(pitch) * math.sin(yaw), -math.sin(pitch)))
    return np.array(dirs, dtype=np.float64)


def serving_stream(n_queries=1000, rate_per_s=100.0, seed=1, N_range=(1e5, 1e8)):
    """Poisson arrivals with log-uniform particle counts, random attitudes and S ~ U[3, 12]."""
    rng = np.random.default_rng(seed)
    gaps = rng.exponential(1.0 / rate_per_s, n_queries)
    t = np.cumsum(gaps)
    lo, hi = math.log(N_range[0]), math.log(N_range[1])
    N = np.exp(rng.uniform(lo, hi, n_queries)).astype(np.int64)
    v = rng.normal(size=(n_queries, 3))
    v /= np.linalg.norm(v, axis=1, keepdims=True)
    S = rng.uniform(3.0, 12.0, n_queries)
    mesh_idx = rng.integers(0, 4, n_queries)
    seeds = rng.integers(1, 2**63 - 1, n_queries, dtype=np.int64)
    return [dict(t_arrival=float(t[i]), N=int(N[i]), dir=tuple(v[i]), S=float(S[i]), mesh=int(mesh_idx[i]),
                 seed=int(seeds[i])) for i in range(n_queries)]
