"""FP64 CPU oracle for the TPMC hot path (test infrastructure only).

Only the test suite, ``__graft_entry__.smoke()`` and the benchmark's CPU-baseline
leg may import this package.  The product library never loads it and shares no
code with it: the oracle is a plain, slow, double-precision statement of the
method in Parham & Barba (arXiv 1312.3691), written in ``tpmc_oracle.cpp`` and
loaded here through ctypes.

Parity status per function (the pins live in ``tests/test_oracle_*.py``):

* Philox4x32-10, uniform mapping ........ pinned (published known-answer vectors)
* Gamma (Eq. 10) ........................ pinned (disk-projection identity, quadrature)
* g(phi|S), H, H^-1 (Eq. 11-13) .......... pinned (quadrature, both limits, KS)
* p(v_n), F_n, F_n^-1 (Eq. 14a) .......... pinned (quadrature, moments, independent sampler)
* Rodrigues (Eq. 15) .................... pinned (rotation matrix identities)
* closest hit ........................... pinned (numpy linear solve, brute force vs BVH)
* re-emission ........................... pinned (half-range Maxwellian moments, KS)
* sphere / plate / cylinder C_D (Eq. 3-4)  pinned (quadrature, textbook cross-flow form)
* full run on convex meshes ............. pinned (panel-sum expectation within 3 sigma)
* full run on concave meshes ............ pinned (Pratt's hemisphere constant, Eq. 5, re-derived by a
                                          view-factor quadrature; exact specular chord construction)
* Cercignani-Lampis-Lord (extension) .... pinned (alpha = 1 is the diffuse law, 0 specular; normal-energy and
                                          tangential-momentum accommodation exactly alpha_n, sigma_t;
                                          reciprocity: a wall-temperature flux comes back unchanged)
* rectangular-CV seeding (§I, §III.A) ... pinned (flux-weighted faces reproduce Eq. 4 at every incidence;
                                          face shares against the flat-plate flux; KS of both face laws)
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "tpmc_oracle.cpp")
_LIB = os.path.join(_HERE, "liboracle_tpmc.so")
_lock = threading.Lock()
_lib = None

MAX_REC = 16


def build(force: bool = False) -> str:
    """Compile the oracle with g++ (plain -O2, no target-specific flags)."""
    with _lock:
        if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
            tmp = _LIB + f".tmp{os.getpid()}"
            subprocess.check_call(["g++", "-O2", "-std=c++17", "-fPIC", "-shared", "-o", tmp, _SRC, "-lpthread"])
            os.replace(tmp, _LIB)
    return _LIB


class Params(ctypes.Structure):
    _fields_ = [
        ("n", ctypes.c_double), ("T_inf", ctypes.c_double), ("m", ctypes.c_double), ("V", ctypes.c_double),
        ("dir", ctypes.c_double * 3),
        ("T_W", ctypes.c_double), ("eps_diffuse", ctypes.c_double),
        ("A_ref", ctypes.c_double), ("ref_point", ctypes.c_double * 3),
        ("r_cv", ctypes.c_double), ("center", ctypes.c_double * 3),
        ("max_bounces", ctypes.c_uint32), ("stream", ctypes.c_uint32), ("seed", ctypes.c_uint64),
        ("t_min_len", ctypes.c_double), ("intersect", ctypes.c_int32), ("threads", ctypes.c_int32),
        ("cv_kind", ctypes.c_int32), ("pad", ctypes.c_int32),
        ("box_lo", ctypes.c_double * 3), ("box_hi", ctypes.c_double * 3), ("l_ref", ctypes.c_double),
        ("gsi_model", ctypes.c_int32), ("pad2", ctypes.c_int32), ("alpha_n", ctypes.c_double),
        ("sigma_t", ctypes.c_double),
    ]

GSI_MAXWELL, GSI_CLL = 0, 1

CV_SPHERE, CV_BOX_FLUX, CV_BOX_MAXWELL = 0, 1, 2


class Result(ctypes.Structure):
    _fields_ = [
        ("force", ctypes.c_double * 3), ("torque", ctypes.c_double * 3),
        ("CD", ctypes.c_double), ("CD_sigma", ctypes.c_double), ("gamma", ctypes.c_double),
        ("weight", ctypes.c_double), ("S", ctypes.c_double), ("S_W", ctypes.c_double),
        ("q_inf", ctypes.c_double), ("c_mp", ctypes.c_double),
        ("sum_dv", ctypes.c_double * 3), ("sum_rdv", ctypes.c_double * 3),
        ("sum_d", ctypes.c_double), ("sum_d2", ctypes.c_double),
        ("n_particles", ctypes.c_uint64), ("n_hits", ctypes.c_uint64),
        ("n_hit_particles", ctypes.c_uint64), ("n_truncated", ctypes.c_uint64),
        ("CF", ctypes.c_double * 3), ("CM", ctypes.c_double * 3),
    ]

    def as_dict(self) -> dict:
        out = {}
        for name, _ in self._fields_:
            v = getattr(self, name)
            out[name] = list(v) if isinstance(v, ctypes.Array) else v
        return out


class Records(ctypes.Structure):
    _fields_ = [
        ("pos", ctypes.POINTER(ctypes.c_double)), ("vel", ctypes.POINTER(ctypes.c_double)),
        ("dv", ctypes.POINTER(ctypes.c_double)), ("n_hits", ctypes.POINTER(ctypes.c_uint32)),
        ("truncated", ctypes.POINTER(ctypes.c_uint32)), ("tri", ctypes.POINTER(ctypes.c_uint32)),
        ("bary", ctypes.POINTER(ctypes.c_double)), ("cosi", ctypes.POINTER(ctypes.c_double)),
        ("edge", ctypes.POINTER(ctypes.c_double)), ("K", ctypes.c_uint32),
    ]


_D = ctypes.c_double
_PD = ctypes.POINTER(ctypes.c_double)
_PU32 = ctypes.POINTER(ctypes.c_uint32)


def lib():
    global _lib
    if _lib is None:
        path = build()
        L = ctypes.CDLL(path)
        for name in ["orc_uniform"]:
            getattr(L, name).restype = _D
            getattr(L, name).argtypes = [ctypes.c_uint32]
        for name in ["orc_gamma_coefficient", "orc_position_norm", "orc_normal_speed_norm", "orc_flux_G",
                     "orc_flux_P"]:
            getattr(L, name).restype = _D
            getattr(L, name).argtypes = [_D]
        for name in ["orc_g_phi", "orc_h_x", "orc_position_cdf", "orc_position_inverse", "orc_normal_speed_pdf",
                     "orc_normal_speed_cdf", "orc_normal_speed_inverse", "orc_sphere_cd_paper",
                     "orc_truncated_normal_cdf", "orc_truncated_normal_inverse"]:
            getattr(L, name).restype = _D
            getattr(L, name).argtypes = [_D, _D]
        for name in ["orc_plate_cd_paper", "orc_plate_cd_derived"]:
            getattr(L, name).restype = _D
            getattr(L, name).argtypes = [_D, _D, _D]
        L.orc_sphere_cd_quadrature.restype = _D
        L.orc_sphere_cd_quadrature.argtypes = [_D, _D, _D, ctypes.c_int]
        L.orc_cylinder_cd_quadrature.restype = _D
        L.orc_cylinder_cd_quadrature.argtypes = [_D, _D, _D, _D, _D, _D, ctypes.c_int]
        L.orc_seed_uniforms.restype = None
        L.orc_seed_uniforms.argtypes = [ctypes.c_uint64, ctypes.c_uint32, ctypes.c_uint64, _PD]
        L.orc_philox4x32_10.restype = None
        L.orc_philox4x32_10.argtypes = [_PU32, _PU32, _PU32]
        L.orc_surface_force.restype = None
        L.orc_surface_force.argtypes = [_PD, _PD, _D, _D, _D, _PD]
        L.orc_rodrigues.restype = None
        L.orc_rodrigues.argtypes = [_PD, _PD, _PD]
        L.orc_gsi.restype = None
        L.orc_gsi.argtypes = [_PD, _PD, _PD, _PD, _D, _D, _PD]
        L.orc_cll.restype = None
        L.orc_cll.argtypes = [_PD, _PD, _PD, _PD, _D, _D, _D, _PD]
        L.orc_panel_sum.restype = None
        L.orc_panel_sum.argtypes = [_PD, _PU32, ctypes.c_uint32, ctypes.c_int, _PD, _D, _D, _D, _PD]
        L.orc_mesh_create.restype = ctypes.c_void_p
        L.orc_mesh_create.argtypes = [_PD, ctypes.c_uint32, _PU32, ctypes.c_uint32]
        L.orc_mesh_destroy.restype = None
        L.orc_mesh_destroy.argtypes = [ctypes.c_void_p]
        L.orc_closest_hit.restype = ctypes.c_int64
        L.orc_closest_hit.argtypes = [ctypes.c_void_p, _PD, _PD, ctypes.c_int64, _D, ctypes.c_int, _PD]
        L.orc_trace.restype = ctypes.c_int
        L.orc_trace.argtypes = [ctypes.c_void_p, ctypes.POINTER(Params), ctypes.c_uint64, ctypes.c_uint64,
                                ctypes.c_uint64, ctypes.POINTER(Result), _PD, ctypes.POINTER(Records)]
        _lib = L
    return _lib


def _pd(a: np.ndarray):
    return a.ctypes.data_as(_PD)


def _pu32(a: np.ndarray):
    return a.ctypes.data_as(_PU32)


def _vec3(v):
    a = np.ascontiguousarray(np.asarray(v, dtype=np.float64).reshape(3))
    return a


# ----------------------------------------------------------------- wrappers
def philox4x32_10(ctr, key) -> np.ndarray:
    c = np.ascontiguousarray(np.asarray(ctr, dtype=np.uint32).reshape(4))
    k = np.ascontiguousarray(np.asarray(key, dtype=np.uint32).reshape(2))
    out = np.zeros(4, dtype=np.uint32)
    lib().orc_philox4x32_10(_pu32(c), _pu32(k), _pu32(out))
    return out


def uniform(word: int) -> float:
    return lib().orc_uniform(int(word))


def _scalar(name):
    def f(*args):
        return getattr(lib(), name)(*[float(a) for a in args])
    f.__name__ = name[4:]
    return f


gamma_coefficient = _scalar("orc_gamma_coefficient")
position_norm = _scalar("orc_position_norm")
g_phi = _scalar("orc_g_phi")
h_x = _scalar("orc_h_x")
position_cdf = _scalar("orc_position_cdf")
position_inverse = _scalar("orc_position_inverse")
normal_speed_norm = _scalar("orc_normal_speed_norm")
normal_speed_pdf = _scalar("orc_normal_speed_pdf")
normal_speed_cdf = _scalar("orc_normal_speed_cdf")
normal_speed_inverse = _scalar("orc_normal_speed_inverse")
truncated_normal_cdf = _scalar("orc_truncated_normal_cdf")
truncated_normal_inverse = _scalar("orc_truncated_normal_inverse")
flux_G = _scalar("orc_flux_G")
flux_P = _scalar("orc_flux_P")
sphere_cd_paper = _scalar("orc_sphere_cd_paper")
plate_cd_paper = _scalar("orc_plate_cd_paper")
plate_cd_derived = _scalar("orc_plate_cd_derived")


def sphere_cd_quadrature(S, eps, cw, nodes=400):
    return lib().orc_sphere_cd_quadrature(float(S), float(eps), float(cw), int(nodes))


def cylinder_cd_quadrature(S, eps, cw, alpha, R=0.5, L=2.0, nodes=4096):
    return lib().orc_cylinder_cd_quadrature(float(S), float(eps), float(cw), float(alpha), float(R), float(L),
                                            int(nodes))


def surface_force(nrm, Vhat, S, eps, cw) -> np.ndarray:
    out = np.zeros(3)
    lib().orc_surface_force(_pd(_vec3(nrm)), _pd(_vec3(Vhat)), float(S), float(eps), float(cw), _pd(out))
    return out


def rodrigues(Vhat, x) -> np.ndarray:
    out = np.zeros(3)
    lib().orc_rodrigues(_pd(_vec3(Vhat)), _pd(_vec3(x)), _pd(out))
    return out


def gsi(v, nrm, t1, u, eps, cw) -> np.ndarray:
    out = np.zeros(3)
    uu = np.ascontiguousarray(np.asarray(u, dtype=np.float64).reshape(4))
    lib().orc_gsi(_pd(_vec3(v)), _pd(_vec3(nrm)), _pd(_vec3(t1)), _pd(uu), float(eps), float(cw), _pd(out))
    return out


def seed_uniforms(seed, stream, pid) -> np.ndarray:
    out = np.zeros(5)
    lib().orc_seed_uniforms(int(seed), int(stream), int(pid), _pd(out))
    return out


def cll(v, nrm, t1, u, alpha_n, alpha_t, cw) -> np.ndarray:
    out = np.zeros(3)
    uu = np.ascontiguousarray(np.asarray(u, dtype=np.float64).reshape(4))
    lib().orc_cll(_pd(_vec3(v)), _pd(_vec3(nrm)), _pd(_vec3(t1)), _pd(uu), float(alpha_n), float(alpha_t), float(cw),
                  _pd(out))
    return out


def panel_sum(xyz, tri, Vhat, S, eps, cw, two_sided=False) -> np.ndarray:
    X = np.ascontiguousarray(np.asarray(xyz, dtype=np.float64))
    T = np.ascontiguousarray(np.asarray(tri, dtype=np.uint32))
    out = np.zeros(3)
    lib().orc_panel_sum(_pd(X), _pu32(T), T.shape[0], int(bool(two_sided)), _pd(_vec3(Vhat)), float(S),
                        float(eps), float(cw), _pd(out))
    return out


class Mesh:
    """Oracle-side triangle mesh (own copy, own median-split BVH)."""

    def __init__(self, xyz, tri):
        self.xyz = np.ascontiguousarray(np.asarray(xyz, dtype=np.float64).reshape(-1, 3))
        self.tri = np.ascontiguousarray(np.asarray(tri, dtype=np.uint32).reshape(-1, 3))
        self._h = lib().orc_mesh_create(_pd(self.xyz), self.xyz.shape[0], _pu32(self.tri), self.tri.shape[0])
        if not self._h:
            raise ValueError("invalid mesh (triangle index out of range)")

    def __del__(self):
        h = getattr(self, "_h", None)
        if h and _lib is not None:
            _lib.orc_mesh_destroy(h)
            self._h = None

    @property
    def n_tri(self) -> int:
        return self.tri.shape[0]

    def closest_hit(self, o, d, exclude=-1, t_min=0.0, mode=0):
        tuv = np.zeros(3)
        i = lib().orc_closest_hit(self._h, _pd(_vec3(o)), _pd(_vec3(d)), int(exclude), float(t_min), int(mode),
                                  _pd(tuv))
        return int(i), tuv


def make_params(*, n, T_inf, m, V, dir, T_W, eps_diffuse, A_ref, ref_point=(0, 0, 0), r_cv=0.0, center=(0, 0, 0),
                max_bounces=64, stream=0, seed=0, t_min_len=1e-9, intersect=0, threads=0, cv_kind=CV_SPHERE,
                box_lo=(0, 0, 0), box_hi=(0, 0, 0), l_ref=0.0, gsi_model=GSI_MAXWELL, alpha_n=1.0,
                sigma_t=1.0) -> Params:
    p = Params()
    p.n, p.T_inf, p.m, p.V = float(n), float(T_inf), float(m), float(V)
    p.dir[:] = [float(x) for x in dir]
    p.T_W, p.eps_diffuse, p.A_ref = float(T_W), float(eps_diffuse), float(A_ref)
    p.ref_point[:] = [float(x) for x in ref_point]
    p.r_cv = float(r_cv)
    p.center[:] = [float(x) for x in center]
    p.max_bounces, p.stream, p.seed = int(max_bounces), int(stream), int(seed)
    p.t_min_len, p.intersect, p.threads = float(t_min_len), int(intersect), int(threads)
    p.cv_kind = int(cv_kind)
    p.box_lo[:] = [float(x) for x in box_lo]
    p.box_hi[:] = [float(x) for x in box_hi]
    p.l_ref = float(l_ref)
    p.gsi_model, p.alpha_n, p.sigma_t = int(gsi_model), float(alpha_n), float(sigma_t)
    return p


def trace(mesh: Mesh, params: Params, N_total: int, pid_begin: int = 0, count: int | None = None,
          panels: bool = False, records: bool = False, K: int = MAX_REC):
    """Run the oracle over particle ids [pid_begin, pid_begin+count) of an N_total run.

    Returns (result dict, panel_dv array or None, records dict or None).
    """
    count = N_total - pid_begin if count is None else count
    res = Result()
    panel = np.zeros((mesh.n_tri, 3)) if panels else None
    rec = None
    recd = None
    if records:
        recd = {
            "pos": np.zeros((count, 3)), "vel": np.zeros((count, 3)), "dv": np.zeros((count, 3)),
            "n_hits": np.zeros(count, np.uint32), "truncated": np.zeros(count, np.uint32),
            "tri": np.full((count, K), 0xFFFFFFFF, np.uint32), "bary": np.ones((count, K)),
            "cosi": np.ones((count, K)), "edge": np.full((count, K), np.inf),
        }
        rec = Records(_pd(recd["pos"]), _pd(recd["vel"]), _pd(recd["dv"]), _pu32(recd["n_hits"]),
                      _pu32(recd["truncated"]), _pu32(recd["tri"]), _pd(recd["bary"]), _pd(recd["cosi"]),
                      _pd(recd["edge"]), K)
    rc = lib().orc_trace(mesh._h, ctypes.byref(params), int(N_total), int(pid_begin), int(count),
                         ctypes.byref(res), _pd(panel) if panels else None,
                         ctypes.byref(rec) if records else None)
    if rc != 0:
        raise ValueError("oracle rejected the parameters")
    return res.as_dict(), panel, recd
