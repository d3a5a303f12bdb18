"""ctypes binding of include/tpmc.h (argument marshalling only).

Every function here has the name of the C entry point it calls, raises
TpmcError on a non-OK status, and runs no part of the method itself: all of
seeding, tracing, re-emission and reduction happen in libtpmc.so.  Device
buffers may be passed as torch CUDA tensors (their data_ptr is used) and
streams as torch.cuda.Stream objects; torch is not needed otherwise.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libtpmc.so")

TPMC_OK, TPMC_EINVAL, TPMC_ENOMEM, TPMC_EBUSY, TPMC_ETIMEOUT, TPMC_ECUDA, TPMC_ENOTFOUND = range(7)
TPMC_FP32, TPMC_FP64 = 0, 1
TPMC_CV_SPHERE, TPMC_CV_BOX_FLUX, TPMC_CV_BOX_MAXWELL = 0, 1, 2
TPMC_GSI_MAXWELL, TPMC_GSI_CLL = 0, 1
STATUS_NAMES = {0: "OK", 1: "EINVAL", 2: "ENOMEM", 3: "EBUSY", 4: "ETIMEOUT", 5: "ECUDA", 6: "ENOTFOUND"}

_D3 = ctypes.c_double * 3


class tpmc_params(ctypes.Structure):
    _fields_ = [
        ("n", ctypes.c_double), ("T_inf", ctypes.c_double), ("m", ctypes.c_double), ("V", ctypes.c_double),
        ("dir", _D3), ("T_W", ctypes.c_double), ("eps_diffuse", ctypes.c_double), ("A_ref", ctypes.c_double),
        ("ref_point", _D3), ("r_cv", ctypes.c_double), ("center", _D3),
        ("max_bounces", ctypes.c_uint32), ("precision", ctypes.c_uint32), ("seed", ctypes.c_uint64),
        ("stream_id", ctypes.c_uint32), ("want_panels", ctypes.c_uint32),
        ("cv_kind", ctypes.c_uint32), ("pad_cv", ctypes.c_uint32), ("box_lo", _D3), ("box_hi", _D3),
        ("l_ref", ctypes.c_double), ("gsi_model", ctypes.c_uint32), ("pad_gsi", ctypes.c_uint32),
        ("alpha_n", ctypes.c_double), ("sigma_t", ctypes.c_double),
    ]


class tpmc_result(ctypes.Structure):
    _fields_ = [
        ("force", _D3), ("torque", _D3), ("CD", ctypes.c_double), ("CD_sigma", ctypes.c_double),
        ("CF", _D3), ("CM", _D3),
        ("S", ctypes.c_double), ("S_W", ctypes.c_double), ("gamma", ctypes.c_double), ("weight", ctypes.c_double),
        ("q_inf", ctypes.c_double), ("c_mp", ctypes.c_double), ("r_cv", ctypes.c_double), ("center", _D3),
        ("fixed_quantum", ctypes.c_double), ("sum_dv_q", ctypes.c_int64 * 3), ("sum_rdv_q", ctypes.c_int64 * 3),
        ("n_particles", ctypes.c_uint64), ("n_hits", ctypes.c_uint64), ("n_hit_particles", ctypes.c_uint64),
        ("n_truncated", ctypes.c_uint64), ("n_node_visits", ctypes.c_uint64), ("n_tri_tests", ctypes.c_uint64),
        ("query_id", ctypes.c_uint64), ("ms", ctypes.c_double), ("status", ctypes.c_int32), ("pad_", ctypes.c_int32),
    ]

    def as_dict(self) -> dict:
        out = {}
        for name, _ in self._fields_:
            v = getattr(self, name)
            out[name] = list(v) if isinstance(v, ctypes.Array) else v
        return out


class tpmc_records(ctypes.Structure):
    _fields_ = [
        ("pos", ctypes.POINTER(ctypes.c_double)), ("vel", ctypes.POINTER(ctypes.c_double)),
        ("dv", ctypes.POINTER(ctypes.c_double)), ("n_hits", ctypes.POINTER(ctypes.c_uint32)),
        ("truncated", ctypes.POINTER(ctypes.c_uint32)), ("tri", ctypes.POINTER(ctypes.c_uint32)),
        ("K", ctypes.c_uint32),
    ]


class tpmc_mesh_stats(ctypes.Structure):
    _fields_ = [
        ("n_tri", ctypes.c_uint32), ("n_vert", ctypes.c_uint32), ("n_nodes", ctypes.c_uint32),
        ("depth", ctypes.c_uint32), ("n_skipped", ctypes.c_uint32), ("leaf_max", ctypes.c_uint32),
        ("bound_center", _D3), ("bound_radius", ctypes.c_double), ("device_bytes", ctypes.c_uint64),
        ("n_refs", ctypes.c_uint32), ("n_exposed", ctypes.c_uint32),
        ("bvh_width", ctypes.c_uint32), ("node_bytes", ctypes.c_uint32),
    ]


class tpmc_launch(ctypes.Structure):
    _fields_ = [("block", ctypes.c_uint32), ("blocks_per_sm", ctypes.c_uint32), ("chunk", ctypes.c_uint32),
                ("smem_nodes", ctypes.c_uint32), ("refill_at", ctypes.c_uint32), ("bvh_leaf", ctypes.c_uint32),
                ("bvh_width", ctypes.c_uint32)]


# (name, argtypes) of every entry point declared in include/tpmc.h
_P = ctypes.c_void_p
_PD = ctypes.POINTER(ctypes.c_double)
_PU32 = ctypes.POINTER(ctypes.c_uint32)
SIGNATURES = {
    "tpmc_create": [ctypes.c_int, ctypes.c_size_t, ctypes.POINTER(_P)],
    "tpmc_destroy": [_P],
    "tpmc_set_stream": [_P, _P],
    "tpmc_last_error": [_P],
    "tpmc_set_counters": [_P, ctypes.c_int],
    "tpmc_memory_info": [_P, ctypes.POINTER(ctypes.c_size_t), ctypes.POINTER(ctypes.c_size_t),
                         ctypes.POINTER(ctypes.c_uint64)],
    "tpmc_mesh_load": [_P, _PD, ctypes.c_uint32, _PU32, ctypes.c_uint32, _PU32],
    "tpmc_mesh_unload": [_P, ctypes.c_uint32],
    "tpmc_mesh_info": [_P, ctypes.c_uint32, ctypes.POINTER(tpmc_mesh_stats)],
    "tpmc_trace": [_P, ctypes.c_uint32, ctypes.POINTER(tpmc_params), ctypes.c_uint64, ctypes.POINTER(tpmc_result)],
    "tpmc_panels": [_P, ctypes.c_uint64, _PD, _PD, ctypes.c_uint32],
    "tpmc_panel_sums": [_P, ctypes.c_uint64, _P, ctypes.c_uint32],
    "tpmc_trace_records": [_P, ctypes.c_uint32, ctypes.POINTER(tpmc_params), ctypes.c_uint64,
                           ctypes.POINTER(tpmc_records), ctypes.POINTER(tpmc_result)],
    "tpmc_sweep": [_P, ctypes.c_uint32, ctypes.POINTER(tpmc_params), _PD, _PD, ctypes.c_uint32, ctypes.c_uint64,
                   ctypes.POINTER(tpmc_result)],
    "tpmc_sweep_device": [_P, ctypes.c_uint32, ctypes.POINTER(tpmc_params), _P, _P, ctypes.c_uint32,
                          ctypes.c_uint64, _P],
    "tpmc_sweep_noalloc": [_P, ctypes.c_uint32, ctypes.POINTER(tpmc_params), _PD, _PD, ctypes.c_uint32,
                           ctypes.c_uint64, ctypes.POINTER(tpmc_result)],
    "tpmc_submit": [_P, ctypes.c_uint32, ctypes.POINTER(tpmc_params), ctypes.c_uint64,
                    ctypes.POINTER(ctypes.c_uint64)],
    "tpmc_poll": [_P, ctypes.c_uint64, ctypes.c_int, ctypes.POINTER(tpmc_result)],
    "tpmc_tune": [_P, ctypes.c_uint32, ctypes.POINTER(tpmc_params), ctypes.c_uint64, ctypes.POINTER(tpmc_launch)],
    "tpmc_set_launch": [_P, ctypes.POINTER(tpmc_launch)],
    "tpmc_get_launch": [_P, ctypes.c_uint32, ctypes.c_uint32, ctypes.POINTER(tpmc_launch)],
    "tpmc_measure_ceilings": [_P, _PD, _PD],
}

_lib = None


class TpmcError(RuntimeError):
    def __init__(self, status: int, where: str, msg: str):
        super().__init__(f"{where}: {STATUS_NAMES.get(status, status)}: {msg}")
        self.status = status


def lib():
    """Loads libtpmc.so; there is no fallback: a missing library is an error."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"{LIB_PATH} is missing: build it with paper_1312_3691_gb300.build.build()")
        L = ctypes.CDLL(LIB_PATH)
        for name, args in SIGNATURES.items():
            f = getattr(L, name)
            f.argtypes = args
            f.restype = ctypes.c_char_p if name == "tpmc_last_error" else ctypes.c_int
        _lib = L
    return _lib


def _check(st: int, where: str, ctx=None):
    if st != TPMC_OK:
        msg = lib().tpmc_last_error(ctx)
        raise TpmcError(st, where, msg.decode() if msg else "")


def _ptr(x):
    """Device pointer of a torch tensor, or an int address."""
    if x is None:
        return None
    if hasattr(x, "data_ptr"):
        return ctypes.c_void_p(x.data_ptr())
    return ctypes.c_void_p(int(x))


def _pd(a):
    return None if a is None else a.ctypes.data_as(_PD)


def _pu32(a):
    return None if a is None else a.ctypes.data_as(_PU32)


# ---------------------------------------------------------------- entry points
def tpmc_create(device: int = 0, mem_budget_bytes: int = 0):
    h = _P()
    _check(lib().tpmc_create(int(device), int(mem_budget_bytes), ctypes.byref(h)), "tpmc_create")
    return h


def tpmc_destroy(ctx):
    _check(lib().tpmc_destroy(ctx), "tpmc_destroy")


def tpmc_set_stream(ctx, stream=None):
    handle = None
    if stream is not None:
        handle = ctypes.c_void_p(stream.cuda_stream if hasattr(stream, "cuda_stream") else int(stream))
    _check(lib().tpmc_set_stream(ctx, handle), "tpmc_set_stream", ctx)


def tpmc_last_error(ctx=None) -> str:
    m = lib().tpmc_last_error(ctx)
    return m.decode() if m else ""


def tpmc_memory_info(ctx) -> dict:
    used, budget, n = ctypes.c_size_t(), ctypes.c_size_t(), ctypes.c_uint64()
    _check(lib().tpmc_memory_info(ctx, ctypes.byref(used), ctypes.byref(budget), ctypes.byref(n)),
           "tpmc_memory_info", ctx)
    return {"used": used.value, "budget": budget.value, "n_allocs": n.value}


def tpmc_set_counters(ctx, enable: bool):
    _check(lib().tpmc_set_counters(ctx, 1 if enable else 0), "tpmc_set_counters", ctx)


def tpmc_mesh_load(ctx, xyz, tri) -> int:
    X = np.ascontiguousarray(np.asarray(xyz, dtype=np.float64).reshape(-1, 3))
    T = np.ascontiguousarray(np.asarray(tri, dtype=np.uint32).reshape(-1, 3))
    out = ctypes.c_uint32()
    _check(lib().tpmc_mesh_load(ctx, _pd(X), X.shape[0], _pu32(T), T.shape[0], ctypes.byref(out)),
           "tpmc_mesh_load", ctx)
    return out.value


def tpmc_mesh_unload(ctx, mesh: int):
    _check(lib().tpmc_mesh_unload(ctx, int(mesh)), "tpmc_mesh_unload", ctx)


def tpmc_mesh_info(ctx, mesh: int) -> dict:
    s = tpmc_mesh_stats()
    _check(lib().tpmc_mesh_info(ctx, int(mesh), ctypes.byref(s)), "tpmc_mesh_info", ctx)
    return {n: (list(getattr(s, n)) if isinstance(getattr(s, n), ctypes.Array) else getattr(s, n))
            for n, _ in s._fields_}


def make_params(*, n, T_inf, m, V, dir, T_W, eps_diffuse, A_ref, ref_point=(0, 0, 0), r_cv=0.0,
                center=(0, 0, 0), max_bounces=64, precision=TPMC_FP32, seed=0, stream_id=0,
                want_panels=False, cv_kind=TPMC_CV_SPHERE, box_lo=(0, 0, 0), box_hi=(0, 0, 0),
                l_ref=0.0, gsi_model=TPMC_GSI_MAXWELL, alpha_n=1.0, sigma_t=1.0) -> tpmc_params:
    p = tpmc_params()
    p.n, p.T_inf, p.m, p.V = float(n), float(T_inf), float(m), float(V)
    p.dir[:] = [float(x) for x in dir]
    p.T_W, p.eps_diffuse, p.A_ref = float(T_W), float(eps_diffuse), float(A_ref)
    p.ref_point[:] = [float(x) for x in ref_point]
    p.r_cv = float(r_cv)
    p.center[:] = [float(x) for x in center]
    p.max_bounces, p.precision, p.seed = int(max_bounces), int(precision), int(seed)
    p.stream_id, p.want_panels = int(stream_id), int(bool(want_panels))
    p.cv_kind = int(cv_kind)
    p.box_lo[:] = [float(x) for x in box_lo]
    p.box_hi[:] = [float(x) for x in box_hi]
    p.l_ref = float(l_ref)
    p.gsi_model, p.alpha_n, p.sigma_t = int(gsi_model), float(alpha_n), float(sigma_t)
    return p


def tpmc_trace(ctx, mesh: int, params: tpmc_params, N: int) -> dict:
    r = tpmc_result()
    _check(lib().tpmc_trace(ctx, int(mesh), ctypes.byref(params), int(N), ctypes.byref(r)), "tpmc_trace", ctx)
    return r.as_dict()


def tpmc_trace_records(ctx, mesh: int, params: tpmc_params, N: int, K: int = 16):
    rec = {
        "pos": np.zeros((N, 3)), "vel": np.zeros((N, 3)), "dv": np.zeros((N, 3)),
        "n_hits": np.zeros(N, np.uint32), "truncated": np.zeros(N, np.uint32),
        "tri": np.full((N, K), 0xFFFFFFFF, np.uint32),
    }
    R = tpmc_records(_pd(rec["pos"]), _pd(rec["vel"]), _pd(rec["dv"]), _pu32(rec["n_hits"]),
                     _pu32(rec["truncated"]), _pu32(rec["tri"]), int(K))
    r = tpmc_result()
    _check(lib().tpmc_trace_records(ctx, int(mesh), ctypes.byref(params), int(N), ctypes.byref(R), ctypes.byref(r)),
           "tpmc_trace_records", ctx)
    return r.as_dict(), rec


def tpmc_panels(ctx, query_id: int, n_tri: int):
    p = np.zeros(n_tri)
    s = np.zeros(n_tri)
    _check(lib().tpmc_panels(ctx, int(query_id), _pd(p), _pd(s), int(n_tri)), "tpmc_panels", ctx)
    return p, s


def tpmc_panel_sums(ctx, query_id: int, n_tri: int):
    q = np.zeros((n_tri, 3), dtype=np.int64)
    _check(lib().tpmc_panel_sums(ctx, int(query_id), q.ctypes.data_as(ctypes.c_void_p), int(n_tri)),
           "tpmc_panel_sums", ctx)
    return q


def tpmc_sweep(ctx, mesh: int, base: tpmc_params, dirs, S, N_each: int):
    D = None if dirs is None else np.ascontiguousarray(np.asarray(dirs, dtype=np.float64).reshape(-1, 3))
    Sv = None if S is None else np.ascontiguousarray(np.asarray(S, dtype=np.float64).reshape(-1))
    K = D.shape[0] if D is not None else Sv.shape[0]
    out = (tpmc_result * K)()
    _check(lib().tpmc_sweep(ctx, int(mesh), ctypes.byref(base), _pd(D), _pd(Sv), K, int(N_each), out),
           "tpmc_sweep", ctx)
    return [o.as_dict() for o in out]


def tpmc_sweep_device(ctx, mesh: int, base: tpmc_params, d_dirs, d_S, K: int, N_each: int, d_out):
    _check(lib().tpmc_sweep_device(ctx, int(mesh), ctypes.byref(base), _ptr(d_dirs), _ptr(d_S), int(K),
                                   int(N_each), _ptr(d_out)), "tpmc_sweep_device", ctx)


def tpmc_sweep_noalloc(ctx, mesh: int, base: tpmc_params, dirs, S, N_each: int):
    """The sweep without any allocation by the library (at most 64 items; see include/tpmc.h)."""
    D = None if dirs is None else np.ascontiguousarray(np.asarray(dirs, dtype=np.float64).reshape(-1, 3))
    Sv = None if S is None else np.ascontiguousarray(np.asarray(S, dtype=np.float64).reshape(-1))
    K = D.shape[0] if D is not None else Sv.shape[0]
    out = (tpmc_result * K)()
    _check(lib().tpmc_sweep_noalloc(ctx, int(mesh), ctypes.byref(base), _pd(D), _pd(Sv), K, int(N_each), out),
           "tpmc_sweep_noalloc", ctx)
    return [o.as_dict() for o in out]


RESULT_BYTES = ctypes.sizeof(tpmc_result)


def results_from_bytes(buf: bytes, K: int):
    arr = (tpmc_result * K).from_buffer_copy(buf)
    return [a.as_dict() for a in arr]


def tpmc_submit(ctx, mesh: int, params: tpmc_params, N: int) -> int:
    q = ctypes.c_uint64()
    _check(lib().tpmc_submit(ctx, int(mesh), ctypes.byref(params), int(N), ctypes.byref(q)), "tpmc_submit", ctx)
    return q.value


def tpmc_poll(ctx, query_id: int, timeout_ms: int = -1):
    """Returns the result dict, or None when the query has not finished (ETIMEOUT)."""
    r = tpmc_result()
    st = lib().tpmc_poll(ctx, int(query_id), int(timeout_ms), ctypes.byref(r))
    if st == TPMC_ETIMEOUT:
        return None
    _check(st, "tpmc_poll", ctx)
    return r.as_dict()


def tpmc_tune(ctx, mesh: int, params: tpmc_params, N_trial: int) -> dict:
    b = tpmc_launch()
    _check(lib().tpmc_tune(ctx, int(mesh), ctypes.byref(params), int(N_trial), ctypes.byref(b)), "tpmc_tune", ctx)
    return {n: getattr(b, n) for n, _ in b._fields_}


def tpmc_set_launch(ctx, block=None, blocks_per_sm=0, chunk=0, smem_nodes=0, refill_at=0, bvh_leaf=0, bvh_width=0):
    """block=None returns to automatic schedules (and the default BVH layout);
    block=0 with bvh_leaf / bvh_width sets only the BVH layout of later loads."""
    if block is None:
        _check(lib().tpmc_set_launch(ctx, None), "tpmc_set_launch", ctx)
        return
    b = tpmc_launch(int(block), int(blocks_per_sm), int(chunk), int(smem_nodes), int(refill_at), int(bvh_leaf),
                    int(bvh_width))
    _check(lib().tpmc_set_launch(ctx, ctypes.byref(b)), "tpmc_set_launch", ctx)


def tpmc_get_launch(ctx, mesh: int, precision: int = TPMC_FP32) -> dict:
    b = tpmc_launch()
    _check(lib().tpmc_get_launch(ctx, int(mesh), int(precision), ctypes.byref(b)), "tpmc_get_launch", ctx)
    return {n: getattr(b, n) for n, _ in b._fields_}


def tpmc_measure_ceilings(ctx) -> dict:
    """FP32 FMA rate (TFLOP/s) and L2 read bandwidth (GB/s) measured on the context's device."""
    f = ctypes.c_double()
    b = ctypes.c_double()
    _check(lib().tpmc_measure_ceilings(ctx, ctypes.byref(f), ctypes.byref(b)), "tpmc_measure_ceilings", ctx)
    return {"fp32_tflops": f.value, "l2_read_gbs": b.value}
