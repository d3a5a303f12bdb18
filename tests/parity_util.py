"""Helpers for comparing the CUDA path with the FP64 oracle on the same Philox streams."""
import json
import os

import numpy as np

# A hit within this distance (metres) of a triangle edge, or at a grazing
# angle, may legitimately land on the neighbouring triangle in float32; the
# particle's path is compared only up to such a hit.  The float32 position
# error grows with every bounce, and along a ray meeting the surface at
# incidence cosine cos it becomes an error of (error / cos) in the hit point,
# so hit b (0-based) counts as near an edge when edge * cos < EDGE_M (1 + b).
EDGE_M = 1e-5
GRAZING_COS = 1e-4
# Largest share of particles whose paths may differ from the oracle's after a
# near-edge or grazing hit (the share the method's float error is expected to
# leave, well below 1e-3).
MAX_EXCUSED_SHARE = 1e-3


def compare_paths(gpu_rec: dict, orc_rec: dict, K: int):
    """Returns (identical, explained, unexplained, first) over particles.

    identical: same hit count and same triangle at every recorded bounce.
    explained: differs, but only after (or at) an oracle hit that is near an
    edge or grazing (the excused particles).
    first: the bounce at which the two paths first differ (-1 when identical).
    """
    nh_g = gpu_rec["n_hits"].astype(np.int64)
    nh_o = orc_rec["n_hits"].astype(np.int64)
    tg = gpu_rec["tri"]
    to = orc_rec["tri"]
    n = nh_o.shape[0]
    identical = (nh_g == nh_o) & (tg == to).all(axis=1)
    explained = np.zeros(n, dtype=bool)
    first_div = np.full(n, -1, dtype=np.int64)
    bad = np.nonzero(~identical)[0]
    bounce = np.arange(orc_rec["edge"].shape[1])[None, :]
    near = (orc_rec["edge"] * orc_rec["cosi"] < EDGE_M * (1 + bounce)) | (orc_rec["cosi"] < GRAZING_COS)
    for i in bad:
        # first bounce where the paths differ
        lim = int(min(max(nh_g[i], nh_o[i]), K))
        first = lim
        for b in range(lim):
            if tg[i, b] != to[i, b]:
                first = b
                break
        if first == lim and nh_g[i] != nh_o[i]:
            first = min(int(min(nh_g[i], nh_o[i])), K - 1)
        first_div[i] = first
        upto = min(first + 1, K, int(nh_o[i]) if nh_o[i] > 0 else 0)
        # the divergence is explained by a near-edge oracle hit at or before it,
        # or (when the oracle's path is the shorter one) by its last hit
        if upto > 0 and near[i, :upto].any():
            explained[i] = True
        elif nh_o[i] > 0 and nh_o[i] <= K and near[i, :int(nh_o[i])].any():
            explained[i] = True
    return identical, explained, ~identical & ~explained, first_div


def path_stats(gpu_rec: dict, orc_rec: dict, K: int) -> dict:
    """Counts of identical, excused (near-edge) and unexplained particles, with
    the excused ones binned by the bounce at which their paths first differ."""
    ident, expl, unexpl, first = compare_paths(gpu_rec, orc_rec, K)
    n = int(len(ident))
    by_bounce = np.bincount(first[expl], minlength=K) if expl.any() else np.zeros(K, dtype=np.int64)
    return {"n": n, "identical": int(ident.sum()), "excused": int(expl.sum()),
            "excused_share": float(expl.sum()) / max(n, 1), "unexplained": int(unexpl.sum()),
            "excused_by_bounce": [int(x) for x in by_bounce[:K]],
            "hit_particles": int((orc_rec["n_hits"] > 0).sum()), "_identical_mask": ident}


def dv_parity(gpu_rec: dict, orc_rec: dict, ident: np.ndarray, vhat) -> dict:
    """Per-particle momentum differences of identical-path particles: relative
    error of each particle's summed dv (c_mp units), and of the drag sum
    sum(dv . Vhat) over those particles (the C_D they make)."""
    g = gpu_rec["dv"][ident]
    o = orc_rec["dv"][ident]
    mag = np.linalg.norm(o, axis=1)
    hit = mag > 0
    rel = np.linalg.norm(g - o, axis=1)[hit] / mag[hit]
    vh = np.asarray(vhat, dtype=np.float64)
    vh = vh / np.linalg.norm(vh)
    dg, do = float((g @ vh).sum()), float((o @ vh).sum())
    out = {"n": int(hit.sum()), "drag_rel": abs(dg - do) / max(abs(do), 1e-300)}
    if hit.any():
        out.update(median_rel=float(np.median(rel)), p99_rel=float(np.percentile(rel, 99)), max_rel=float(rel.max()))
    return out


def report(name: str, stats: dict) -> None:
    """Appends a test's parity figures to the JSON-lines file named by
    TPMC_PARITY_REPORT (when set), so that a run records what it excused."""
    path = os.environ.get("TPMC_PARITY_REPORT")
    if not path:
        return
    row = {"test": name, **{k: v for k, v in stats.items() if not k.startswith("_")}}
    with open(path, "a") as f:
        f.write(json.dumps(row) + "\n")


def cd_close(gpu_cd, orc_cd, orc_sigma, gpu_sigma=0.0):
    """The stated tolerance: 1e-4 relative plus three standard errors."""
    return abs(gpu_cd - orc_cd) <= 1e-4 * abs(orc_cd) + 3.0 * max(orc_sigma, gpu_sigma)
