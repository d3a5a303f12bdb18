"""Helpers for comparing the CUDA path with the FP64 oracle on the same Philox streams."""
import numpy as np

# A hit within this distance (metres) of a triangle edge, or at a grazing
# angle, may legitimately land on the neighbouring triangle in float32; the
# particle's path is compared only up to such a hit.  The float32 position
# error grows with every bounce, and along a ray meeting the surface at
# incidence cosine cos it becomes an error of (error / cos) in the hit point,
# so hit b (0-based) counts as near an edge when edge * cos < EDGE_M (1 + b).
EDGE_M = 1e-5
GRAZING_COS = 1e-4


def compare_paths(gpu_rec: dict, orc_rec: dict, K: int):
    """Returns (identical, explained, unexplained) boolean masks over particles.

    identical: same hit count and same triangle at every recorded bounce.
    explained: differs, but only after (or at) an oracle hit that is near an
    edge or grazing.
    """
    nh_g = gpu_rec["n_hits"].astype(np.int64)
    nh_o = orc_rec["n_hits"].astype(np.int64)
    tg = gpu_rec["tri"]
    to = orc_rec["tri"]
    n = nh_o.shape[0]
    identical = (nh_g == nh_o) & (tg == to).all(axis=1)
    explained = np.zeros(n, dtype=bool)
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
        upto = min(first + 1, K, int(nh_o[i]) if nh_o[i] > 0 else 0)
        # the divergence is explained by a near-edge oracle hit at or before it,
        # or (when the oracle's path is the shorter one) by its last hit
        if upto > 0 and near[i, :upto].any():
            explained[i] = True
        elif nh_o[i] > 0 and nh_o[i] <= K and near[i, :int(nh_o[i])].any():
            explained[i] = True
    return identical, explained, ~identical & ~explained


def cd_close(gpu_cd, orc_cd, orc_sigma, gpu_sigma=0.0):
    """The stated tolerance: 1e-4 relative plus three standard errors."""
    return abs(gpu_cd - orc_cd) <= 1e-4 * abs(orc_cd) + 3.0 * max(orc_sigma, gpu_sigma)
