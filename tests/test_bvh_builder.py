"""The BVH builder on the host (CPU only): closest hits through the built tree
equal brute force over all triangles, ray by ray.

tests/bvh_check.cpp compiles the library's own builder (bvh.cpp) and walks the
tree it lays out for the GPU.  The rays aim at the places where the spatial
splits cut triangles: the fan centres that close the cylinder and the
hemisphere's pole, vertices and edge midpoints (ties between neighbours),
axis-parallel directions, and a soup of overlapping slivers.
"""
import os
import subprocess

import numpy as np
import pytest

from tpmc_inputs import meshes as M

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_1312_3691_gb300", "csrc")
CUDA_INC = os.path.join(os.environ.get("CUDA_HOME", "/usr/local/cuda"), "include")


@pytest.fixture(scope="module")
def checker(tmp_path_factory):
    exe = tmp_path_factory.mktemp("bvh") / "bvh_check"
    subprocess.check_call(["g++", "-O2", "-std=c++17", "-I", CSRC, "-I", CUDA_INC,
                           os.path.join(ROOT, "tests", "bvh_check.cpp"), os.path.join(CSRC, "bvh.cpp"),
                           "-o", str(exe)])
    return exe


def _rays(xyz, tri, rng, n_random=6000, n_vertex=1500, n_edge=1500, n_axis=1000):
    """Ray origins outside the mesh's bounding sphere, aimed at random points of
    the bounding box, at vertices, at edge midpoints, and along the axes."""
    c = 0.5 * (xyz.min(0) + xyz.max(0))
    R = np.sqrt(((xyz - c) ** 2).sum(1)).max() * 1.5 + 1e-3
    lo, hi = xyz.min(0), xyz.max(0)

    def origins(n):
        v = rng.normal(size=(n, 3))
        return c + R * v / np.linalg.norm(v, axis=1, keepdims=True)

    out = []
    o = origins(n_random)
    out.append(np.hstack([o, lo + rng.random((n_random, 3)) * (hi - lo) - o]))
    used = np.unique(tri)
    tv = xyz[rng.choice(used, size=n_vertex)]
    o = origins(n_vertex)
    out.append(np.hstack([o, tv - o]))
    e = rng.integers(0, len(tri), size=n_edge)
    k = rng.integers(0, 3, size=n_edge)
    mid = 0.5 * (xyz[tri[e, k]] + xyz[tri[e, (k + 1) % 3]])
    o = origins(n_edge)
    out.append(np.hstack([o, mid - o]))
    axis = rng.integers(0, 3, size=n_axis)
    sign = rng.choice([-1.0, 1.0], size=n_axis)
    d = np.zeros((n_axis, 3))
    d[np.arange(n_axis), axis] = sign
    tgt = np.where(rng.random((n_axis, 1)) < 0.5, xyz[rng.choice(used, size=n_axis)],
                   lo + rng.random((n_axis, 3)) * (hi - lo))
    out.append(np.hstack([tgt - 2.0 * R * d, d]))
    return np.vstack(out)


def _check(checker, tmp_path, xyz, tri, rays, leaf=4, width=2):
    xyz = np.ascontiguousarray(xyz, np.float64)
    tri = np.ascontiguousarray(tri, np.uint32)
    mesh = tmp_path / "mesh.bin"
    ray = tmp_path / "rays.bin"
    mesh.write_bytes(np.array([len(xyz), len(tri)], np.uint32).tobytes() + xyz.tobytes() + tri.tobytes())
    ray.write_bytes(np.array([len(rays)], np.uint32).tobytes() + np.ascontiguousarray(rays, np.float64).tobytes())
    out = subprocess.check_output([str(checker), str(mesh), str(ray), str(leaf), str(width)], text=True).split()
    keys = ["rays", "mismatches", "hits", "n_tri", "n_refs", "n_nodes", "depth", "leaf_max", "unreferenced",
            "oversized", "exposed", "wrong_exposed", "width", "node_bytes", "bad_index"]
    return dict(zip(keys, (int(x) for x in out)))


def _fan(n=256, radius=0.5):
    a = 2 * np.pi * np.arange(n) / n
    xyz = np.vstack([[0.0, 0.0, 0.0], np.c_[radius * np.cos(a), radius * np.sin(a), np.zeros(n)]])
    tri = np.c_[np.zeros(n, int), 1 + np.arange(n), 1 + (np.arange(n) + 1) % n]
    return xyz, tri


def _soup(rng, n=600):
    """Overlapping random triangles, slivers, duplicates and zero-area ones."""
    xyz = rng.random((3 * n, 3))
    tri = np.arange(3 * n).reshape(n, 3)
    xyz[3 * np.arange(0, n, 7) + 2] = xyz[3 * np.arange(0, n, 7) + 1] + 1e-6 * rng.random((len(range(0, n, 7)), 3))
    xyz = np.vstack([xyz, xyz[:30]])                       # duplicated triangles
    tri = np.vstack([tri, 3 * n + np.arange(30).reshape(10, 3)])
    xyz = np.vstack([xyz, [[0.2, 0.2, 0.2], [0.4, 0.4, 0.4], [0.6, 0.6, 0.6]]])
    tri = np.vstack([tri, [[len(xyz) - 3, len(xyz) - 2, len(xyz) - 1]]])  # collinear: zero area
    return xyz, tri


CASES = {
    "cylinder": lambda rng: M.cylinder(),
    "hemisphere": lambda rng: M.hemisphere_shell(),
    "icosphere": lambda rng: M.icosphere(3, 1.0),
    "satellite": lambda rng: M.satellite(8_000),
    "fan": lambda rng: _fan(),
    "soup": _soup,
    "plate": lambda rng: M.plate(),
}


@pytest.mark.parametrize("width", [2, 4, 8])
@pytest.mark.parametrize("name", sorted(CASES))
def test_tree_closest_hits_equal_brute_force(checker, tmp_path, name, width):
    """Binary and compressed wide layouts (the wide walk decodes the 8-bit
    child boxes as the GPU does)."""
    rng = np.random.default_rng(sorted(CASES).index(name) + 11)
    xyz, tri = CASES[name](rng)
    xyz, tri = np.asarray(xyz, float), np.asarray(tri)
    rays = _rays(xyz, tri, np.random.default_rng(17))
    r = _check(checker, tmp_path, xyz, tri, rays, width=width)
    assert r["width"] == width and r["node_bytes"] == {2: 32, 4: 64, 8: 80}[width], r
    assert r["mismatches"] == 0 and r["bad_index"] == 0, r
    assert r["unreferenced"] == 0 and r["oversized"] == 0, r
    assert r["hits"] > 0.2 * r["rays"], r
    assert len(tri) - 1 <= r["n_refs"] <= 1.5 * len(tri) + 1, r
    assert r["wrong_exposed"] == 0, r
    assert r["exposed"] == EXPOSED[name](len(tri)), r


# Exposed triangle sides (the whole mesh behind the side's plane): one side of
# every face of a closed convex body or of the hemisphere's outside, both sides
# of the flat plate and of the flat fan; of the satellite, the bus faces that
# neither a panel nor the dish stands in front of; none of the soup.
EXPOSED = {
    "cylinder": lambda n: n, "icosphere": lambda n: n, "hemisphere": lambda n: n,
    "plate": lambda n: 2 * n, "fan": lambda n: 2 * n, "soup": lambda n: 0,
    "satellite": lambda n: _satellite_exposed(),
}


def _satellite_exposed():
    """Sides of the satellite(8000) bus faces with nothing in front, counted
    by brute force in numpy: independent of the builder."""
    xyz, tri = M.satellite(8_000)
    xyz, tri = np.asarray(xyz, float), np.asarray(tri)
    a, b, c = (xyz[tri[:, k]] for k in range(3))
    n = np.cross(b - a, c - a)
    n /= np.linalg.norm(n, axis=1, keepdims=True)
    count = 0
    for i in range(len(tri)):
        d = (xyz - a[i]) @ n[i]
        count += int(d.max() <= 1e-12) + int(d.min() >= -1e-12)
    return count


def test_spatial_splits_cut_the_fans(checker, tmp_path):
    """The cylinder's caps and a bare fan get extra references; each stays
    within the budget of half a reference per triangle."""
    rng = np.random.default_rng(3)
    for xyz, tri in (M.cylinder(), _fan()):
        xyz, tri = np.asarray(xyz, float), np.asarray(tri)
        r = _check(checker, tmp_path, xyz, tri, _rays(xyz, tri, rng, 200, 50, 50, 50))
        assert r["mismatches"] == 0
        assert len(tri) < r["n_refs"] <= 1.5 * len(tri) + 1, r


@pytest.mark.parametrize("width", [2, 8])
@pytest.mark.parametrize("leaf", [1, 2, 8])
def test_leaf_sizes(checker, tmp_path, leaf, width):
    """Wide layouts keep leaves of at most 4 references whatever the binary
    leaf size: larger binary leaves are split into leaves with the same box,
    and subtrees of at most 4 references are merged into one leaf."""
    xyz, tri = M.cylinder()
    xyz, tri = np.asarray(xyz, float), np.asarray(tri)
    r = _check(checker, tmp_path, xyz, tri, _rays(xyz, tri, np.random.default_rng(5), 3000, 500, 500, 500), leaf,
               width)
    assert r["mismatches"] == 0 and r["unreferenced"] == 0, r
    assert r["leaf_max"] <= (max(leaf, 1) if width == 2 else 4) or r["depth"] >= 40, r


def test_wide_trees_are_shallow(checker, tmp_path):
    """Collapsing the binary tree into 8-wide nodes at least halves its depth
    and divides its node count by more than five; the 4-wide tree lies between."""
    xyz, tri = M.satellite(60_000)
    xyz, tri = np.asarray(xyz, float), np.asarray(tri)
    rays = _rays(xyz, tri, np.random.default_rng(9), 400, 100, 100, 100)
    r2, r4, r8 = (_check(checker, tmp_path, xyz, tri, rays, width=w) for w in (2, 4, 8))
    for r in (r2, r4, r8):
        assert r["mismatches"] == 0, r
    assert r8["depth"] < r4["depth"] < r2["depth"] and 2 * r8["depth"] <= r2["depth"] + 1, (r2, r4, r8)
    assert r8["n_nodes"] * 5 < r2["n_nodes"] and r8["n_nodes"] < r4["n_nodes"] < r2["n_nodes"], (r2, r4, r8)
    assert r2["n_refs"] == r4["n_refs"] == r8["n_refs"]
    print({w: (r["depth"], r["n_nodes"]) for w, r in ((2, r2), (4, r4), (8, r8))})
