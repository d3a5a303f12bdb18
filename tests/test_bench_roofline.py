"""The bench's roofline arithmetic (no GPU): % roofline = particles/s over
min(B_L2 / bytes per particle, P_FP32 / flops per particle), with the work
counted per run, and every number of the reported object reproducible from
the object's own fields."""
import math

import bench

CEIL = {"l2_read_gbs": 19_000.0, "fp32_tflops": 70.0}


def _work(particles, hits, nodes, tris):
    return {"particles": particles, "hits": hits, "nodes": nodes, "tris": tris}


def _recompute(r):
    """frac and achieved from the reported fields alone."""
    w, u, c = r["work"], r["units"], r["ceilings"]
    n = w["particles"]
    node_bytes = sum(b["node_bytes"] for b in r["bvh"]) / len(r["bvh"])
    width = r["bvh"][0]["width"]
    flops = (u["flops_per_child_box"] * width * w["nodes"] + u["flops_per_tri_test"] * w["tris"] +
             u["flops_per_particle"] * n + u["flops_per_hit"] * w["hits"])
    l2 = node_bytes * w["nodes"] + u["bytes_per_tri_test"] * w["tris"]
    rate = r["particles_per_s"]
    b_l2 = c["l2_read_gbs"] * 1e9 / (l2 / n)
    b_fp = c["fp32_tflops"] * 1e12 / (flops / n)
    return rate / min(b_l2, b_fp), ("l2" if b_l2 <= b_fp else "fp32"), l2 / n, flops / n


def test_l2_binds_on_traversal_heavy_work():
    # 3.84e9 particles with about 4.2 node visits and 1.1 triangle tests each (the sweep's counts)
    w = _work(3_840_000_000, 1_489_227_003, 16_109_142_821, 4_149_353_810)
    r = bench.roofline_of([(w, 32, 2)], 0.40, CEIL)
    frac, bound, bpp, fpp = _recompute(r)
    assert r["bound"] == bound == "l2"
    assert r["unit"] == "GB/s" and r["peak"] == CEIL["l2_read_gbs"]
    assert math.isclose(r["frac"], frac, rel_tol=1e-12)
    assert math.isclose(r["bytes_per_particle"], bpp, rel_tol=1e-12)
    assert math.isclose(r["flops_per_particle"], fpp, rel_tol=1e-12)
    # achieved = algorithmic bytes per second; frac = achieved / peak when L2 binds
    assert math.isclose(r["achieved"], r["particles_per_s"] * bpp / 1e9, rel_tol=1e-12)
    assert math.isclose(r["frac"], r["achieved"] / r["peak"], rel_tol=1e-12)
    assert math.isclose(r["frac"], r["l2_frac"], rel_tol=1e-12)
    # the hand count: 32 B per node visit and 48 B per triangle test
    assert math.isclose(bpp, (32 * 16_109_142_821 + 48 * 4_149_353_810) / 3.84e9, rel_tol=1e-12)


def test_fp32_binds_when_the_work_is_arithmetic():
    # no traversal at all: only seeding and hits, so the FP32 bound is the lower one
    w = _work(1_000_000, 1_000_000, 1, 0)
    r = bench.roofline_of([(w, 32, 2)], 1e-3, CEIL)
    frac, bound, _, fpp = _recompute(r)
    assert r["bound"] == bound == "fp32"
    assert r["unit"] == "TFLOP/s" and r["peak"] == CEIL["fp32_tflops"]
    assert math.isclose(r["frac"], frac, rel_tol=1e-12)
    assert math.isclose(r["achieved"], r["particles_per_s"] * fpp / 1e12, rel_tol=1e-12)
    assert math.isclose(r["frac"], r["fp32_frac"], rel_tol=1e-12)


def test_wide_nodes_count_every_child_box():
    w = _work(1_000_000, 100_000, 2_000_000, 500_000)
    r2 = bench.roofline_of([(w, 32, 2)], 1e-3, CEIL)
    r8 = bench.roofline_of([(w, 80, 8)], 1e-3, CEIL)
    # an 8-wide visit tests 8 boxes and reads 80 bytes
    assert math.isclose(r8["flops_per_particle"] - r2["flops_per_particle"],
                        bench.FLOPS_PER_CHILD_BOX * 6 * 2.0, rel_tol=1e-12)
    assert math.isclose(r8["bytes_per_particle"] - r2["bytes_per_particle"], 48 * 2.0, rel_tol=1e-12)


def test_parts_add_before_dividing():
    a = _work(1_000_000, 10, 4_000_000, 1_000_000)
    b = _work(3_000_000, 20, 1_000_000, 500_000)
    r = bench.roofline_of([(a, 32, 2), (b, 32, 2)], 2e-3, CEIL)
    assert r["work"] == _work(4_000_000, 30, 5_000_000, 1_500_000)
    assert math.isclose(r["node_visits_per_particle"], 5_000_000 / 4_000_000, rel_tol=1e-12)
    assert math.isclose(r["particles_per_s"], 4_000_000 / 2e-3, rel_tol=1e-12)


def test_work_of_sums_the_result_counters():
    res = [{"n_particles": 5, "n_hits": 2, "n_node_visits": 11, "n_tri_tests": 3},
           {"n_particles": 7, "n_hits": 0, "n_node_visits": 4, "n_tri_tests": 1}]
    assert bench.work_of(res) == _work(12, 2, 15, 4)


def test_groups_are_the_sweep_workload():
    gs = bench.groups()
    assert [(g["shape"], g["eps"]) for g in gs] == [("plate", 0.0), ("plate", 1.0), ("cylinder", 0.0),
                                                   ("cylinder", 1.0)]
    assert all(len(g["dirs"]) == len(g["S"]) == 96 for g in gs)
    assert sorted(set(float(s) for s in gs[0]["S"])) == [2.0, 5.0, 10.0]
