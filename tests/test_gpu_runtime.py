"""Runtime behaviour through the C ABI on the GPU: the launch autotuner, serving
time-outs and validation, and schedule independence of tuned launches."""
import numpy as np
import pytest

from tpmc_inputs import meshes as M
from tpmc_inputs import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def T():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1312_3691_gb300.build import build

    build()
    from paper_1312_3691_gb300 import tpmc

    return tpmc


@pytest.fixture(scope="module")
def ctx(T):
    c = T.tpmc_create(0)
    yield c
    T.tpmc_destroy(c)


def test_tune_picks_a_valid_schedule_that_keeps_results(T, ctx):
    xyz, tri = M.cylinder()
    mesh = T.tpmc_mesh_load(ctx, xyz, tri)
    try:
        p = T.make_params(**W.base_state(S=5.0), dir=(1.0, 0.2, -0.5), eps_diffuse=1.0, A_ref=2.0, seed=77)
        before = T.tpmc_trace(ctx, mesh, p, 500_000)
        best = T.tpmc_tune(ctx, mesh, p, 200_000)
        assert best["block"] in (64, 128, 256) and best["blocks_per_sm"] >= 1
        assert best["bvh_width"] in (2, 4, 8)
        # the mesh now has the chosen layout, and later loads of its size class get it too
        assert T.tpmc_mesh_info(ctx, mesh)["bvh_width"] == best["bvh_width"]
        got = T.tpmc_get_launch(ctx, mesh, T.TPMC_FP32)
        assert got["block"] == best["block"] and got["smem_nodes"] == best["smem_nodes"]
        assert got["bvh_width"] == best["bvh_width"]
        after = T.tpmc_trace(ctx, mesh, p, 500_000)
        assert after["sum_dv_q"] == before["sum_dv_q"] and after["n_hits"] == before["n_hits"]
        mesh2 = T.tpmc_mesh_load(ctx, xyz, tri)
        assert T.tpmc_mesh_info(ctx, mesh2)["bvh_width"] == best["bvh_width"]
        T.tpmc_mesh_unload(ctx, mesh2)
    finally:
        T.tpmc_mesh_unload(ctx, mesh)


def test_poll_times_out_then_returns_the_result(T, ctx):
    xyz, tri = M.satellite(60_000)
    mesh = T.tpmc_mesh_load(ctx, xyz, tri)
    try:
        case = W.satellite_case(N=1)
        h = T.tpmc_submit(ctx, mesh, T.make_params(**case["params"]), 300_000_000)
        assert T.tpmc_poll(ctx, h, 0) is None  # ETIMEOUT: still running
        r = T.tpmc_poll(ctx, h, -1)
        assert r["n_particles"] == 300_000_000 and r["status"] == 0
        # a short query submitted alone matches the direct trace
        h2 = T.tpmc_submit(ctx, mesh, T.make_params(**case["params"]), 123_457)
        r2 = T.tpmc_poll(ctx, h2, -1)
        d = T.tpmc_trace(ctx, mesh, T.make_params(**case["params"]), 123_457)
        assert r2["sum_dv_q"] == d["sum_dv_q"]
    finally:
        T.tpmc_mesh_unload(ctx, mesh)


def test_submit_validates_like_trace(T, ctx):
    xyz, tri = M.icosphere(1)
    mesh = T.tpmc_mesh_load(ctx, xyz, tri)
    good = dict(**W.base_state(), dir=(0, 0, 1), eps_diffuse=1.0, A_ref=1.0, r_cv=1.5)
    try:
        with pytest.raises(T.TpmcError) as e:
            T.tpmc_submit(ctx, mesh, T.make_params(**{**good, "eps_diffuse": -0.1}), 100)
        assert e.value.status == T.TPMC_EINVAL
        with pytest.raises(T.TpmcError) as e:
            T.tpmc_submit(ctx, mesh + 1000, T.make_params(**good), 100)
        assert e.value.status == T.TPMC_ENOTFOUND
        with pytest.raises(T.TpmcError) as e:
            T.tpmc_poll(ctx, 987654321, 0)
        assert e.value.status == T.TPMC_ENOTFOUND
        # a mesh with queries in flight cannot be unloaded
        h = T.tpmc_submit(ctx, mesh, T.make_params(**good), 50_000_000)
        with pytest.raises(T.TpmcError) as e:
            T.tpmc_mesh_unload(ctx, mesh)
        assert e.value.status == T.TPMC_EBUSY
        assert T.tpmc_poll(ctx, h, -1)["status"] == 0
    finally:
        T.tpmc_mesh_unload(ctx, mesh)


def test_panels_through_serving(T, ctx):
    xyz, tri = M.icosphere(2)
    mesh = T.tpmc_mesh_load(ctx, xyz, tri)
    try:
        p = T.make_params(**W.base_state(S=4.0), dir=(0, 1.0, 0.2), eps_diffuse=0.7, A_ref=np.pi, r_cv=1.4, seed=9,
                          max_bounces=8, want_panels=True)
        direct = T.tpmc_trace(ctx, mesh, p, 200_000)
        pd, sd = T.tpmc_panels(ctx, direct["query_id"], tri.shape[0])
        h = T.tpmc_submit(ctx, mesh, p, 200_000)
        r = T.tpmc_poll(ctx, h, -1)
        ps, ss = T.tpmc_panels(ctx, r["query_id"], tri.shape[0])
        np.testing.assert_array_equal(pd, ps)
        np.testing.assert_array_equal(sd, ss)
    finally:
        T.tpmc_mesh_unload(ctx, mesh)


def test_measured_ceilings_are_plausible_for_the_device(T, ctx):
    """The FMA loop cannot beat the SM count x 128 FP32 lanes x 2 flops at the
    maximum clock by more than the packed-FMA factor, and the L2 stream must be
    faster than a DRAM copy yet below the L1 rate of all SMs."""
    import torch

    props = torch.cuda.get_device_properties(0)
    c = T.tpmc_measure_ceilings(ctx)
    lanes_peak = props.multi_processor_count * 128 * 2 * 2.2e9 / 1e12
    assert 0.2 * lanes_peak < c["fp32_tflops"] < 2.05 * lanes_peak, (c, lanes_peak)
    assert 2_000.0 < c["l2_read_gbs"] < props.multi_processor_count * 128 * 2.2, c
    assert T.lib().tpmc_measure_ceilings(ctx, None, None) == T.TPMC_EINVAL


def test_sweep_rejects_more_items_than_a_queue_slot_can_name(T, ctx):
    """A queued particle names its query in 24 bits, so a sweep holds at most
    2^24 items; one more is rejected before any work is enqueued."""
    import ctypes

    import torch

    xyz, tri = M.plate(1.0)
    mesh = T.tpmc_mesh_load(ctx, xyz, tri)
    try:
        p = T.make_params(**W.base_state(S=5.0), dir=(0.0, 0.0, 1.0), eps_diffuse=1.0, A_ref=1.0)
        out = torch.zeros(T.RESULT_BYTES, dtype=torch.uint8, device="cuda")
        st = T.lib().tpmc_sweep_device(ctx, mesh, ctypes.byref(p), None, None, (1 << 24) + 1, 1,
                                       ctypes.c_void_p(out.data_ptr()))
        assert st == T.TPMC_EINVAL
        assert "2^24" in T.lib().tpmc_last_error(ctx).decode()
    finally:
        T.tpmc_mesh_unload(ctx, mesh)
