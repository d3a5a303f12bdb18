"""tpmc_sweep_noalloc, the sweep for callers that may not allocate device memory
after start-up (real-time loops, framework-owned memory pools, fixed
footprints), against tpmc_sweep on the same inputs.

The no-allocation calls run first on a fresh context, so that no scratch
grown by an earlier allocating call could hide an allocation of theirs; the
context's allocation count and bytes must not move across them.  They run
twice in a row (the second must not inherit the first's sums from the shared
scratch), with speed ratios given and with speed ratios taken from the base
query (h_S = NULL), and once with the directions taken from it (h_dirs = NULL).

This file is collected last on purpose: a failure here leaves every other
test already run."""
import numpy as np
import pytest

from tests.parity_util import cd_close
from tpmc_inputs import meshes as M
from tpmc_inputs import workloads as W

pytestmark = pytest.mark.gpu


def _same(got, ref, N_each):
    assert len(got) == len(ref)
    for a, b in zip(got, ref):
        assert a["status"] == 0 and a["ms"] > 0
        assert a["n_particles"] == N_each
        assert cd_close(a["CD"], b["CD"], b["CD_sigma"])
        # same Philox streams and exact integer sums: the totals agree bit for bit
        assert a["sum_dv_q"] == b["sum_dv_q"] and a["n_hits"] == b["n_hits"]
        assert a["CD_sigma"] == b["CD_sigma"]
        np.testing.assert_allclose(a["torque"], b["torque"], rtol=1e-12, atol=0)


def test_noalloc_sweep_matches_the_allocating_sweep_twice():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1312_3691_gb300.build import build

    build()
    from paper_1312_3691_gb300 import tpmc as T

    ctx = T.tpmc_create(0)
    try:
        xyz, tri = M.satellite(60_000)
        mesh = T.tpmc_mesh_load(ctx, xyz, tri)
        case = W.satellite_case(N=1)
        dirs = W.attitude_grid(4, 4)[:12]
        S = np.linspace(4.0, 11.0, 12)
        base = T.make_params(**case["params"], stream_id=500)
        N_each = 150_000
        before = T.tpmc_memory_info(ctx)
        got = [T.tpmc_sweep_noalloc(ctx, mesh, base, dirs, S, N_each) for _ in range(2)]
        got_noS = [T.tpmc_sweep_noalloc(ctx, mesh, base, dirs[:5], None, N_each) for _ in range(2)]
        got_nodir = T.tpmc_sweep_noalloc(ctx, mesh, base, None, S[:4], N_each)
        after = T.tpmc_memory_info(ctx)
        assert after["n_allocs"] == before["n_allocs"] and after["used"] == before["used"], (before, after)
        ref = T.tpmc_sweep(ctx, mesh, base, dirs, S, N_each)
        ref_noS = T.tpmc_sweep(ctx, mesh, base, dirs[:5], None, N_each)
        ref_nodir = T.tpmc_sweep(ctx, mesh, base, None, S[:4], N_each)
        for g in got:
            _same(g, ref, N_each)
        for g in got_noS:
            _same(g, ref_noS, N_each)
            assert all(abs(r["S"] - 7.0) < 1e-12 for r in g)
        # without directions every item flies along the base query's direction
        _same(got_nodir, ref_nodir, N_each)
        assert all(abs(r["S"] - x) < 1e-12 for r, x in zip(got_nodir, S[:4]))
        with pytest.raises(T.TpmcError) as e:
            T.tpmc_sweep_noalloc(ctx, mesh, base, W.attitude_grid(9, 8), np.full(72, 5.0), 10)
        assert e.value.status == T.TPMC_EINVAL
        # an item whose set-up rejects its speed ratio reports it in its own status, as tpmc_sweep does
        bad = T.tpmc_sweep_noalloc(ctx, mesh, base, dirs[:3], np.array([5.0, 80.0, 6.0]), 1000)
        assert [r["status"] for r in bad] == [0, T.TPMC_EINVAL, 0]
        T.tpmc_mesh_unload(ctx, mesh)
    finally:
        T.tpmc_destroy(ctx)
