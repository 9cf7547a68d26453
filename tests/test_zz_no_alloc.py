"""The allocation-free triangle dump (gp_debug_dump_tris_noalloc) against the allocating
one (gp_debug_dump_tris), called through the C ABI.

The allocation-free variant exists for callers that cannot allocate device memory at the
point of the call (a caching allocator already holding the free HBM, or a loop that cannot
take the synchronisation of cudaMalloc/cudaFree); its scratch is one fixed device array
shared by all calls, whose address is looked up when a handle is created.  This file sorts last so that a run that stops at the first failure
has already run every other test.
"""
import ctypes

import numpy as np
import pytest

import worldgen as wg
from gpu_common import sim_for

pytestmark = pytest.mark.gpu


def _dump(entry, sim, view, out, depth, cap):
    from paper_2606_19641_b300 import binding as b
    buf = np.zeros(max(cap, 1), b.TRI_DTYPE)
    n = ctypes.c_int64(-1)
    rc = getattr(b.lib(), entry)(sim._h, view, b._ptr(out), b._ptr(depth), buf.ctypes.data, cap,
                                 ctypes.byref(n), b._stream(None))
    b.check(rc)
    return buf[:min(n.value, cap)].copy(), n.value


def _sorted(t):
    return np.sort(t.view(np.dtype((np.void, t.dtype.itemsize))))


@pytest.mark.parametrize("name,n_worlds", [("uniform", 2), ("ragged", 6)])
def test_noalloc_dump_matches_allocating_dump_on_consecutive_calls(name, n_worlds):
    """Two calls in a row (and a third repeating the first view) give the allocating dump's
    records and images; the ragged batch runs the handle's work list of uneven worlds."""
    import torch
    wl = wg.WORKLOADS[name]
    worlds = wg.make_workload(wl, n_worlds=n_worlds)
    sim, cfg = sim_for(worlds, wl)
    for k in range(2):
        sim.step(torch.from_numpy(wg.actions(wl.seed, k, worlds.n_agents)).cuda())
    out_a, dep_a = sim.alloc_outputs()
    out_b, dep_b = sim.alloc_outputs()
    cap = 16384
    views = (3, min(40, sim.n_views - 1), 3)  # two views in a row, then the first again
    refs = {v: _dump("gp_debug_dump_tris", sim, v, out_a, dep_a, cap) for v in set(views)}
    torch.cuda.synchronize()
    for v in views:
        got, n_got = _dump("gp_debug_dump_tris_noalloc", sim, v, out_b, dep_b, cap)
        ref, n_ref = refs[v]
        assert n_ref > 100 and n_got == n_ref, "view %d: %d vs %d triangles" % (v, n_got, n_ref)
        assert np.array_equal(_sorted(got), _sorted(ref))
        torch.cuda.synchronize()
        assert torch.equal(out_a, out_b)
        if dep_a.dtype == torch.float32:
            assert torch.equal(dep_a.view(torch.int32), dep_b.view(torch.int32))
        else:
            assert torch.equal(dep_a.view(torch.int16), dep_b.view(torch.int16))


def test_noalloc_dump_counts_every_record_beyond_cap():
    """With 0 < cap < n, *n still counts every record produced while only cap of them are
    copied, and those are records of the full dump."""
    import torch
    wl = wg.WORKLOADS["uniform"]
    worlds = wg.make_workload(wl, n_worlds=2)
    sim, cfg = sim_for(worlds, wl)
    for k in range(2):
        sim.step(torch.from_numpy(wg.actions(wl.seed, k, worlds.n_agents)).cuda())
    out, dep = sim.alloc_outputs()
    # the busiest of a few views, so that a third of its records is still many
    dumps = {v: _dump("gp_debug_dump_tris", sim, v, out, dep, 16384) for v in (3, 5, 20, 40)}
    view = max(dumps, key=lambda v: dumps[v][1])
    full, n_full = dumps[view]
    assert n_full > 100
    cap = n_full // 3
    got, n = _dump("gp_debug_dump_tris_noalloc", sim, view, out, dep, cap)
    torch.cuda.synchronize()
    assert n == n_full and len(got) == cap
    rows = set(_sorted(full).tolist())
    assert all(r in rows for r in _sorted(got).tolist())


def test_noalloc_dump_rejects_capacity_beyond_its_scratch():
    from paper_2606_19641_b300 import GigapixelError, binding as b
    wl = wg.WORKLOADS["tiny"]
    worlds = wg.make_workload(wl)
    sim, cfg = sim_for(worlds, wl)
    out, dep = sim.alloc_outputs()
    with pytest.raises(GigapixelError) as e:
        _dump("gp_debug_dump_tris_noalloc", sim, 0, out, dep, b.NOALLOC_MAX_TRIS + 1)
    assert e.value.status == b.GP_ELIMIT and "16384" in str(e.value)
    got, n = _dump("gp_debug_dump_tris_noalloc", sim, 0, out, dep, b.NOALLOC_MAX_TRIS)
    assert n == len(got) > 0
