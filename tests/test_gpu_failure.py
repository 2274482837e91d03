"""Failure detection without a GPU fault.

Every wait inside a persistent launch (the grid barrier between the claim and
commit phases) is bounded.  The first test makes that wait run out -- the
barrier awaits arrivals from a block that does not exist, a flag nothing ever
sets -- and checks that the error reaches the host as PSC_E_TIMEOUT, that the
lattice keeps reporting it, and that the device stays usable: a new lattice
afterwards runs and matches the oracle.  The second injects allocation
failures on the host through the allocator hook and checks that each one is
reported as PSC_E_NOMEM with every allocation that did succeed given back.
"""
import time

import numpy as np
import pytest

import oracle
import paper_1605_03726_gb300 as psc

pytestmark = pytest.mark.gpu

SHAPE = (48, 48, 48)
N = 3000
D = 1e-12


def _walkers(L, seed=17):
    s = L.add_species(D, N)
    L.populate(seed)
    return s


def test_barrier_wait_runs_out_and_is_reported():
    L = psc.Lattice(*SHAPE, voxel_radius=1e-8)
    # 20 ms bound; one phantom arrival that never comes
    L.set_options(persistent=1, resort_period=-1, barrier_timeout_us=20000, barrier_phantom=1)
    _walkers(L)
    t0 = time.monotonic()
    L.run_events(8)                          # queued: one persistent launch
    with pytest.raises(psc.EngineError) as err:
        L.synchronize()
    assert err.value.rc == psc.E_TIMEOUT
    assert time.monotonic() - t0 < 10.0
    # the lattice keeps the error; nothing more is launched on it
    with pytest.raises(psc.EngineError) as err:
        L.run_events(1)
    assert err.value.rc == psc.E_TIMEOUT
    with pytest.raises(psc.EngineError) as err:
        L.counts()
    assert err.value.rc == psc.E_TIMEOUT
    L.close()

    # the context is still usable: the same run without the phantom matches the oracle
    G = psc.Lattice(*SHAPE, voxel_radius=1e-8)
    G.set_options(persistent=1, resort_period=-1, barrier_timeout_us=20000)
    s = _walkers(G)
    G.run_events(8)
    G.synchronize()
    o = oracle.Lattice(*SHAPE, 1e-8, oracle.PERIODIC_ALL, oracle.RULE_SYNC)
    o.add_species(D, N)
    o.populate(17)
    o.run_events(8)
    a, b = G.coords(s), o.coords(s)
    assert np.array_equal(a[0], b[0]) and np.array_equal(a[1], b[1])
    G.close()


@pytest.mark.parametrize("regions,lean", [(8, 0), (16, 1)])
def test_tile_neighbour_wait_runs_out_and_is_reported(regions, lean):
    # the tile kernels' phases wait on neighbouring boxes' flags, bounded the
    # same way; 8 boxes (one along i) take the general kernel, 16 the lean one
    G0 = psc.Lattice(*SHAPE, voxel_radius=1e-8)
    G0.set_options(persistent=1, tiles=1, tile_regions=regions, time_kernels=1)
    _walkers(G0)
    G0.run_events(2)
    assert (G0.kernel_times()["tile_lean_events"] > 0) == bool(lean)
    G0.close()
    L = psc.Lattice(*SHAPE, voxel_radius=1e-8)
    L.set_options(persistent=1, tiles=1, tile_regions=regions, barrier_timeout_us=20000, barrier_phantom=1)
    _walkers(L)
    t0 = time.monotonic()
    L.run_events(4)
    with pytest.raises(psc.EngineError) as err:
        L.synchronize()
    assert err.value.rc == psc.E_TIMEOUT
    assert time.monotonic() - t0 < 10.0
    L.close()
    G = psc.Lattice(*SHAPE, voxel_radius=1e-8)
    G.set_options(persistent=1, tiles=1, tile_regions=regions)
    s = _walkers(G)
    G.run_events(8)
    o = oracle.Lattice(*SHAPE, 1e-8, oracle.PERIODIC_ALL, oracle.RULE_SYNC)
    o.add_species(D, N)
    o.populate(17)
    o.run_events(8)
    a, b = G.coords(s), o.coords(s)
    assert np.array_equal(a[0], b[0]) and np.array_equal(a[1], b[1])
    G.close()


class _FailingAllocator:
    """Device memory from PyTorch's caching allocator; the allocation numbered
    `fail_at` (0-based) returns NULL."""

    def __init__(self, fail_at):
        import torch
        self.torch = torch
        self.fail_at = fail_at
        self.calls = 0
        self.live = set()
        self.hooks = (psc.ALLOC_FN(self.alloc), psc.FREE_FN(self.free))

    def alloc(self, nbytes, device, stream, ctx):
        k = self.calls
        self.calls += 1
        if k == self.fail_at:
            return None
        p = self.torch.cuda.caching_allocator_alloc(int(nbytes), device, stream or 0)
        self.live.add(p)
        return p

    def free(self, ptr, device, stream, ctx):
        self.live.discard(ptr)
        self.torch.cuda.caching_allocator_delete(ptr)


def test_allocation_failures_are_reported_and_cleaned_up():
    lib = psc.lib()
    # how many allocations a populated lattice makes
    probe = _FailingAllocator(fail_at=-1)
    assert lib.psc_set_allocator(probe.hooks[0], probe.hooks[1], None) == psc.OK
    try:
        L = psc.Lattice(*SHAPE, voxel_radius=1e-8)
        L.add_species(D, N)
        L.add_species(0.0, 50)
        L.add_reaction((0, 1), (1,), 1e-19)
        L.populate(3)
        L.run_events(3)
        L.synchronize()
        L.close()
        total = probe.calls
        assert total > 0 and not probe.live
        for k in range(total):
            fa = _FailingAllocator(fail_at=k)
            assert lib.psc_set_allocator(fa.hooks[0], fa.hooks[1], None) == psc.OK
            L = psc.Lattice(*SHAPE, voxel_radius=1e-8)
            L.add_species(D, N)
            L.add_species(0.0, 50)
            L.add_reaction((0, 1), (1,), 1e-19)
            with pytest.raises(psc.EngineError) as err:
                L.populate(3)
                L.run_events(3)
                L.synchronize()
            assert err.value.rc == psc.E_NOMEM, k
            L.close()
            assert not fa.live, "allocation %d: %d blocks not given back" % (k, len(fa.live))
    finally:
        psc.use_cuda_malloc()
    # plain cudaMalloc again: a lattice still works
    L = psc.Lattice(*SHAPE, voxel_radius=1e-8)
    _walkers(L)
    L.run_events(2)
    L.synchronize()
    L.close()


def test_subvolume_barrier_wait_runs_out_and_is_reported():
    # the sub-volume rule's persistent launch waits at bounded grid barriers too
    shape = (48, 48, 48)
    L = psc.Lattice(*shape, voxel_radius=1e-8)
    L.set_options(subvolume=1, barrier_timeout_us=20000, barrier_phantom=1)
    _walkers(L)
    t0 = time.monotonic()
    L.run_events(4)
    with pytest.raises(psc.EngineError) as err:
        L.synchronize()
    assert err.value.rc == psc.E_TIMEOUT
    assert time.monotonic() - t0 < 10.0
    L.close()
    G = psc.Lattice(*shape, voxel_radius=1e-8)
    G.set_options(subvolume=1)
    s = _walkers(G)
    G.run_events(6)
    o = oracle.Lattice(*shape, 1e-8, oracle.PERIODIC_ALL, oracle.RULE_SUBVOL)
    o.add_species(D, N)
    o.populate(17)
    o.run_events(6)
    a, b = G.coords(s), o.coords(s)
    assert np.array_equal(a[0], b[0]) and np.array_equal(a[1], b[1])
    G.close()
