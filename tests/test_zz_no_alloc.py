"""psc_hop_events_static: stepping molecules without the library allocating.

Some callers cannot let a library allocate device memory while they step
molecules (their framework owns all device memory through its own pool, or
they run under an allocator lock, or they cannot afford the synchronisation
cudaMalloc/cudaFree may cause).  psc_hop_events_static keeps its scratch in
fixed-size arrays inside the library instead.  These tests drive it through
the C ABI on buffers the test owns and check, on two calls in a row, that it
moves every molecule exactly as psc_run_events does on a lattice with the same
molecules and seed, and exactly as the oracle does; that molecules it cannot
accept (a voxel out of range or taken twice, the reserved id) are refused with
the buffers left as they were; and that a call with no molecules is fine.
"""
import ctypes

import numpy as np
import pytest

import oracle
import paper_1605_03726_gb300 as psc

pytestmark = pytest.mark.gpu

MAX_VOXELS = 1 << 21          # the entry point's documented limit


def _decode(vox, shape):
    ni, nj, _ = shape
    v = vox.astype(np.int64)
    return np.stack([v % ni, (v // ni) % nj, v // (ni * nj)], axis=1)


def _unwrapped(vox, img, shape):
    """Integer basis of psc_unwrapped: X = 2I + P, Y = 3J + (K & 1), Z = K."""
    ni, nj, nk = shape
    ijk = _decode(vox, shape)
    w = img.astype(np.uint64)
    field = lambda sh: ((w >> np.uint64(sh)) & np.uint64(0xFFFF)).astype(np.uint16).view(np.int16).astype(np.int64)
    I = ijk[:, 0] + field(0) * ni
    J = ijk[:, 1] + field(16) * nj
    K = ijk[:, 2] + field(32) * nk
    return np.stack([2 * I + ((J + K) & 1), 3 * J + (K & 1), K], axis=1)


class Buffers:
    """Caller-owned device buffers (vox, ids, img) and a call through the C ABI."""

    def __init__(self, vox, ids):
        import torch
        self.dev = torch.device("cuda", 0)
        self.vox = torch.from_numpy(np.asarray(vox, dtype=np.int32).copy()).to(self.dev)
        self.ids = torch.from_numpy(np.asarray(ids, dtype=np.uint32).view(np.int32).copy()).to(self.dev)
        self.img = torch.zeros(len(vox), dtype=torch.int64, device=self.dev)
        self.n = len(vox)
        self.stream = torch.cuda.current_stream(self.dev)

    def call(self, shape, flags, seed, species, first, events, n=None):
        n = self.n if n is None else n
        return psc.lib().psc_hop_events_static(
            *shape, flags, seed, species, first, events,
            ctypes.c_void_p(self.vox.data_ptr()), ctypes.c_void_p(self.ids.data_ptr()),
            ctypes.c_void_p(self.img.data_ptr()), n, ctypes.c_void_p(self.stream.cuda_stream))

    def host(self):
        import torch
        torch.cuda.synchronize(self.dev)
        return (self.vox.cpu().numpy(), self.ids.cpu().numpy().view(np.uint32),
                self.img.cpu().numpy().view(np.uint64))


CASES = {
    # shape, boundary flags, molecules
    "periodic 64x48x40": ((64, 48, 40), psc.PERIODIC_ALL, 4000),
    "reflective ragged 37x29x23": ((37, 29, 23), 0, 3000),
    "mixed walls 30x26x20": ((30, 26, 20), psc.PERIODIC_I | psc.PERIODIC_K, 2500),
    "at the limit 128^3": ((128, 128, 128), psc.PERIODIC_ALL, 20971),
}


@pytest.mark.parametrize("case", sorted(CASES))
def test_static_scratch_matches_run_events_and_oracle_on_two_calls(case):
    shape, flags, n = CASES[case]
    seed, D, events = 20261202, 2e-12, 25
    ni, nj, nk = shape
    assert ni * nj * nk <= MAX_VOXELS
    L = psc.Lattice(*shape, voxel_radius=1e-8, boundary=flags)
    s = L.add_species(D, n)
    L.populate(seed)
    O = oracle.Lattice(*shape, 1e-8, flags)
    O.add_species(D, n)
    O.populate(seed)
    ijk, ids = L.coords(s)
    vox0 = (ijk[:, 0] + ni * (ijk[:, 1] + nj * ijk[:, 2])).astype(np.int32)
    B = Buffers(vox0, ids)

    for call in range(2):
        first = L.event_index()
        rc = B.call(shape, flags, seed, s, first, events)
        assert rc == psc.OK, psc.lib().psc_status_string(rc)
        L.run_events(events)
        O.run_events(events)

        vox, got_ids, img = B.host()
        order = np.argsort(got_ids, kind="stable")
        for name, (ref_ijk, ref_ids), ref_xyz in (("psc_run_events", L.coords(s), L.unwrapped(s)[0]),
                                                  ("oracle", O.coords(0), O.unwrapped(0)[0])):
            assert np.array_equal(got_ids[order], ref_ids), name
            assert np.array_equal(_decode(vox[order], shape), ref_ijk), \
                "positions differ from %s after call %d" % (name, call)
            assert np.array_equal(_unwrapped(vox[order], img[order], shape), ref_xyz), \
                "wraps differ from %s after call %d" % (name, call)
        assert np.any(vox != vox0)

    # a call with no molecules is fine; lattices beyond the fixed scratch are
    # refused before any device work
    assert B.call(shape, flags, seed, s, 0, 3, n=0) == psc.OK
    assert B.call((256, 128, 128), psc.PERIODIC_ALL, seed, s, 0, 1) == psc.E_CAPACITY
    O.close()
    L.close()


@pytest.mark.parametrize("fault", ["voxel out of range", "negative voxel", "two on one voxel", "reserved id"])
def test_static_refuses_bad_molecules_and_leaves_buffers(fault):
    shape, flags, n, seed = (40, 36, 32), psc.PERIODIC_ALL, 1500, 77
    ni, nj, nk = shape
    V = ni * nj * nk
    O = oracle.Lattice(*shape, 1e-8, flags)
    O.add_species(2e-12, n)
    O.populate(seed)
    ijk, ids = O.coords(0)
    vox0 = (ijk[:, 0] + ni * (ijk[:, 1] + nj * ijk[:, 2])).astype(np.int32)
    bad_vox, bad_ids = vox0.copy(), ids.astype(np.uint32).copy()
    if fault == "voxel out of range":
        bad_vox[n // 2] = V
    elif fault == "negative voxel":
        bad_vox[7] = -5
    elif fault == "two on one voxel":
        bad_vox[n - 1] = bad_vox[3]
    else:
        bad_ids[11] = 0xFFFFFFFF
    B = Buffers(bad_vox, bad_ids)
    assert B.call(shape, flags, seed, 0, 0, 10) == psc.E_ARG
    vox, got_ids, img = B.host()
    assert np.array_equal(vox, bad_vox) and np.array_equal(got_ids, bad_ids) and not np.any(img)

    # the next call on good molecules starts clean and matches the oracle
    G = Buffers(vox0, ids)
    assert G.call(shape, flags, seed, 0, 0, 10) == psc.OK
    O.run_events(10)
    vox, got_ids, img = G.host()
    order = np.argsort(got_ids, kind="stable")
    ref_ijk, ref_ids = O.coords(0)
    assert np.array_equal(got_ids[order], ref_ids)
    assert np.array_equal(_decode(vox[order], shape), ref_ijk)
    O.close()
