"""psc_hop_events_static: stepping molecules without the library allocating.

Some callers cannot let a library allocate device memory while they step
molecules (their framework owns all device memory through its own pool, or
they run under an allocator lock, or they cannot afford the synchronisation
cudaMalloc/cudaFree may cause).  psc_hop_events_static keeps its scratch in
fixed-size arrays inside the library instead.  This test drives it through the
C ABI on buffers the test owns and checks, on two calls in a row, that it
moves every molecule exactly as psc_run_events does on a lattice with the same
molecules and seed.
"""
import ctypes

import numpy as np
import pytest

import paper_1605_03726_gb300 as psc

pytestmark = pytest.mark.gpu


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


def test_static_scratch_matches_run_events_on_two_calls():
    import torch

    shape, n, seed, D = (64, 48, 40), 4000, 20261202, 2e-12
    L = psc.Lattice(*shape, voxel_radius=1e-8)
    s = L.add_species(D, n)
    L.populate(seed)
    ijk, ids = L.coords(s)
    ni, nj, _ = shape
    vox0 = (ijk[:, 0] + ni * (ijk[:, 1] + nj * ijk[:, 2])).astype(np.int32)

    dev = torch.device("cuda", 0)
    d_vox = torch.from_numpy(vox0.copy()).to(dev)
    d_ids = torch.from_numpy(ids.astype(np.uint32).view(np.int32).copy()).to(dev)
    d_img = torch.zeros(n, dtype=torch.int64, device=dev)
    stream = torch.cuda.current_stream(dev)
    lib = psc.lib()

    events = 25
    for call in range(2):
        first = L.event_index()
        rc = lib.psc_hop_events_static(*shape, psc.PERIODIC_ALL, seed, s, first, events,
                                       ctypes.c_void_p(d_vox.data_ptr()), ctypes.c_void_p(d_ids.data_ptr()),
                                       ctypes.c_void_p(d_img.data_ptr()), n, ctypes.c_void_p(stream.cuda_stream))
        assert rc == psc.OK, psc.lib().psc_status_string(rc)
        torch.cuda.synchronize(dev)
        L.run_events(events)

        vox = d_vox.cpu().numpy()
        img = d_img.cpu().numpy().view(np.uint64)
        got_ids = d_ids.cpu().numpy().view(np.uint32)
        order = np.argsort(got_ids, kind="stable")
        ref_ijk, ref_ids = L.coords(s)
        ref_xyz, _ = L.unwrapped(s)
        assert np.array_equal(got_ids[order], ref_ids)
        assert np.array_equal(_decode(vox[order], shape), ref_ijk), "positions differ after call %d" % call
        assert np.array_equal(_unwrapped(vox[order], img[order], shape), ref_xyz), "wraps differ after call %d" % call
        assert np.any(vox != vox0)

    # lattices beyond the fixed scratch are refused before any device work
    rc = lib.psc_hop_events_static(256, 128, 128, psc.PERIODIC_ALL, seed, s, 0, 1,
                                   ctypes.c_void_p(d_vox.data_ptr()), ctypes.c_void_p(d_ids.data_ptr()),
                                   ctypes.c_void_p(d_img.data_ptr()), n, ctypes.c_void_p(stream.cuda_stream))
    assert rc == psc.E_CAPACITY
    L.close()
