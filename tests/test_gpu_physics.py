"""Properties of long runs at full size, where the oracle cannot follow.

The 512^3 lattice at 1 % occupancy (1,342,177 molecules, D = 10 um^2/s) in
the launch configuration the benchmark times, run for 1000 events (ten
re-sorts).  What must hold at any size:

  exclusion      one molecule per voxel; the grid and the lists agree; ids kept
  Eq. 1-2        a single event moves a molecule by 0 or exactly one voxel
                 diameter (2 r_v), and the number moved equals the hops counted
  App. C/Eq. 14  mean squared displacement = (2 r_v)^2 x successful hops per
                 molecule (walkers at 1 % barely correlate), split evenly over
                 the three axes (the HCP stencil's second moment is isotropic)
  Sec. 2.3       simulated time = events x tau
"""
import numpy as np
import pytest

import paper_1605_03726_gb300 as psc

pytestmark = pytest.mark.gpu

N = int(0.01 * 512 ** 3)
RV = 1e-8
D = 10e-12


def axes3(a, b):
    """Per-axis 3 |dr|^2 / r_v^2 in the integer basis X, Y, Z."""
    d = b.astype(np.int64) - a.astype(np.int64)
    return np.stack([3 * d[:, 0] ** 2, d[:, 1] ** 2, 8 * d[:, 2] ** 2], axis=1)


def test_512cubed_long_run_properties():
    L = psc.Lattice(512, 512, 512, voxel_radius=RV)
    s = L.add_species(D, N)
    L.set_options(resort_period=100, collect_stats=1)
    L.populate(1)
    x0, id0 = L.unwrapped(s)
    assert np.array_equal(id0, np.arange(N, dtype=np.uint32))

    L.run_events(1000)
    st = L.stats()
    assert st["events"] == 1000 and st["attempts"] == 1000 * N
    assert L.time() == pytest.approx(1000 * 2 * RV * RV / (3 * D), rel=1e-12)

    # exclusion and bookkeeping
    ijk, ids = L.coords(s)
    assert np.array_equal(ids, id0)
    v = ijk[:, 0].astype(np.int64) + 512 * (ijk[:, 1] + 512 * ijk[:, 2].astype(np.int64))
    assert np.unique(v).size == N
    grid = L.grid()
    assert int(np.count_nonzero(grid)) == N
    assert (grid[v] == s + 1).all()

    # mean squared displacement against the counted hops
    x1, _ = L.unwrapped(s)
    a = axes3(x0, x1)
    hops_per_mol = st["hops"] / N
    ratio = a.sum(axis=1).mean() / (12.0 * hops_per_mol)
    assert 0.99 < ratio < 1.005, ratio
    share = a.mean(axis=0) / a.sum(axis=1).mean()
    assert np.allclose(share, 1.0 / 3.0, atol=0.005), share
    assert 0.97 < st["hops"] / st["attempts"] < 1.0

    # one more event: every molecule moves by 0 or one voxel diameter
    h0 = L.stats()["hops"]
    L.run_events(1)
    x2, _ = L.unwrapped(s)
    d = axes3(x1, x2).sum(axis=1)
    assert set(np.unique(d).tolist()) <= {0, 12}
    assert int(np.count_nonzero(d)) == L.stats()["hops"] - h0
    L.close()


def test_fcc_long_run_properties():
    # FCC lattice (App. B), 192^3 periodic, 1 % walkers, 500 events: exclusion,
    # one-diameter hops, MSD = (2 r_v)^2 x hops, isotropic second moment
    shape = (192, 192, 192)
    n = int(0.01 * shape[0] * shape[1] * shape[2])
    L = psc.Lattice(*shape, voxel_radius=RV, boundary=psc.PERIODIC_ALL | psc.FCC)
    s = L.add_species(D, n)
    L.set_options(collect_stats=1)
    L.populate(2)
    x0, id0 = L.unwrapped(s)
    L.run_events(500)
    st = L.stats()
    ijk, ids = L.coords(s)
    assert np.array_equal(ids, id0)
    v = ijk[:, 0].astype(np.int64) + shape[0] * (ijk[:, 1] + shape[1] * ijk[:, 2].astype(np.int64))
    assert np.unique(v).size == n
    assert int(np.count_nonzero(L.grid())) == n
    x1, _ = L.unwrapped(s)
    a = axes3(x0, x1)
    ratio = a.sum(axis=1).mean() / (12.0 * st["hops"] / n)
    assert 0.985 < ratio < 1.01, ratio
    share = a.mean(axis=0) / a.sum(axis=1).mean()
    assert np.allclose(share, 1.0 / 3.0, atol=0.01), share
    h0 = L.stats()["hops"]
    L.run_events(1)
    x2, _ = L.unwrapped(s)
    d = axes3(x1, x2).sum(axis=1)
    assert set(np.unique(d).tolist()) <= {0, 12}
    assert int(np.count_nonzero(d)) == L.stats()["hops"] - h0
    L.close()


def test_cell_long_run_properties():
    # 256^3 lattice holding a round cell (cytoplasm 35 % of the voxels); 2^20
    # walkers confined to the cytoplasm, 1000 events under the automatic
    # kernel choice: exclusion, ids kept, every molecule still in the
    # cytoplasm, and one more event moves each by 0 or one voxel diameter
    import models
    shape = (256, 256, 256)
    lab = models.cell_labels(*shape, radius=200.0)
    n = 1 << 20
    L = psc.Lattice(*shape, voxel_radius=RV)
    L.set_compartments(lab, 3)
    s = L.add_species(D, n, compartment=2)
    L.set_options(collect_stats=1)
    L.populate(5)
    _, id0 = L.unwrapped(s)
    L.run_events(1000)
    ijk, ids = L.coords(s)
    assert np.array_equal(ids, id0)
    v = ijk[:, 0].astype(np.int64) + 256 * (ijk[:, 1] + 256 * ijk[:, 2].astype(np.int64))
    assert np.unique(v).size == n
    assert (lab[v] == 2).all()
    assert int(np.count_nonzero(L.grid())) == n
    x1, _ = L.unwrapped(s)
    h0 = L.stats()["hops"]
    L.run_events(1)
    x2, _ = L.unwrapped(s)
    d = axes3(x1, x2).sum(axis=1)
    assert set(np.unique(d).tolist()) <= {0, 12}
    assert int(np.count_nonzero(d)) == L.stats()["hops"] - h0
    L.close()
