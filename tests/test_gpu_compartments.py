"""Compartments on the GPU (Sec. 2: a cell as groups of voxels; Sec. 2.3: a
hop into another compartment fails) against the oracle, bit-exact: grid,
counts, positions sorted by id, unwrapped positions, event index and clock.

Models: a round cell (outside, membrane shell, cytoplasm) with a ligand, a
membrane receptor that diffuses, binding across the membrane, release of the
ligand into the cytoplasm, a conversion whose products trade places when the
receptor moves, and walkers outside; and walkers of three species in random
compartments.  Paths: per-event claim / commit kernels (hash and per-voxel
claims), the persistent molecule-list kernel, the tile kernel, the sub-volume
rule, FCC, a batch of lattices with different compartments, and a 128^3
cell at 1-2 % occupancy.
"""
import numpy as np
import pytest

import oracle
import paper_1605_03726_gb300 as psc
import models

pytestmark = pytest.mark.gpu


def same(g, o, ns, tag=""):
    assert g.event_index() == o.event_index(), tag
    assert g.time() == o.time(), tag
    assert (g.counts() == o.counts()).all(), (tag, g.counts(), o.counts())
    assert np.array_equal(g.grid(), o.grid()), tag
    for s in range(ns):
        a, b = g.coords(s), o.coords(s)
        assert np.array_equal(a[1], b[1]) and np.array_equal(a[0], b[0]), (tag, s)
        assert np.array_equal(g.unwrapped(s)[0], o.unwrapped(s)[0]), (tag, s)


def pair(shape, boundary, recipe, seed, rule=oracle.RULE_SYNC, **opts):
    g = psc.Lattice(*shape, voxel_radius=1e-8, boundary=boundary)
    if opts:
        g.set_options(**opts)
    o = oracle.Lattice(*shape, 1e-8, boundary, rule)
    ns = recipe(g)
    recipe(o)
    assert g.populate(seed) == o.populate(seed)
    same(g, o, ns, "populate")
    return g, o, ns


def cell(shape, radius, n_lig, n_rec, n_x, n_out, koff=2e3):
    lab = models.cell_labels(*shape, radius=radius)

    def recipe(L):
        models.receptor_binding(L, lab, n_lig, n_rec, n_x=n_x, n_outside=n_out, koff=koff)
        return 5
    return recipe


def random_walkers(shape, seed=3):
    V = shape[0] * shape[1] * shape[2]
    lab = np.random.default_rng(seed).choice(3, size=V, p=[0.3, 0.3, 0.4]).astype(np.uint8)

    def recipe(L):
        L.set_compartments(lab, 3)
        L.add_species(1e-12, int(0.10 * V), compartment=0)
        L.add_species(3e-12, int(0.05 * V), compartment=1)
        L.add_species(2e-12, int(0.20 * V), compartment=2)
        return 3
    return recipe


@pytest.mark.parametrize("claim_table", [1, 2])
@pytest.mark.parametrize("persistent", [1, -1])
def test_cell_with_membrane_receptors(claim_table, persistent):
    shape = (40, 36, 32)
    g, o, ns = pair(shape, 0, cell(shape, 30.0, 1500, 600, 400, 1500), 5,
                    claim_table=claim_table, persistent=persistent, tiles=1)
    for chunk in (3, 30, 100):
        g.run_events(chunk)
        o.run_events(chunk)
        same(g, o, ns, chunk)
    st = o.stats()
    assert st["reactions2"] > 50 and st["reactions1"] > 10 and st["births"] > 10


@pytest.mark.parametrize("opts", [dict(persistent=-1, claim_table=1), dict(persistent=-1, claim_table=2),
                                  dict(persistent=1, claim_table=2), dict(tiles=1, claim_table=1),
                                  dict(tiles=1, tile_regions=8, claim_table=2)])
def test_walkers_in_random_compartments(opts):
    shape = (48, 44, 40)
    g, o, ns = pair(shape, psc.PERIODIC_ALL, random_walkers(shape), 9, **opts)
    for chunk in (1, 9, 40):
        g.run_events(chunk)
        o.run_events(chunk)
        same(g, o, ns, chunk)


def test_subvolume_rule_with_compartments():
    shape = (32, 28, 24)
    g, o, ns = pair(shape, psc.PERIODIC_ALL, random_walkers(shape, seed=4), 6, rule=oracle.RULE_SUBVOL,
                    subvolume=1)
    for chunk in (1, 6, 25):
        g.run_events(chunk)
        o.run_events(chunk)
        same(g, o, ns, chunk)


@pytest.mark.parametrize("persistent", [1, -1])
def test_fcc_cell(persistent):
    shape = (37, 29, 23)
    g, o, ns = pair(shape, psc.FCC, cell(shape, 24.0, 800, 300, 200, 900), 12, persistent=persistent)
    for chunk in (4, 40, 80):
        g.run_events(chunk)
        o.run_events(chunk)
        same(g, o, ns, chunk)


def test_batch_members_with_different_compartments():
    import torch
    stream = torch.cuda.Stream()
    B = psc.Batch(stream=stream.cuda_stream)
    cases = [((24, 24, 20), 0, cell((24, 24, 20), 18.0, 300, 150, 100, 300), 5, 21),
             ((32, 28, 24), psc.PERIODIC_ALL, random_walkers((32, 28, 24), seed=8), 3, 22),
             ((20, 20, 20), psc.PERIODIC_ALL, lambda L: (models.reaction_diffusion_ab(L, 300, 300), 3)[1], 3, 23)]
    members = []
    for shape, bnd, recipe, ns, seed in cases:
        m = psc.Lattice(*shape, voxel_radius=1e-8, boundary=bnd, stream=stream.cuda_stream)
        m.set_options(claim_table=1, resort_period=-1)
        recipe(m)
        m.populate(seed)
        B.add(m)
        members.append(m)
    B.run_events(120)
    for m, (shape, bnd, recipe, ns, seed) in zip(members, cases):
        o = oracle.Lattice(*shape, 1e-8, bnd, oracle.RULE_SYNC)
        recipe(o)
        o.populate(seed)
        o.run_events(120)
        same(m, o, ns)
    B.close()


def test_cell_128cubed():
    shape = (128, 128, 128)
    g, o, ns = pair(shape, 0, cell(shape, 100.0, 20000, 8000, 5000, 20000), 31)
    for chunk in (10, 40):
        g.run_events(chunk)
        o.run_events(chunk)
        same(g, o, ns, chunk)
    lab = models.cell_labels(*shape, radius=100.0)
    for s, c in zip(range(5), (2, 1, 1, 2, 0)):
        ijk, _ = g.coords(s)
        v = ijk[:, 0].astype(np.int64) + 128 * (ijk[:, 1] + 128 * ijk[:, 2].astype(np.int64))
        assert (lab[v] == c).all()


def test_compartment_errors_match_oracle():
    shape = (16, 16, 16)
    V = 16 ** 3
    lab = np.zeros(V, np.uint8)
    lab[V // 2:] = 1
    for L, err in ((psc.Lattice(*shape, voxel_radius=1e-8), psc.EngineError),
                   (oracle.Lattice(*shape, 1e-8), oracle.OracleError)):
        with pytest.raises(err):
            L.set_compartments(np.full(V, 3, np.uint8), 3)
        with pytest.raises(err):
            L.set_compartments(lab, 17)
        a = L.add_species(1e-12, V // 2 + 1)
        with pytest.raises(err):
            L.species_compartment(a, 1)
        L.set_compartments(lab, 2)
        with pytest.raises(err) as e:
            L.populate(1)                         # more than compartment 0 holds
        assert e.value.rc == -4
        L.close()


def test_auto_kernel_follows_box_loads():
    # 256^3, 2^20 + 1 walkers: spread over the lattice the automatic choice
    # takes the tile kernel; confined to a round cell (the boxes outside hold
    # nothing, those inside about 3x the mean) it takes the molecule-list
    # kernel.  Either way the result is the one every kernel gives.
    shape = (256, 256, 256)
    n = (1 << 20) + 1
    lab = models.cell_labels(*shape, radius=200.0)
    for confined in (False, True):
        out = {}
        for tiles in (0, 1, -1):
            L = psc.Lattice(*shape, voxel_radius=1e-8)
            if confined:
                L.set_compartments(lab, 3)
                L.add_species(10e-12, n, compartment=2)
            else:
                L.add_species(10e-12, n)
            L.set_options(time_kernels=1, **({"tiles": tiles} if tiles else {}))
            L.populate(4)
            L.run_events(60)
            kt = L.kernel_times()
            out[tiles] = (L.coords(0), kt["tile_launches"], kt["run_launches"])
            L.close()
        for t in (1, -1):
            assert np.array_equal(out[t][0][0], out[0][0][0]) and np.array_equal(out[t][0][1], out[0][0][1])
        tile_launches, stretch_launches = out[0][1], out[0][2]     # tile stretches count as both
        if confined:
            assert tile_launches == 0 and stretch_launches > 0
        else:
            assert tile_launches > 0 and tile_launches == stretch_launches


def test_tile_kernel_fcc_with_compartments():
    # FCC, periodic (k a multiple of 6), walkers of three species in random
    # compartments, forced onto the tile kernel with several box counts
    shape = (48, 44, 42)
    for regions in (0, 6):
        g, o, ns = pair(shape, psc.PERIODIC_ALL | psc.FCC, random_walkers(shape, seed=5), 14,
                        tiles=1, tile_regions=regions, time_kernels=1)
        for chunk in (1, 9, 40):
            g.run_events(chunk)
            o.run_events(chunk)
            same(g, o, ns, chunk)
        assert g.kernel_times()["tile_launches"] > 0
        g.close()
        o.close()


def test_autotuned_cell_matches_untuned():
    # the tuner's trials are real events: a tuned cell lattice ends where an
    # untuned one ends after as many events, and both stay with the oracle
    shape = (96, 96, 96)
    recipe = cell(shape, 75.0, 8000, 3000, 2000, 8000)
    T = psc.Lattice(*shape, voxel_radius=1e-8, boundary=0)
    U = psc.Lattice(*shape, voxel_radius=1e-8, boundary=0)
    o = oracle.Lattice(*shape, 1e-8, 0, oracle.RULE_SYNC)
    for L in (T, U, o):
        recipe(L)
        L.populate(17)
    r = T.autotune(600)
    assert 0 < r["events"] <= 600
    U.run_events(r["events"])
    o.run_events(r["events"])
    same(T, o, 5, "tuned")
    same(U, o, 5, "untuned")
    T.run_events(150)
    o.run_events(150)
    same(T, o, 5, "after")
    for L in (T, U, o):
        L.close()


def test_device_bytes_count_one_mirror_per_compartment():
    shape = (64, 64, 64)
    lab = models.cell_labels(*shape, radius=50.0)
    sizes = []
    for n_comp in (None, 3):
        L = psc.Lattice(*shape, voxel_radius=1e-8)
        if n_comp:
            L.set_compartments(lab, n_comp)
        L.add_species(1e-12, 1000, compartment=2 if n_comp else None)
        L.populate(1)
        sizes.append(L.device_bytes())
        L.close()
    words = (64 // 4) * (64 // 4) * (64 // 2)
    assert sizes[1] - sizes[0] == 2 * words * 4
