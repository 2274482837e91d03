"""Bit-exact parity of the CUDA engine with the synchronous-rule oracle.

Both sides get the same model and seed; at every checkpoint the occupancy
grid, the counts, every molecule's (i, j, k) and unwrapped position sorted by
id, the event index and the clock must be identical.  Sizes run from tiny and
ragged shapes to the full 64^3 reaction case and the 512^3 diffusion lattice.
"""
import numpy as np
import pytest

import oracle
import paper_1605_03726_gb300 as psc
import models

pytestmark = pytest.mark.gpu


def make_pair(shape, rv=1e-8, boundary=psc.PERIODIC_ALL, **opts):
    g = psc.Lattice(*shape, voxel_radius=rv, boundary=boundary)
    if opts:
        g.set_options(**opts)
    o = oracle.Lattice(*shape, rv, boundary, oracle.RULE_SYNC)
    return g, o


def assert_same(g, o, tag=""):
    n = o.n_species
    assert g.event_index() == o.event_index(), tag
    assert g.time() == o.time(), tag
    assert (g.counts() == o.counts()).all(), (tag, g.counts(), o.counts())
    assert (g.grid() == o.grid()).all(), tag
    for s in range(n):
        gi, gid = g.coords(s)
        oi, oid = o.coords(s)
        assert np.array_equal(gid, oid), (tag, s)
        assert np.array_equal(gi, oi), (tag, s)
        gu, _ = g.unwrapped(s)
        ou, _ = o.unwrapped(s)
        assert np.array_equal(gu, ou), (tag, s)


def build_both(shape, recipe, seed, boundary=psc.PERIODIC_ALL, rv=1e-8, **opts):
    g, o = make_pair(shape, rv, boundary, **opts)
    recipe(g)
    recipe(o)
    rg = g.populate(seed)
    ro = o.populate(seed)
    assert rg == ro
    assert_same(g, o, "populate")
    return g, o


@pytest.mark.parametrize("seed", [1, 2, 3])
def test_ab_to_c_64cubed_full_run(seed):
    # 64^3 periodic, r_v 10 nm, A and B 2000 each (D 1 um^2/s), A + B -> C with
    # k = 1e-19 m^3/s, C immobile; run to 1000 hop intervals of A
    g, o = build_both((64, 64, 64), lambda L: models.reaction_diffusion_ab(L, 2000, 2000), seed,
                      claim_table=1 + seed % 2)
    tau = g.tau(0)
    assert tau == o.tau(0)
    assert g.p_ab(0) == o.p_ab(0)
    for t in (1, 10, 100, 1000):
        g.run(t * tau)
        o.run(t * tau)
        assert_same(g, o, "t=%d tau" % t)


@pytest.mark.parametrize("persistent", [1, -1])
@pytest.mark.parametrize("claim_table", [1, 2])
@pytest.mark.parametrize("shape,frac", [((96, 80, 64), 0.01), ((37, 24, 18), 0.30), ((50, 44, 30), 0.60)])
def test_diffusion_ragged_shapes(shape, frac, claim_table, persistent):
    V = shape[0] * shape[1] * shape[2]
    g, o = build_both(shape, lambda L: models.diffusion_only(L, int(frac * V)), 11, resort_period=7,
                      claim_table=claim_table, persistent=persistent)
    for _ in range(4):
        g.run_events(13)
        o.run_events(13)
        assert_same(g, o)


@pytest.mark.parametrize("claim_table", [1, 2])
def test_reflective_crowded_reversible(claim_table):
    shape = (40, 36, 32)
    V = 40 * 36 * 32
    g, o = build_both(shape, lambda L: models.crowded_reversible(L, V, kb=2000.0), 5, boundary=0,
                      collect_stats=1, claim_table=claim_table)
    for _ in range(5):
        g.run_events(60)
        o.run_events(60)
        assert_same(g, o)
    sg, so = g.stats(), o.stats()
    for key in ("attempts", "hops", "collisions", "accepted", "reactions2", "fires", "reactions1", "births"):
        assert sg[key] == so[key], key
    assert so["reactions2"] > 0 and so["births"] > 0


@pytest.mark.parametrize("claim_table", [1, 2])
def test_mapk_like_cascade(claim_table):
    shape = (40, 40, 40)
    recipe = lambda L: models.mapk_like(L, 7, scale=0.3, uni_scale=300, bi_scale=3)
    g, o = build_both(shape, recipe, 7, collect_stats=1, claim_table=claim_table)
    for _ in range(6):
        g.run_events(500)
        o.run_events(500)
        assert_same(g, o)
    so = o.stats()
    assert so["births"] > 50 and so["reactions2"] > 100
    assert g.stats()["births"] == so["births"]


@pytest.mark.parametrize("claim_table", [1, 2])
@pytest.mark.parametrize("products", [[], [2], [2, 3]])
def test_second_order_product_counts(products, claim_table):
    def recipe(L):
        a = L.add_species(2e-12, 1500)
        b = L.add_species(1e-12, 1500)
        L.add_species(0.5e-12, 0)
        L.add_species(0.0, 0)
        L.add_reaction([a, b], products, 5e-19)
    g, o = build_both((32, 32, 32), recipe, 9, claim_table=claim_table)
    for _ in range(3):
        g.run_events(40)
        o.run_events(40)
        assert_same(g, o)


@pytest.mark.parametrize("claim_table", [1, 2])
@pytest.mark.parametrize("products", [[], [1], [1, 2], [0, 2]])
def test_first_order_product_counts(products, claim_table):
    def recipe(L):
        a = L.add_species(1e-12, 3000)
        L.add_species(0.3e-12, 0)
        L.add_species(0.0, 0)
        L.add_reaction([a], products, 3000.0)
    g, o = build_both((24, 24, 24), recipe, 4, claim_table=claim_table)
    for _ in range(3):
        g.run_events(25)
        o.run_events(25)
        assert_same(g, o)


@pytest.mark.parametrize("claim_table", [1, 2])
def test_walkers_without_reactions_among_reacting_species(claim_table):
    # T moves but takes part in no reaction, so it keeps no codes in the grid
    # while moving; A + B -> C + D and C -> A + B react around it
    def recipe(L):
        t = L.add_species(3e-12, 4000)
        a = L.add_species(1e-12, 2500)
        b = L.add_species(2e-12, 2500)
        c = L.add_species(0.5e-12, 0)
        d = L.add_species(1.5e-12, 0)
        L.add_species(0.0, 3000)                   # immobile crowders, no reactions
        L.add_reaction([a, b], [c, d], 4e-19)
        L.add_reaction([c], [a, b], 5000.0)
    g, o = build_both((36, 40, 30), recipe, 13, claim_table=claim_table, collect_stats=1)
    for _ in range(6):
        g.run_events(40)
        o.run_events(40)
        assert_same(g, o)
    assert o.stats()["reactions2"] > 0


def test_edge_cases():
    # empty lattice
    g, o = build_both((8, 8, 8), lambda L: L.add_species(1e-12, 0), 1)
    g.run_events(3); o.run_events(3)
    assert_same(g, o, "empty")
    # full lattice: nothing can move
    g, o = build_both((6, 6, 6), lambda L: L.add_species(1e-12, 216), 1)
    g.run_events(3); o.run_events(3)
    assert_same(g, o, "full")
    # single molecule on the smallest periodic lattice
    g, o = build_both((3, 4, 4), lambda L: L.add_species(1e-12, 1), 2)
    g.run_events(50); o.run_events(50)
    assert_same(g, o, "single")
    # one voxel, reflective: every hop hits a wall
    g, o = build_both((1, 1, 1), lambda L: L.add_species(1e-12, 1), 3, boundary=0)
    g.run_events(5); o.run_events(5)
    assert_same(g, o, "one voxel")
    # only immobile species: no events at all
    g, o = build_both((8, 8, 8), lambda L: L.add_species(0.0, 100), 4)
    g.run(1.0); o.run(1.0)
    assert_same(g, o, "immobile")
    # mixed boundaries, odd reflective extents
    g, o = build_both((7, 9, 8), lambda L: L.add_species(1e-12, 150), 5, boundary=psc.PERIODIC_K)
    g.run_events(30); o.run_events(30)
    assert_same(g, o, "mixed")


def test_results_do_not_depend_on_launch_shape_or_resort():
    recipe = lambda L: models.reaction_diffusion_ab(L, 3000, 3000, k=3e-19)
    states = []
    for opts in (dict(resort_period=-1), dict(resort_period=1), dict(block_threads=64, blocks_per_sm=1),
                 dict(block_threads=128, blocks_per_sm=3, resort_period=5)):
        g = psc.Lattice(48, 48, 48)
        g.set_options(**opts)
        recipe(g)
        g.populate(21)
        g.run_events(120)
        states.append((g.grid(), [g.coords(s) for s in range(3)]))
    for grid, coords in states[1:]:
        assert np.array_equal(grid, states[0][0])
        for (a, b), (c, d) in zip(coords, states[0][1]):
            assert np.array_equal(a, c) and np.array_equal(b, d)


@pytest.mark.parametrize("persistent", [1, -1])
def test_diffusion_256cubed_one_percent(persistent):
    g, o = build_both((256, 256, 256), lambda L: models.diffusion_only(L, 167772), 2, persistent=persistent)
    for _ in range(2):
        g.run_events(10)
        o.run_events(10)
        assert_same(g, o)


@pytest.mark.slow
def test_diffusion_512cubed_full_size():
    # the 512^3 lattice at 1 % occupancy (1,342,177 molecules, D = 10 um^2/s) in
    # the launch configuration the benchmark times: one persistent stretch of
    # 100 events, the re-sort, then part of the next stretch
    n = int(0.01 * 512 ** 3)
    g, o = build_both((512, 512, 512), lambda L: models.diffusion_only(L, n, D=10e-12), 1, resort_period=100)
    for chunk in (3, 97, 40):
        g.run_events(chunk)
        o.run_events(chunk)
        assert_same(g, o, chunk)


@pytest.mark.slow
def test_crowded_reversible_256cubed_full_size():
    # the crowded reversible workload at its full size: 256^3 with reflective
    # walls, 30 % immobile crowders, A 5 % (5 um^2/s), B 1 % (1 um^2/s),
    # A + B <-> C (kf = 1e-19 m^3/s, kb = 10 /s, C 0.5 um^2/s).  200 events:
    # A's list is re-sorted after 64 of its events, every A and B event reacts
    # (reconcile passes over lists sized for the lattice), C molecules fire
    # back (births); hash claim tables at this size
    V = 256 ** 3
    g, o = build_both((256, 256, 256), lambda L: models.crowded_reversible(L, V), 1, boundary=0)
    for chunk in (5, 70, 125):
        g.run_events(chunk)
        o.run_events(chunk)
        assert_same(g, o, chunk)
    st = o.stats()
    assert st["reactions2"] > 0 and st["reactions1"] > 0


@pytest.mark.slow
def test_mapk_like_200cubed_full_size():
    # the MAPK-like cascade at its full size: 200^3 periodic, three tiers of
    # dual phosphorylation with phosphatases (22 species, 30 reactions, counts,
    # D and rates drawn from the seed); 10^4 events (about 14 ms of simulated
    # time) cross many re-sorts of the fastest species, and complexes form,
    # dissociate and convert (reconcile passes, births)
    g, o = build_both((200, 200, 200), lambda L: models.mapk_like(L, 5), 1)
    for chunk in (10, 1990, 8000):
        g.run_events(chunk)
        o.run_events(chunk)
        assert_same(g, o, chunk)
    st = o.stats()
    assert st["reactions2"] > 0 and st["reactions1"] > 0


# Owner-computes tile kernel (forced on, with a given number of boxes): every
# stretch scatters the list into boxes, runs, and gathers it back; molecules
# cross boxes every event.  Shapes: periodic with whole bricks, reflective
# ragged, one periodic axis; densities from sparse to crowded.
TILE_CASES = [
    ((48, 44, 40), psc.PERIODIC_ALL, 0.01, 1),
    ((48, 44, 40), psc.PERIODIC_ALL, 0.05, 8),
    ((48, 44, 40), psc.PERIODIC_ALL, 0.30, 0),
    ((36, 30, 26), 0, 0.10, 0),
    ((36, 30, 26), 0, 0.60, 5),
    ((40, 30, 22), psc.PERIODIC_I, 0.20, 0),
    ((8, 8, 4), psc.PERIODIC_ALL, 0.25, 0),
]


@pytest.mark.parametrize("claim_table", [1, 2])
@pytest.mark.parametrize("shape,boundary,frac,regions", TILE_CASES)
def test_tile_kernel_matches_oracle(shape, boundary, frac, regions, claim_table):
    n = max(1, int(frac * shape[0] * shape[1] * shape[2]))
    g, o = build_both(shape, lambda L: models.diffusion_only(L, n), 21, boundary=boundary,
                      claim_table=claim_table, tiles=1, tile_regions=regions)
    for chunk in (1, 7, 40):
        g.run_events(chunk)
        o.run_events(chunk)
        assert_same(g, o, chunk)


# The lean tile kernel (HCP lattices of whole bricks, boxes of two or more
# bricks, several boxes along periodic axes): the same cases with both tile
# kernels forced, each bit-exact against the oracle, and the lean kernel
# shown to have run where it applies.
LEAN_CASES = [
    ((64, 64, 64), psc.PERIODIC_ALL, 0.30, 12),
    ((96, 64, 40), psc.PERIODIC_ALL, 0.01, 16),
    ((96, 64, 40), psc.PERIODIC_ALL, 0.05, 0),
    ((48, 40, 36), 0, 0.10, 0),
    ((48, 40, 36), 0, 0.60, 5),
    ((40, 32, 22), psc.PERIODIC_I, 0.20, 12),
    ((32, 24, 18), psc.PERIODIC_J | psc.PERIODIC_K, 0.15, 18),
    ((56, 48, 30), psc.PERIODIC_I | psc.PERIODIC_K, 0.02, 27),
]


@pytest.mark.parametrize("lean", [1, -1])
@pytest.mark.parametrize("shape,boundary,frac,regions", LEAN_CASES)
def test_lean_tile_kernel_matches_oracle(shape, boundary, frac, regions, lean):
    n = max(1, int(frac * shape[0] * shape[1] * shape[2]))
    g, o = build_both(shape, lambda L: models.diffusion_only(L, n), 31, boundary=boundary,
                      claim_table=1, tiles=1, tile_regions=regions, tile_lean=lean, time_kernels=1)
    for chunk in (1, 6, 45):
        g.run_events(chunk)
        o.run_events(chunk)
        assert_same(g, o, chunk)
    kt = g.kernel_times()
    assert kt["tile_events"] == 52
    assert (kt["tile_lean_events"] == 52) if lean > 0 else (kt["tile_lean_events"] == 0)


def _walkers_and_crowders(L, V):
    # immobile crowders, two walker species with different hop intervals
    L.add_species(0.0, int(0.2 * V))
    L.add_species(2e-12, int(0.03 * V))
    L.add_species(5e-12, int(0.02 * V))


@pytest.mark.parametrize("claim_table", [1, 2])
def test_tile_kernel_interleaved_species_with_crowders(claim_table):
    shape = (44, 40, 36)
    V = shape[0] * shape[1] * shape[2]
    g, o = build_both(shape, lambda L: _walkers_and_crowders(L, V), 4, claim_table=claim_table, tiles=1)
    for chunk in (5, 60):
        g.run_events(chunk)
        o.run_events(chunk)
        assert_same(g, o, chunk)


# FCC lattice (App. B): the per-event kernels (reactions), the molecule-list
# persistent kernel and the tile kernel (walkers), periodic with k a multiple
# of 3 and reflective ragged shapes.
FCC_CASES = [
    ((24, 24, 24), psc.PERIODIC_ALL | psc.FCC, "ab"),
    ((48, 40, 30), psc.PERIODIC_ALL | psc.FCC, "walk"),
    ((37, 29, 23), psc.FCC, "walk"),
    ((30, 28, 27), psc.FCC, "crowded"),
    ((24, 20, 18), psc.PERIODIC_ALL | psc.FCC, "mapk"),
]


@pytest.mark.parametrize("persistent", [1, -1])
@pytest.mark.parametrize("shape,boundary,model", FCC_CASES)
def test_fcc_lattice_matches_oracle(shape, boundary, model, persistent):
    V = shape[0] * shape[1] * shape[2]
    recipe = {
        "ab": lambda L: models.reaction_diffusion_ab(L, 600, 500, k=5e-19),
        "walk": lambda L: models.diffusion_only(L, int(0.1 * V)),
        "crowded": lambda L: models.crowded_reversible(L, V, kb=2000.0),
        "mapk": lambda L: models.mapk_like(L, 5, scale=0.1, uni_scale=300, bi_scale=3),
    }[model]
    g, o = build_both(shape, recipe, 13, boundary=boundary, persistent=persistent, tiles=1)
    for chunk in (3, 30, 90):
        g.run_events(chunk)
        o.run_events(chunk)
        assert_same(g, o, chunk)


# The tile kernel on FCC lattices: stencil and neighbourhood masks by layer
# class k mod 3; periodic k a multiple of 6 (whole bricks and whole ABC
# periods), reflective ragged shapes, one box or many, sparse to crowded.
FCC_TILE_CASES = [
    ((48, 44, 42), psc.PERIODIC_ALL | psc.FCC, 0.02, 0),
    ((48, 44, 42), psc.PERIODIC_ALL | psc.FCC, 0.30, 8),
    ((40, 36, 30), psc.PERIODIC_ALL | psc.FCC, 0.10, 1),
    ((37, 29, 23), psc.FCC, 0.05, 0),
    ((37, 29, 23), psc.FCC, 0.55, 5),
    ((40, 30, 25), psc.PERIODIC_I | psc.FCC, 0.20, 0),
]


@pytest.mark.parametrize("claim_table", [1, 2])
@pytest.mark.parametrize("shape,boundary,frac,regions", FCC_TILE_CASES)
def test_tile_kernel_fcc_matches_oracle(shape, boundary, frac, regions, claim_table):
    n = max(1, int(frac * shape[0] * shape[1] * shape[2]))
    g, o = build_both(shape, lambda L: models.diffusion_only(L, n), 23, boundary=boundary,
                      claim_table=claim_table, tiles=1, tile_regions=regions, time_kernels=1)
    for chunk in (1, 7, 40):
        g.run_events(chunk)
        o.run_events(chunk)
        assert_same(g, o, chunk)
    assert g.kernel_times()["tile_launches"] > 0


def test_tile_kernel_above_molecule_list_capacity():
    # 256^3 periodic at 25 % occupancy: 4,194,304 walkers, more than the
    # molecule-list kernel holds (16 per thread); the tile kernel takes them
    # by default, the per-event kernels when stretches are off
    shape = (256, 256, 256)
    n = 256 ** 3 // 4
    o = oracle.Lattice(*shape, 1e-8, oracle.PERIODIC_ALL, oracle.RULE_SYNC)
    models.diffusion_only(o, n)
    o.populate(8)
    o.run_events(6)
    for persistent in (0, -1):
        g = psc.Lattice(*shape, voxel_radius=1e-8)
        models.diffusion_only(g, n)
        g.set_options(time_kernels=1, **({"persistent": persistent} if persistent else {}))
        g.populate(8)
        g.run_events(6)
        assert_same(g, o, persistent)
        kt = g.kernel_times()
        if persistent == 0:
            assert kt["tile_events"] == 6
        else:
            assert kt["tile_events"] == 0 and kt["claim_launches"] == 6
        g.close()


@pytest.mark.parametrize("claim_table", [1, 2])
def test_many_reactions_per_event(claim_table):
    # A + B -> C with p_AB clamped to 1 and A + C -> D, both at 20 % on a ragged
    # periodic lattice: thousands of molecules react in every early event, so
    # the list upkeep has thousands of leavers and holes to fill per event
    shape = (46, 44, 40)
    V = shape[0] * shape[1] * shape[2]

    def recipe(L):
        a = L.add_species(2e-12, int(0.2 * V))
        b = L.add_species(1e-12, int(0.2 * V))
        c = L.add_species(0.5e-12, 0)
        d = L.add_species(0.0, 0)
        L.add_reaction([a, b], [c], 1e-17)
        L.add_reaction([a, c], [d], 1e-17)
        L.add_reaction([c], [a, b], 50.0)

    g, o = build_both(shape, recipe, 29, claim_table=claim_table)
    for chunk in (1, 2, 5, 20):
        g.run_events(chunk)
        o.run_events(chunk)
        assert_same(g, o, chunk)
    st = o.stats()
    assert st["reactions2"] > 10000
