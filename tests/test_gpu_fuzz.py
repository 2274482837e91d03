"""Randomised reaction models, bit for bit against the oracle.

Each seed draws a ragged lattice and walls, two to six species (some
immobile), their counts, and a set of first- and second-order reactions with
zero to two products each (Sec. 2.4: products on the partner's voxel, then on
the mover's, a second first-order product on a vacant neighbour), within the
limits the library documents.  The whole state is compared with the oracle's
synchronous rule every 60 events.  Together the seeds reach every branch of the
event kernels' reaction paths: the due species' own list kept by its commit,
partner lists reconciled, products appended, births, one-block events for
short lists and the grid classes of growing and shrinking lists.  A second
set adds compartments (slabs, a round cell or voxel noise; Sec. 2) and FCC
lattices, and checks that the library accepts and refuses every step of the
model exactly as the oracle does.  A third set runs diffusion workloads (whole
or partial bricks, walls, crowders, several walkers, a drawn box count) on
both owner-computes tile kernels, and a fourth the same kind of workloads
under the sub-volume rule (Sec. 2.5) against the oracle's sub-volume mode;
and the first set's models also run as members of one batch.
"""
import random

import numpy as np
import pytest

import models
import oracle
import paper_1605_03726_gb300 as psc
from test_gpu_parity import assert_same, build_both

pytestmark = pytest.mark.gpu


def random_model(seed):
    """(shape, walls, recipe) of seed: the recipe replays the same model on
    the GPU lattice and on the oracle."""
    rnd = random.Random(seed)
    shape = (rnd.choice([16, 20, 24, 28, 32, 36]), rnd.choice([16, 18, 20, 24, 28]),
             rnd.choice([16, 18, 20, 22, 24, 30]))
    V = shape[0] * shape[1] * shape[2]
    walls = rnd.randrange(8)
    ns = rnd.randint(2, 6)
    D = [0.0 if (s > 0 and rnd.random() < 0.25) else rnd.choice([0.3e-12, 1e-12, 3e-12]) for s in range(ns)]
    counts = [int(V * rnd.uniform(0.0, 0.07)) for _ in range(ns)]
    reactions = []
    pairs = set()
    for s in range(ns):
        if D[s] == 0.0:
            continue
        for _ in range(rnd.choice([0, 0, 1, 2])):              # first order (mobile reactant)
            prods = [rnd.randrange(ns) for _ in range(rnd.choice([0, 1, 1, 2]))]
            reactions.append(([s], prods, rnd.uniform(50.0, 1500.0)))
    for _ in range(rnd.randint(0, 4)):                          # second order
        a, b = rnd.sample(range(ns), 2)
        if (min(a, b), max(a, b)) in pairs or (D[a] == 0.0 and D[b] == 0.0):
            continue
        pairs.add((min(a, b), max(a, b)))
        prods = [rnd.randrange(ns) for _ in range(rnd.choice([0, 1, 1, 2]))]
        reactions.append(([a, b], prods, 10.0 ** rnd.uniform(-20.5, -18.5)))

    def recipe(L):
        for s in range(ns):
            L.add_species(D[s], counts[s])
        for r, p, k in reactions:
            L.add_reaction(r, p, k)

    return shape, walls, recipe, len(reactions)


@pytest.mark.parametrize("seed", range(64))
def test_random_reaction_models(seed):
    shape, walls, recipe, n_rx = random_model(seed)
    g, o = build_both(shape, recipe, 100 + seed, boundary=walls)
    for step in range(3):
        g.run_events(60)
        o.run_events(60)
        assert_same(g, o, "seed %d (%d reactions) after %d events" % (seed, n_rx, 60 * (step + 1)))


def _outcome(fn, *args, **kw):
    """(return value, None) or (None, status code of the refusal)"""
    try:
        return fn(*args, **kw), None
    except (psc.EngineError, oracle.OracleError) as e:
        return None, e.rc


def random_compartment_model(seed):
    """Ops of a seeded model with compartments (slabs, a round cell or voxel
    noise), species placed in them and random reactions, on an HCP or FCC
    lattice; the library must accept and refuse exactly what the oracle does."""
    rnd = random.Random(10_000 + seed)
    shape = (rnd.choice([16, 20, 24]), rnd.choice([16, 18, 24]), rnd.choice([12, 18, 24]))
    ni, nj, nk = shape
    V = ni * nj * nk
    flags = rnd.randrange(8) | (oracle.FCC if rnd.random() < 0.3 else 0)
    kind = rnd.choice(["slabs", "cell", "noise"])
    if kind == "slabs":
        nc = rnd.randint(2, 3)
        axis = rnd.randrange(3)
        idx = np.indices((nk, nj, ni))[2 - axis].reshape(-1)
        lab = (idx * nc // shape[axis]).astype(np.uint8)
    elif kind == "cell":
        nc = 3
        lab = models.cell_labels(ni, nj, nk, radius=rnd.uniform(8.0, 14.0))
    else:
        nc = rnd.randint(2, 4)
        lab = np.random.default_rng(seed).integers(0, nc, V).astype(np.uint8)
    ns = rnd.randint(2, 5)
    species = [(0.0 if (s > 0 and rnd.random() < 0.2) else rnd.choice([0.5e-12, 1e-12, 3e-12]),
                int(V * rnd.uniform(0.0, 0.05)), rnd.randrange(nc)) for s in range(ns)]
    comp = [c for _, _, c in species]

    def in_comp(c):
        # a species of compartment c, or any species when none is there (the
        # model may then be refused, as it must be on both sides)
        pool = [s for s in range(ns) if comp[s] == c]
        return rnd.choice(pool) if pool and rnd.random() < 0.8 else rnd.randrange(ns)

    reactions = []
    for _ in range(rnd.randint(1, 6)):
        npr = rnd.choice([0, 1, 1, 2])
        if rnd.random() < 0.4:
            r = [rnd.randrange(ns)]
            k = rnd.uniform(50.0, 1500.0)
            prods = [in_comp(comp[r[0]]) for _ in range(npr)]
        else:
            r = rnd.sample(range(ns), 2)
            k = 10.0 ** rnd.uniform(-20.5, -18.5)
            prods = [in_comp(comp[r[1]]), in_comp(comp[r[0]])][:npr]
        reactions.append((r, prods, k))
    return shape, flags, lab, nc, species, reactions


@pytest.mark.parametrize("seed", range(48))
def test_random_models_with_compartments(seed):
    shape, flags, lab, nc, species, reactions = random_compartment_model(seed)
    (g, eg), (o, eo) = (_outcome(psc.Lattice, *shape, voxel_radius=1e-8, boundary=flags),
                        _outcome(oracle.Lattice, *shape, 1e-8, flags, oracle.RULE_SYNC))
    assert eg == eo, (seed, eg, eo)
    if eg is not None:
        return                                   # both refuse the lattice (e.g. periodic FCC k)
    assert _outcome(g.set_compartments, lab, nc)[1] == _outcome(o.set_compartments, lab, nc)[1]
    for D, n, c in species:
        sg, sg_err = _outcome(g.add_species, D, n, compartment=c)
        so, so_err = _outcome(o.add_species, D, n)
        if so_err is None:
            so_err = _outcome(o.species_compartment, so, c)[1]
        assert sg_err == so_err, (seed, sg_err, so_err)
    for r, p, k in reactions:
        assert _outcome(g.add_reaction, r, p, k)[1] == _outcome(o.add_reaction, r, p, k)[1], (seed, r, p)
    rg, eg = _outcome(g.populate, 200 + seed)
    ro, eo = _outcome(o.populate, 200 + seed)
    assert (rg, eg) == (ro, eo), seed
    if eg is None:
        assert_same(g, o, "seed %d populate" % seed)
        for step in range(3):
            g.run_events(50)
            o.run_events(50)
            assert_same(g, o, "seed %d after %d events" % (seed, 50 * (step + 1)))
    g.close()
    o.close()


def random_tile_case(seed):
    """A seeded diffusion workload for the owner-computes tile kernels: shape
    (whole or partial bricks), walls, occupancy, crowders and box count."""
    rnd = random.Random(20_000 + seed)
    ni = rnd.choice([24, 32, 40, 48, 64, 30, 38])
    nj = rnd.choice([16, 24, 32, 40, 22, 34])
    nk = rnd.choice([12, 16, 20, 24, 30, 40])
    walls = rnd.randrange(8)
    V = ni * nj * nk
    crowd = rnd.choice([0.0, 0.0, 0.1, 0.3])
    walkers = [(rnd.choice([1e-12, 2e-12, 5e-12]), int(V * rnd.uniform(0.005, 0.15)))
               for _ in range(rnd.randint(1, 2))]
    regions = rnd.choice([0, 0, 4, 8, 12, 16, 27])

    def recipe(L):
        if crowd:
            L.add_species(0.0, int(crowd * V))
        for D, n in walkers:
            L.add_species(D, n)

    return (ni, nj, nk), walls, recipe, regions


@pytest.mark.parametrize("lean", [1, -1])
@pytest.mark.parametrize("seed", range(24))
def test_random_tile_kernel_workloads(seed, lean):
    shape, walls, recipe, regions = random_tile_case(seed)
    g, o = build_both(shape, recipe, 300 + seed, boundary=walls, tiles=1, tile_regions=regions, tile_lean=lean)
    for chunk in (1, 9, 30):
        g.run_events(chunk)
        o.run_events(chunk)
        assert_same(g, o, "seed %d lean %d after chunk %d" % (seed, lean, chunk))


def random_subvolume_case(seed):
    """A seeded workload for the sub-volume rule: shape (periodic axes a
    multiple of 4), walls, immobile crowders and one to three walker species
    with different hop intervals."""
    rnd = random.Random(30_000 + seed)
    walls = rnd.randrange(8)
    dims = []
    for a in range(3):
        choices = [16, 20, 24, 32] if walls & (1 << a) else [14, 18, 22, 26, 30]
        dims.append(rnd.choice(choices))
    V = dims[0] * dims[1] * dims[2]
    crowd = rnd.choice([0.0, 0.15, 0.3])
    walkers = [(rnd.choice([0.5e-12, 1e-12, 4e-12]), int(V * rnd.uniform(0.01, 0.2)))
               for _ in range(rnd.randint(1, 3))]

    def recipe(L):
        if crowd:
            L.add_species(0.0, int(crowd * V))
        for D, n in walkers:
            L.add_species(D, n)

    return tuple(dims), walls, recipe


@pytest.mark.parametrize("seed", range(16))
def test_random_subvolume_workloads(seed):
    shape, walls, recipe = random_subvolume_case(seed)
    g = psc.Lattice(*shape, voxel_radius=1e-8, boundary=walls)
    g.set_options(subvolume=1)
    o = oracle.Lattice(*shape, 1e-8, walls, oracle.RULE_SUBVOL)
    recipe(g)
    recipe(o)
    assert g.populate(400 + seed) == o.populate(400 + seed)
    assert_same(g, o, "populate")
    for chunk in (1, 9, 30):
        g.run_events(chunk)
        o.run_events(chunk)
        assert_same(g, o, "seed %d after chunk %d" % (seed, chunk))


def test_random_reaction_models_in_one_batch():
    """The randomised reaction models of the first set as members of one batch
    (one launch per event phase over all members), each bit-exact with the
    oracle at every checkpoint."""
    import torch
    stream = torch.cuda.Stream()
    B = psc.Batch(stream=stream.cuda_stream)
    pairs = []
    for seed in range(24):
        shape, walls, recipe, _ = random_model(seed)
        g = psc.Lattice(*shape, voxel_radius=1e-8, boundary=walls, stream=stream.cuda_stream)
        g.set_options(claim_table=1)
        o = oracle.Lattice(*shape, 1e-8, walls, oracle.RULE_SYNC)
        recipe(g)
        recipe(o)
        assert g.populate(100 + seed) == o.populate(100 + seed)
        B.add(g)
        pairs.append((seed, g, o))
    for chunk in (20, 40, 60):
        B.run_events(chunk)
        torch.cuda.synchronize()
        for seed, g, o in pairs:
            o.run_events(chunk)
            assert_same(g, o, "batch member %d after chunk %d" % (seed, chunk))
    B.close()
