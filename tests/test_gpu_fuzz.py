"""Randomised reaction models, bit for bit against the oracle.

Each seed draws a ragged lattice and walls, two to six species (some
immobile), their counts, and a set of first- and second-order reactions with
zero to two products each (Sec. 2.4: products on the partner's voxel, then on
the mover's, a second first-order product on a vacant neighbour), within the
limits the library documents.  The whole state is compared with the oracle's
synchronous rule every 60 events.  Together the seeds reach every branch of the
event kernels' reaction paths: the due species' own list kept by its commit,
partner lists reconciled, products appended, births, one-block events for
short lists and the grid classes of growing and shrinking lists.
"""
import random

import pytest

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
