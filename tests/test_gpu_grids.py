"""Lists whose length crosses the engine's grid classes during a run.

Per-event launches of a species with reactions take a grid sized from a
background estimate of its list length, and lists of a few hundred molecules
run a whole event in one block.  Estimates lag the device, so a list can be
served by a grid (or a single block) far too small for it for a while; the
kernels stride over the count in device memory, so results must not change.
Here one list grows a hundredfold (a first-order split A -> A + A) while its
partner shrinks, and in the other case a large list decays to a few dozen
molecules; both are compared bit for bit with the oracle every 50 events,
with CUDA-graph replay on (the default) and off.
"""
import pytest

from test_gpu_parity import assert_same, build_both

pytestmark = pytest.mark.gpu

TAU_A = 6.666666666666667e-05        # hop interval of a species with D = 1 um^2/s at r_v = 10 nm


def growing(L):
    a = L.add_species(1e-12, 100)
    b = L.add_species(0.5e-12, 300)
    c = L.add_species(0.0, 0)
    L.add_reaction([a], [a, a], 0.014 / TAU_A)     # about 1.4 % of A splits per event of A
    L.add_reaction([a, b], [c], 1e-19)


def decaying(L):
    a = L.add_species(1e-12, 20000)
    b = L.add_species(0.5e-12, 300)
    L.add_reaction([a], [], 0.012 / TAU_A)
    L.add_reaction([a, b], [b], 1e-19)


@pytest.mark.parametrize("graphs", [32, -1])
@pytest.mark.parametrize("recipe,seed", [(growing, 3), (decaying, 5)])
def test_lists_crossing_grid_classes(recipe, seed, graphs):
    g, o = build_both((48, 48, 48), recipe, seed, boundary=7, graph_events=graphs)
    assert g.tau(0) == o.tau(0) == pytest.approx(TAU_A)
    first = o.counts()[0]
    for step in range(12):
        g.run_events(50)
        o.run_events(50)
        assert_same(g, o, "after %d events" % (50 * (step + 1)))
    last = o.counts()[0]
    # the list really crossed the classes (4, 32, 256 blocks, full grid)
    assert (last > 100 * first) if recipe is growing else (last * 100 < first)
