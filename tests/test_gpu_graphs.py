"""Per-event runs replayed from CUDA graphs (psc_options.graph_events, on by
default) give the same lattice as ordinary launches (graph_events = -1) and as
the oracle, whatever the run length, the claim tables, the re-sort period or
the species mix; options set between runs drop the captured graphs; with
kernel timing on, graphs stay off.
"""
import numpy as np
import pytest

import oracle
import paper_1605_03726_gb300 as psc
import models

pytestmark = pytest.mark.gpu


def state(L, ns):
    return (L.grid().copy(), [L.coords(s) for s in range(ns)], [L.unwrapped(s)[0] for s in range(ns)],
            L.event_index(), L.time(), L.counts().copy())


def same(a, b, tag=""):
    assert np.array_equal(a[0], b[0]), tag
    for (x, y), (u, v) in zip(a[1], b[1]):
        assert np.array_equal(x, u) and np.array_equal(y, v), tag
    for x, u in zip(a[2], b[2]):
        assert np.array_equal(x, u), tag
    assert a[3] == b[3] and a[4] == b[4] and np.array_equal(a[5], b[5]), tag


CASES = [
    ("ab", (64, 64, 64), psc.PERIODIC_ALL, lambda L: models.reaction_diffusion_ab(L, 2000, 2000), 3),
    ("crowded", (40, 36, 32), 0, lambda L: models.crowded_reversible(L, 40 * 36 * 32, kb=2000.0), 4),
    ("mapk", (48, 48, 48), psc.PERIODIC_ALL,
     lambda L: models.mapk_like(L, 2, scale=0.05, uni_scale=300, bi_scale=3), 22),
]


@pytest.mark.parametrize("k", [2, 16, 64])
@pytest.mark.parametrize("claim_table", [1, 2])
@pytest.mark.parametrize("name,shape,bnd,recipe,ns", CASES)
def test_graph_replay_matches_ordinary_launches_and_oracle(name, shape, bnd, recipe, ns, claim_table, k):
    runs = {}
    for graphs in (0, k):
        L = psc.Lattice(*shape, voxel_radius=1e-8, boundary=bnd)
        L.set_options(claim_table=claim_table, resort_period=24, graph_events=graphs or -1)
        recipe(L)
        L.populate(6)
        for chunk in (5, 200, 333):
            L.run_events(chunk)
        st = L.stats()
        runs[graphs] = (state(L, ns), st["launches"])
        L.close()
    same(runs[0][0], runs[k][0], name)
    o = oracle.Lattice(*shape, 1e-8, bnd, oracle.RULE_SYNC)
    recipe(o)
    o.populate(6)
    o.run_events(538)
    assert np.array_equal(o.grid(), runs[k][0][0])
    for s in range(ns):
        a, b = o.coords(s), runs[k][0][1][s]
        assert np.array_equal(a[0], b[0]) and np.array_equal(a[1], b[1])


def test_graphs_replay_and_follow_option_changes():
    shape = (64, 64, 64)
    L = psc.Lattice(*shape, voxel_radius=1e-8)
    U = psc.Lattice(*shape, voxel_radius=1e-8)
    for M in (L, U):
        models.reaction_diffusion_ab(M, 2000, 2000)
        M.populate(2)
    L.set_options(graph_events=32)
    U.set_options(graph_events=-1)                   # ordinary launches
    L.run(0.02)
    U.run(0.02)
    same(state(L, 3), state(U, 3), "run to t")
    # replays: runs of 32 events recur every re-sort period
    L.run_events(64 * 8)
    U.run_events(64 * 8)
    same(state(L, 3), state(U, 3), "replays")
    # options that change the launches drop the graphs; results stay the same
    L.set_options(block_threads=128, blocks_per_sm=4)
    U.set_options(block_threads=128, blocks_per_sm=4)
    L.run_events(300)
    U.run_events(300)
    same(state(L, 3), state(U, 3), "new launch shape")
    # kernel timing keeps graphs off
    L.set_options(time_kernels=1)
    L.run_events(64)
    U.run_events(64)
    kt = L.kernel_times()
    assert kt["claim_launches"] == 64
    same(state(L, 3), state(U, 3), "timed")
    L.close()
    U.close()


def test_graph_replay_with_compartments_and_fcc():
    # the membrane-receptor cell (reactions across compartments, births into
    # the cytoplasm) on HCP and FCC lattices: graphs or not, the same lattice
    lab_shape = [((40, 36, 32), 0), ((37, 29, 23), psc.FCC)]
    for shape, bnd in lab_shape:
        lab = models.cell_labels(*shape, radius=28.0 if bnd == 0 else 24.0)
        runs = {}
        for graphs in (0, 16):
            L = psc.Lattice(*shape, voxel_radius=1e-8, boundary=bnd)
            L.set_options(resort_period=16, graph_events=graphs or -1)
            models.receptor_binding(L, lab, 1200, 500, n_x=300, n_outside=1000, koff=2e3)
            L.populate(3)
            L.run_events(40)
            L.run_events(400)
            runs[graphs] = state(L, 5)
            L.close()
        same(runs[0], runs[16], shape)
        o = oracle.Lattice(*shape, 1e-8, bnd, oracle.RULE_SYNC)
        models.receptor_binding(o, lab, 1200, 500, n_x=300, n_outside=1000, koff=2e3)
        o.populate(3)
        o.run_events(440)
        assert np.array_equal(o.grid(), runs[16][0])
