"""Slabs of a lattice along k with ghost layers (Sec. 2.5's sub-domains) on one GPU.

The lattice is split into slabs that exchange, at every event, the claims on
the layers at each face and then the molecules that crossed with the
refreshed boundary layers.  Several slabs held by one process exchange by
device copies; the results must equal the oracle's synchronous rule on the
whole lattice bit for bit: every molecule's position, id and unwrapped
position.  Also: one slab on a periodic axis (its own neighbour), caller-owned
exchange buffers driven through the per-rank protocol, the refusals, and
randomised splits (shapes, walls, slab counts, crowders, occupancy).
"""
import numpy as np
import pytest

import oracle
import paper_1605_03726_gb300 as psc

pytestmark = pytest.mark.gpu


def _models(L, V, crowd, frac, D=2e-12):
    if crowd:
        L.add_species(0.0, int(crowd * V))
    return L.add_species(D, int(frac * V))


def _gather(slabs):
    ijk, ids, xyz = zip(*(s.coords() for s in slabs))
    ijk, ids, xyz = np.concatenate(ijk), np.concatenate(ids), np.concatenate(xyz)
    order = np.argsort(ids, kind="stable")
    return ijk[order], ids[order], xyz[order]


def _same(slabs, o, species, tag):
    ijk, ids, xyz = _gather(slabs)
    oi, oid = o.coords(species)
    ou, _ = o.unwrapped(species)
    assert np.array_equal(ids, oid), tag
    assert np.array_equal(ijk, oi), tag
    assert np.array_equal(xyz, ou), tag


SLAB_CASES = [
    ((48, 40, 24), psc.PERIODIC_ALL, 2, 0.0, 0.05),
    ((48, 40, 24), psc.PERIODIC_ALL, 3, 0.0, 0.30),
    ((40, 32, 30), 0, 3, 0.2, 0.10),
    ((40, 32, 32), psc.PERIODIC_J | psc.PERIODIC_K, 4, 0.1, 0.15),
    ((36, 30, 20), psc.PERIODIC_I, 5, 0.0, 0.60),
    ((32, 32, 16), psc.PERIODIC_ALL, 1, 0.0, 0.10),
    ((32, 28, 12), 0, 1, 0.05, 0.20),
    ((40, 36, 24), psc.PERIODIC_I | psc.PERIODIC_J, 6, 0.0, 0.35),
]


@pytest.mark.parametrize("shape,boundary,count,crowd,frac", SLAB_CASES)
def test_slabs_match_oracle(shape, boundary, count, crowd, frac):
    V = shape[0] * shape[1] * shape[2]
    L = psc.Lattice(*shape, voxel_radius=1e-8, boundary=boundary)
    o = oracle.Lattice(*shape, 1e-8, boundary, oracle.RULE_SYNC)
    s = _models(L, V, crowd, frac)
    _models(o, V, crowd, frac)
    L.populate(17)
    o.populate(17)
    L.run_events(3)                           # the slabs start from a lattice mid-run
    o.run_events(3)
    slabs = [psc.Slab(L, s, q, count) for q in range(count)]
    assert all(sl.event_index() == 3 for sl in slabs)
    for chunk in (1, 6, 40):
        psc.run_slabs(slabs, chunk)
        o.run_events(chunk)
        _same(slabs, o, s, chunk)
    assert slabs[0].event_index() == o.event_index()
    for sl in slabs:
        sl.synchronize()
        sl.close()
    L.close()


def test_slab_with_caller_buffers_through_the_rank_protocol():
    # one slab on a periodic k axis (its own neighbour), exchange buffers the
    # caller owns (torch tensors), driven by the per-rank protocol
    import torch

    shape = (40, 36, 20)
    V = shape[0] * shape[1] * shape[2]
    L = psc.Lattice(*shape, voxel_radius=1e-8)
    o = oracle.Lattice(*shape, 1e-8, oracle.PERIODIC_ALL, oracle.RULE_SYNC)
    s = _models(L, V, 0.15, 0.2)
    _models(o, V, 0.15, 0.2)
    L.populate(5)
    o.populate(5)
    # the slab's kernels and the exchange copies on one stream (a NULL stream
    # would give the slab a stream of its own, unordered with torch's)
    stream = torch.cuda.Stream()
    sl = psc.Slab(L, s, 0, 1, stream=stream.cuda_stream)
    _, claim_bytes, commit_bytes = sl.buffers()
    dev = torch.device("cuda", 0)
    mk = lambda nb: [torch.zeros(nb, dtype=torch.uint8, device=dev) for _ in (0, 1)]
    bufs = {"send_claim": mk(claim_bytes), "recv_claim": mk(claim_bytes),
            "send_commit": mk(commit_bytes), "recv_commit": mk(commit_bytes)}
    sl.set_buffers(*[[t.data_ptr() for t in bufs[k]] for k in ("send_claim", "recv_claim", "send_commit",
                                                                 "recv_commit")])
    ranks = psc.SlabRanks(0, 1, True)
    with torch.cuda.stream(stream):
        ranks.run_events(sl, bufs, 25)
    stream.synchronize()
    o.run_events(25)
    _same([sl], o, s, "rank protocol")
    sl.close()
    L.close()


def test_slab_refusals():
    L = psc.Lattice(32, 32, 18, voxel_radius=1e-8)
    a = L.add_species(1e-12, 500)
    b = L.add_species(1e-12, 500)
    c = L.add_species(0.0, 0)
    L.add_reaction([a, b], [c], 1e-19)
    L.populate(1)
    with pytest.raises(psc.EngineError) as e:
        psc.Slab(L, a, 0, 2)                  # reactions, and a second mobile species
    assert e.value.rc == psc.E_UNSUPPORTED
    L.close()
    L = psc.Lattice(32, 32, 18, voxel_radius=1e-8)
    w = L.add_species(1e-12, 500)
    L.populate(1)
    for count in (4, 18):                     # 18 / 4 not whole; 18 / 18 = one layer per slab
        with pytest.raises(psc.EngineError) as e:
            psc.Slab(L, w, 0, count)
        assert e.value.rc == psc.E_DIMS
    L.close()
    L = psc.Lattice(32, 32, 18, voxel_radius=1e-8, boundary=psc.PERIODIC_ALL | psc.FCC)
    w = L.add_species(1e-12, 500)
    L.populate(1)
    with pytest.raises(psc.EngineError) as e:
        psc.Slab(L, w, 0, 2)                  # HCP only
    assert e.value.rc == psc.E_UNSUPPORTED
    L.close()


@pytest.mark.slow
def test_slabs_at_full_size_match_the_whole_lattice():
    # the 512^3 lattice at 1 % occupancy split into four slabs of 128 layers:
    # after 30 events every molecule stands where the whole lattice's run put
    # it (the whole lattice's stretch kernels are themselves checked against
    # the oracle at this size, test_gpu_parity.py)
    n = int(0.01 * 512 ** 3)
    L = psc.Lattice(512, 512, 512, voxel_radius=1e-8)
    s = L.add_species(10e-12, n)
    L.populate(3)
    slabs = [psc.Slab(L, s, q, 4) for q in range(4)]
    psc.run_slabs(slabs, 30)
    L.run_events(30)
    ijk, ids, xyz = _gather(slabs)
    li, lid = L.coords(s)
    lu, _ = L.unwrapped(s)
    assert np.array_equal(ids, lid) and np.array_equal(ijk, li) and np.array_equal(xyz, lu)
    for sl in slabs:
        sl.close()
    L.close()


def _random_slab_case(seed):
    """A seeded slab workload: shape (nk a multiple of the slab count, every
    slab at least two layers thick), walls, crowders, occupancy, slab count."""
    import random
    rnd = random.Random(40_000 + seed)
    count = rnd.randint(1, 6)
    m = rnd.randint(2, 8)
    nk = count * m
    if nk % 2:
        nk += count                          # nk even: one more layer per slab
    walls = rnd.randrange(8)
    if walls & psc.PERIODIC_K and nk < 4:
        walls &= ~psc.PERIODIC_K
    shape = (rnd.choice([16, 20, 24, 30, 40]), rnd.choice([12, 16, 20, 28]), nk)
    return shape, walls, count, rnd.choice([0.0, 0.1, 0.3]), rnd.uniform(0.01, 0.4)


@pytest.mark.parametrize("seed", range(16))
def test_random_slab_splits_match_oracle(seed):
    shape, boundary, count, crowd, frac = _random_slab_case(seed)
    V = shape[0] * shape[1] * shape[2]
    L = psc.Lattice(*shape, voxel_radius=1e-8, boundary=boundary)
    o = oracle.Lattice(*shape, 1e-8, boundary, oracle.RULE_SYNC)
    s = _models(L, V, crowd, frac)
    _models(o, V, crowd, frac)
    L.populate(50 + seed)
    o.populate(50 + seed)
    slabs = [psc.Slab(L, s, q, count) for q in range(count)]
    for chunk in (1, 9, 30):
        psc.run_slabs(slabs, chunk)
        o.run_events(chunk)
        _same(slabs, o, s, "seed %d chunk %d" % (seed, chunk))
    for sl in slabs:
        sl.synchronize()
        sl.close()
    L.close()
