"""Pin the FCC lattice of the oracle (App. B: the same twisted Cartesian
coordinates, ABC stacking; the appendix has only figures).

Pinned by what an FCC lattice of touching spheres must be: 12 nearest
neighbours at 2 r_v with every other voxel farther, the same packing fraction
as HCP, ABC stacking (layers k and k+3 coincide, k and k+1, k+2 do not, and
unlike HCP k and k+2 differ), a neighbour relation symmetric under periodic
wrap, exact one-diameter hops, uniform directions and MSD = 6 D t.
"""
import itertools
import math

import numpy as np
import pytest
from scipy import stats

import oracle

FCC_ALL = oracle.PERIODIC_ALL | oracle.FCC


def _centres(ni, nj, nk):
    c = np.zeros((ni, nj, nk, 3))
    for i, j, k in itertools.product(range(ni), range(nj), range(nk)):
        c[i, j, k] = oracle.center_fcc(i, j, k)
    return c


def sqdisp3(a, b):
    d = b.astype(np.int64) - a.astype(np.int64)
    return 3 * d[:, 0] ** 2 + d[:, 1] ** 2 + 8 * d[:, 2] ** 2


@pytest.mark.parametrize("dims", [(6, 6, 6), (5, 4, 9), (3, 8, 3)])
def test_fcc_stencil_is_the_twelve_nearest_voxels(golden, dims):
    ni, nj, nk = dims
    L = oracle.Lattice(ni, nj, nk, 1e-8, FCC_ALL)
    cen = _centres(ni, nj, nk)
    A = np.array(oracle.center_fcc(ni, 0, 0)) - oracle.center_fcc(0, 0, 0)
    B = np.array(oracle.center_fcc(0, nj, 0)) - oracle.center_fcc(0, 0, 0)
    C = np.array(oracle.center_fcc(0, 0, nk)) - oracle.center_fcc(0, 0, 0)
    flat = cen.transpose(2, 1, 0, 3).reshape(-1, 3)
    shifts = [a * A + b * B + c * C for a in (-1, 0, 1) for b in (-1, 0, 1) for c in (-1, 0, 1)]
    for i, j, k in itertools.product(range(ni), range(nj), range(nk)):
        d = np.min([np.linalg.norm(flat + s - cen[i, j, k], axis=1) for s in shifts], axis=0)
        v = i + ni * (j + nj * k)
        d[v] = np.inf
        nearest = set(np.flatnonzero(np.abs(d - 2.0) < 1e-9).tolist())
        assert len(nearest) == golden["hcp_neighbours"]            # 12, as for HCP
        assert d.min() == pytest.approx(2.0)
        stencil = set()
        for dd in range(12):
            inside, o, _ = L.neighbor(i, j, k, dd)
            assert inside
            stencil.add(o[0] + ni * (o[1] + nj * o[2]))
        assert stencil == nearest


def test_fcc_packing_fraction_matches_paper(golden):
    # Sec. 2.1: FCC has the same density as HCP (the printed 74.048 %)
    A = np.array(oracle.center_fcc(1, 0, 0)) - oracle.center_fcc(0, 0, 0)
    B = np.array(oracle.center_fcc(0, 2, 0)) - oracle.center_fcc(0, 0, 0)
    C = np.array(oracle.center_fcc(0, 0, 3)) - oracle.center_fcc(0, 0, 0)
    vol = abs(np.linalg.det(np.array([A, B, C]))) / 6.0      # 6 voxels in that cell
    frac = (4.0 / 3.0) * math.pi / vol
    assert vol == pytest.approx(4 * math.sqrt(2))
    assert frac == pytest.approx(golden["hcp_packing_fraction"], abs=1e-5)


def test_fcc_is_abc_stacking_not_abab():
    off = [np.array(oracle.center_fcc(0, 0, k))[:2] for k in range(6)]
    for k in range(3):
        assert np.allclose(off[k], off[k + 3])                      # period three
    assert not np.allclose(off[0], off[1]) and not np.allclose(off[0], off[2])
    assert not np.allclose(off[1], off[2])
    hcp = [np.array(oracle.center(0, 0, k))[:2] for k in range(3)]
    assert np.allclose(hcp[0], hcp[2])                              # HCP: ABAB


def test_fcc_neighbour_relation_symmetric():
    ni, nj, nk = 5, 6, 6
    L = oracle.Lattice(ni, nj, nk, 1e-8, FCC_ALL)
    for i, j, k in itertools.product(range(ni), range(nj), range(nk)):
        for d in range(12):
            _, o, w = L.neighbor(i, j, k, d)
            back = set()
            for d2 in range(12):
                _, o2, w2 = L.neighbor(o[0], o[1], o[2], d2)
                if tuple(o2) == (i, j, k) and all(a + b == 0 for a, b in zip(w, w2)):
                    back.add(d2)
            assert len(back) == 1


def test_fcc_rejects_periods_that_break_the_stacking():
    with pytest.raises(oracle.OracleError):
        oracle.Lattice(6, 6, 4, 1e-8, FCC_ALL)                      # k period not a multiple of 3
    oracle.Lattice(6, 6, 3, 1e-8, FCC_ALL).close()
    oracle.Lattice(6, 6, 5, 1e-8, oracle.FCC).close()               # reflective k: any extent


def test_fcc_hops_are_one_diameter_and_uniform():
    L = oracle.Lattice(48, 48, 48, 1e-8, FCC_ALL)
    s = L.add_species(1e-12, 3000)
    L.populate(5)
    before, _ = L.unwrapped(s)
    by_layer = {0: {}, 1: {}, 2: {}}
    for _ in range(40):
        L.run_events(1)
        after, _ = L.unwrapped(s)
        q = sqdisp3(before, after)
        assert set(np.unique(q).tolist()) <= {0, 12}
        d = after.astype(np.int64) - before
        moved = q == 12
        for src, dv in zip(before[moved], d[moved]):
            key = tuple(int(x) for x in dv)
            c = int(src[2]) % 3
            by_layer[c][key] = by_layer[c].get(key, 0) + 1
        before = after
    assert L.check() == 0
    for c, cnt in by_layer.items():
        assert len(cnt) == 12
        assert stats.chisquare(list(cnt.values())).pvalue > 0.01


def test_fcc_msd_equals_6Dt_for_isolated_walkers(golden):
    rv, D, n_events = 5e-9, 10e-12, 64
    msd = []
    for seed in (1, 2):
        L = oracle.Lattice(192, 192, 192, rv, FCC_ALL)
        s = L.add_species(D, 32768)
        L.populate(seed)
        x0, _ = L.unwrapped(s)
        L.run_events(n_events)
        x1, _ = L.unwrapped(s)
        t_end = L.time()
        msd.append(sqdisp3(x0, x1) / 3.0 * rv * rv)
        L.close()
    msd = np.concatenate(msd)
    theory = golden["es_coefficient"] * D * t_end
    assert msd.mean() / theory == pytest.approx(1.0, abs=0.012)
