"""Pin the HCP geometry of the oracle (Sec. 2.1, twisted Cartesian coordinates).

The stencil is given in the paper only as a figure, so it is pinned by what the
lattice must be: spheres of radius r_v touching their 12 nearest neighbours at
distance 2 r_v, the HCP packing fraction the paper prints, ABAB stacking of the
k layers, and a neighbour relation that is symmetric under periodic wrap.
"""
import itertools
import math

import numpy as np
import pytest

import oracle


def _centres(ni, nj, nk):
    c = np.zeros((ni, nj, nk, 3))
    for i, j, k in itertools.product(range(ni), range(nj), range(nk)):
        c[i, j, k] = oracle.center(i, j, k)
    return c


def _periods(ni, nj, nk):
    # periodic images: shifting i by ni, j by nj (even), k by nk (even) maps the
    # lattice onto itself
    a = np.array(oracle.center(ni, 0, 0)) - oracle.center(0, 0, 0)
    b = np.array(oracle.center(0, nj, 0)) - oracle.center(0, 0, 0)
    c = np.array(oracle.center(0, 0, nk)) - oracle.center(0, 0, 0)
    return a, b, c


@pytest.mark.parametrize("dims", [(6, 6, 6), (5, 4, 8), (3, 8, 4)])
def test_stencil_is_the_twelve_nearest_voxels(golden, dims):
    ni, nj, nk = dims
    L = oracle.Lattice(ni, nj, nk, 1e-8, oracle.PERIODIC_ALL)
    cen = _centres(ni, nj, nk)
    A, B, C = _periods(ni, nj, nk)
    flat = cen.transpose(2, 1, 0, 3).reshape(-1, 3)   # voxel index v = i + ni*(j + nj*k)
    shifts = [a * A + b * B + c * C for a in (-1, 0, 1) for b in (-1, 0, 1) for c in (-1, 0, 1)]
    for i, j, k in itertools.product(range(ni), range(nj), range(nk)):
        # brute force: minimum-image distance to every voxel
        d = np.min([np.linalg.norm(flat + s - cen[i, j, k], axis=1) for s in shifts], axis=0)
        v = i + ni * (j + nj * k)
        d[v] = np.inf
        nearest = set(np.flatnonzero(np.abs(d - 2.0) < 1e-9).tolist())
        assert len(nearest) == golden["hcp_neighbours"]
        assert d.min() == pytest.approx(2.0)            # touching spheres of radius r_v
        stencil = set()
        for dd in range(12):
            inside, o, _ = L.neighbor(i, j, k, dd)
            assert inside
            stencil.add(o[0] + ni * (o[1] + nj * o[2]))
        assert stencil == nearest


def test_packing_fraction_matches_paper(golden):
    # volume per voxel from the lattice period vectors, in units of r_v^3
    A = np.array(oracle.center(1, 0, 0)) - oracle.center(0, 0, 0)
    B = np.array(oracle.center(0, 2, 0)) - oracle.center(0, 0, 0)
    C = np.array(oracle.center(0, 0, 2)) - oracle.center(0, 0, 0)
    # the cell spanned by (A, B, C) holds 1 x 2 x 2 voxels
    vol_per_voxel = abs(np.linalg.det(np.stack([A, B, C]))) / 4.0
    assert vol_per_voxel == pytest.approx(4.0 * math.sqrt(2.0))
    frac = (4.0 / 3.0) * math.pi / vol_per_voxel
    # the paper prints five digits, truncated: allow one unit in the last digit
    assert frac == pytest.approx(golden["hcp_packing_fraction"], abs=1e-5)
    # the paper's Cartesian figure is the same computation on a cube of side 2
    assert (4.0 / 3.0) * math.pi / 8.0 == pytest.approx(golden["cartesian_packing_fraction"], abs=1e-5)


def test_abab_stacking_is_hcp_not_fcc():
    xy = lambda k: sorted((round(float(x), 9), round(float(y), 9))
                          for x, y, _ in (oracle.center(i, j, k) for i in range(4) for j in range(4)))
    # the (i, j) grid of layer k projected onto the plane: layers 0 and 2 coincide,
    # layer 1 is shifted (ABAB); an FCC stacking would need three distinct layers
    assert xy(0) == xy(2)
    assert xy(1) == xy(3)
    assert xy(0) != xy(1)
    for k in range(3):
        z = {round(float(oracle.center(i, j, k)[2]), 12) for i in range(3) for j in range(3)}
        assert len(z) == 1


def test_neighbour_relation_symmetric_and_opposites():
    ni, nj, nk = 5, 6, 8
    L = oracle.Lattice(ni, nj, nk, 1e-8, oracle.PERIODIC_ALL)
    opposite = {0: 1, 1: 0, 2: 5, 5: 2, 3: 4, 4: 3, 6: 10, 10: 6, 7: 9, 9: 7, 8: 11, 11: 8}
    for i, j, k in itertools.product(range(ni), range(nj), range(nk)):
        for d in range(12):
            _, o, w = L.neighbor(i, j, k, d)
            _, back, w2 = L.neighbor(*o, opposite[d])
            assert back == (i, j, k)
            assert tuple(-x for x in w) == w2


def test_reflective_walls_drop_out_of_box_neighbours():
    L = oracle.Lattice(4, 4, 4, 1e-8, 0)
    inside = [L.neighbor(0, 0, 0, d)[0] for d in range(12)]
    # the corner voxel keeps only the neighbours that lie inside the box
    assert sum(inside) < 12
    for d in range(12):
        ok, o, w = L.neighbor(0, 0, 0, d)
        assert w == (0, 0, 0)
        if ok:
            assert all(0 <= x < 4 for x in o)
    assert all(L.neighbor(1, 1, 1, d)[0] for d in range(12))


def test_unwrapped_basis_distance():
    # X = 2I + P, Y = 3J + (K&1), Z = K gives |r|^2 = X^2 + Y^2/3 + 8 Z^2/3 (r_v^2):
    # it must agree with the centre formula for every voxel
    for i, j, k in itertools.product(range(-3, 4), range(-3, 4), range(-3, 4)):
        c = oracle.center(i, j, k)
        X, Y, Z = 2 * i + ((j + k) & 1), 3 * j + (k & 1), k
        assert (X, Y / math.sqrt(3), Z * 2 * math.sqrt(2 / 3)) == pytest.approx(tuple(c))
