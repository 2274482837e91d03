"""ctypes view of the CPU oracle (oracle/psco.c).

TEST INFRASTRUCTURE ONLY: imported by tests/, by __graft_entry__.smoke() and by
the CPU-baseline leg of bench.py.  The product package never imports it.
"""
import ctypes
import os

import numpy as np

from .build import build as _build

OK, E_ARG, E_DIMS, E_ORDER, E_FULL, E_UNSUPPORTED, E_NOMEM, E_LIMIT = 0, -1, -2, -3, -4, -5, -6, -9
MAX_COMPARTMENTS = 16
W_PCLAMP = 1
RULE_SYNC, RULE_SEQ_ID, RULE_SEQ_RANDOM, RULE_SUBVOL = 0, 1, 2, 3
PERIODIC_I, PERIODIC_J, PERIODIC_K = 1, 2, 4
PERIODIC_ALL = 7
FCC = 8                  # lattice flag: FCC (ABC stacking) instead of HCP

_lib = None


class Stats(ctypes.Structure):
    _fields_ = [(n, ctypes.c_uint64) for n in
                ("attempts", "hops", "collisions", "accepted", "reactions2", "fires",
                 "reactions1", "births", "events")] + [("dir_count", ctypes.c_uint64 * 12)]

    def as_dict(self):
        d = {n: int(getattr(self, n)) for n, _ in self._fields_ if n != "dir_count"}
        d["dir_count"] = [int(x) for x in self.dir_count]
        return d


def load(path):
    """Open an oracle shared library at `path` and declare its C signatures."""
    L = ctypes.CDLL(path)
    P = ctypes.c_void_p
    i32, i64, u32, u64, dbl = ctypes.c_int32, ctypes.c_int64, ctypes.c_uint32, ctypes.c_uint64, ctypes.c_double
    sig = {
        "psco_lattice_create": (ctypes.c_int, [ctypes.POINTER(P), i32, i32, i32, dbl, u32, i32]),
        "psco_add_species": (ctypes.c_int, [P, dbl, i64, ctypes.POINTER(i32)]),
        "psco_add_reaction": (ctypes.c_int, [P, ctypes.POINTER(i32), i32, ctypes.POINTER(i32), i32, dbl, ctypes.POINTER(i32)]),
        "psco_set_compartments": (ctypes.c_int, [P, P, i32]),
        "psco_species_compartment": (ctypes.c_int, [P, i32, i32]),
        "psco_populate": (ctypes.c_int, [P, u64]),
        "psco_run": (ctypes.c_int, [P, dbl]),
        "psco_run_events": (ctypes.c_int, [P, i64]),
        "psco_counts": (ctypes.c_int, [P, P, i32]),
        "psco_coords": (ctypes.c_int, [P, i32, P, P, i64, ctypes.POINTER(i64)]),
        "psco_unwrapped": (ctypes.c_int, [P, i32, P, P, i64, ctypes.POINTER(i64)]),
        "psco_grid": (ctypes.c_int, [P, P]),
        "psco_time": (ctypes.c_int, [P, ctypes.POINTER(dbl)]),
        "psco_event_index": (ctypes.c_int, [P, ctypes.POINTER(u32)]),
        "psco_stats_get": (ctypes.c_int, [P, ctypes.POINTER(Stats)]),
        "psco_check": (ctypes.c_int, [P]),
        "psco_place": (ctypes.c_int, [P, i32, i32, ctypes.POINTER(u32)]),
        "psco_lattice_destroy": (None, [P]),
        "psco_tau": (dbl, [P, i32]),
        "psco_p_ab": (dbl, [P, i32]),
        "psco_threshold": (u64, [dbl]),
        "psco_philox4x32_10": (None, [P, P, P]),
        "psco_neighbor": (ctypes.c_int, [P, i32, i32, i32, i32, P, P]),
        "psco_center": (None, [i32, i32, i32, P]),
        "psco_center_fcc": (None, [i32, i32, i32, P]),
    }
    for name, (res, args) in sig.items():
        f = getattr(L, name)
        f.restype = res
        f.argtypes = args
    return L


def lib():
    global _lib
    if _lib is None:
        _lib = load(_build())
    return _lib


def _ptr(a):
    return a.ctypes.data_as(ctypes.c_void_p)


def philox(ctr, key):
    """Philox4x32-10 of the oracle: ctr = 4 words, key = 2 words -> 4 words."""
    c = np.asarray(ctr, dtype=np.uint32)
    k = np.asarray(key, dtype=np.uint32)
    o = np.zeros(4, dtype=np.uint32)
    lib().psco_philox4x32_10(_ptr(c), _ptr(k), _ptr(o))
    return [int(x) for x in o]


def threshold(p):
    return int(lib().psco_threshold(float(p)))


def center_fcc(i, j, k):
    o = np.zeros(3)
    lib().psco_center_fcc(i, j, k, _ptr(o))
    return o


def center(i, j, k):
    o = np.zeros(3, dtype=np.float64)
    lib().psco_center(i, j, k, _ptr(o))
    return o


class OracleError(RuntimeError):
    def __init__(self, fn, rc):
        super().__init__("%s returned %d" % (fn, rc))
        self.rc = rc


def _check(fn, rc, allow=(OK,)):
    if rc not in allow:
        raise OracleError(fn, rc)
    return rc


class Lattice:
    """One oracle lattice; methods mirror the psc_* C ABI."""

    def __init__(self, ni, nj, nk, voxel_radius=10e-9, boundary=PERIODIC_ALL, rule=RULE_SYNC):
        self._h = ctypes.c_void_p()
        _check("psco_lattice_create", lib().psco_lattice_create(
            ctypes.byref(self._h), ni, nj, nk, voxel_radius, boundary, rule))
        self.shape = (ni, nj, nk)
        self.n_species = 0

    def close(self):
        if self._h:
            lib().psco_lattice_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def add_species(self, D, count, compartment=None):
        s = ctypes.c_int32()
        _check("psco_add_species", lib().psco_add_species(self._h, float(D), int(count), ctypes.byref(s)))
        self.n_species += 1
        if compartment is not None:
            self.species_compartment(s.value, compartment)
        return s.value

    def add_reaction(self, reactants, products, k):
        r = (ctypes.c_int32 * max(1, len(reactants)))(*reactants)
        p = (ctypes.c_int32 * max(1, len(products)))(*products)
        out = ctypes.c_int32()
        _check("psco_add_reaction", lib().psco_add_reaction(
            self._h, r, len(reactants), p, len(products), float(k), ctypes.byref(out)))
        return out.value

    def set_compartments(self, labels, n):
        """labels: uint8 per voxel, flat (v = i + ni (j + nj k)) or shaped (nk, nj, ni)."""
        lab = np.ascontiguousarray(np.asarray(labels, dtype=np.uint8).reshape(-1))
        if lab.size != self.shape[0] * self.shape[1] * self.shape[2]:
            raise ValueError("labels: one byte per voxel")
        _check("psco_set_compartments", lib().psco_set_compartments(self._h, _ptr(lab), int(n)))

    def species_compartment(self, species, c):
        _check("psco_species_compartment", lib().psco_species_compartment(self._h, species, int(c)))

    def populate(self, seed):
        return _check("psco_populate", lib().psco_populate(self._h, int(seed)), (OK, W_PCLAMP))

    def run(self, t_end):
        _check("psco_run", lib().psco_run(self._h, float(t_end)))

    def run_events(self, n):
        _check("psco_run_events", lib().psco_run_events(self._h, int(n)))

    def counts(self):
        c = np.zeros(max(1, self.n_species), dtype=np.int64)
        _check("psco_counts", lib().psco_counts(self._h, _ptr(c), self.n_species))
        return c[: self.n_species]

    def coords(self, species):
        n = ctypes.c_int64()
        lib().psco_coords(self._h, species, None, None, 0, ctypes.byref(n))
        ijk = np.zeros((max(1, n.value), 3), dtype=np.int32)
        ids = np.zeros(max(1, n.value), dtype=np.uint32)
        _check("psco_coords", lib().psco_coords(self._h, species, _ptr(ijk), _ptr(ids), n.value, ctypes.byref(n)))
        return ijk[: n.value], ids[: n.value]

    def unwrapped(self, species):
        n = ctypes.c_int64()
        lib().psco_unwrapped(self._h, species, None, None, 0, ctypes.byref(n))
        xyz = np.zeros((max(1, n.value), 3), dtype=np.int32)
        ids = np.zeros(max(1, n.value), dtype=np.uint32)
        _check("psco_unwrapped", lib().psco_unwrapped(self._h, species, _ptr(xyz), _ptr(ids), n.value, ctypes.byref(n)))
        return xyz[: n.value], ids[: n.value]

    def grid(self):
        ni, nj, nk = self.shape
        g = np.zeros(ni * nj * nk, dtype=np.uint16)
        _check("psco_grid", lib().psco_grid(self._h, _ptr(g)))
        return g

    def time(self):
        t = ctypes.c_double()
        _check("psco_time", lib().psco_time(self._h, ctypes.byref(t)))
        return t.value

    def event_index(self):
        g = ctypes.c_uint32()
        _check("psco_event_index", lib().psco_event_index(self._h, ctypes.byref(g)))
        return g.value

    def stats(self):
        s = Stats()
        _check("psco_stats_get", lib().psco_stats_get(self._h, ctypes.byref(s)))
        return s.as_dict()

    def check(self):
        return lib().psco_check(self._h)

    def place(self, species, v):
        i = ctypes.c_uint32()
        _check("psco_place", lib().psco_place(self._h, species, int(v), ctypes.byref(i)))
        return i.value

    def tau(self, species):
        return lib().psco_tau(self._h, species)

    def p_ab(self, reaction):
        return lib().psco_p_ab(self._h, reaction)

    def neighbor(self, i, j, k, d):
        o = np.zeros(3, dtype=np.int32)
        w = np.zeros(3, dtype=np.int32)
        inside = lib().psco_neighbor(self._h, i, j, k, d, _ptr(o), _ptr(w))
        return bool(inside), tuple(int(x) for x in o), tuple(int(x) for x in w)
