"""GB300 voxel hop engine: pSpatiocyte's diffusion-and-collision step on an HCP lattice.

Thin ctypes binding over the C ABI declared in include/psc.h (Miyauchi et al.,
arXiv:1605.03726, Sec. 2.1-2.4).  It only marshals arguments: every step of an
event runs in the sm_103a kernels of _build/libpsc.so, and importing fails
loudly if that library cannot be built or loaded -- there is no CPU path.
"""
import ctypes
import os

import numpy as np

from .build import LIB as _LIB_PATH
from .build import build as _build

OK, E_ARG, E_DIMS, E_ORDER, E_FULL, E_UNSUPPORTED, E_NOMEM, E_CUDA, E_TIMEOUT, E_LIMIT, E_CAPACITY = (
    0, -1, -2, -3, -4, -5, -6, -7, -8, -9, -10)
W_PCLAMP = 1
PERIODIC_I, PERIODIC_J, PERIODIC_K, PERIODIC_ALL = 1, 2, 4, 7
FCC = 8                       # lattice flag: FCC (ABC stacking) instead of HCP
MAX_SPECIES = 32
MAX_COMPARTMENTS = 16

_lib = None


class Stats(ctypes.Structure):
    _fields_ = [(n, ctypes.c_uint64) for n in (
        "attempts", "hops", "collisions", "accepted", "reactions2", "fires", "reactions1", "births",
        "events", "launches", "h2d_bytes", "d2h_bytes")]

    def as_dict(self):
        return {n: int(getattr(self, n)) for n, _ in self._fields_}


class Options(ctypes.Structure):
    _fields_ = [(n, ctypes.c_int32) for n in (
        "resort_period", "block_threads", "blocks_per_sm", "collect_stats", "graph_events", "time_kernels",
        "claim_table", "persistent", "slot_map", "claim_slots", "run_per_thread", "barrier_timeout_us", "barrier_phantom", "tiles",
        "tile_regions", "subvolume", "tile_lean")]


class SlabBuffers(ctypes.Structure):
    """psc_slab_buffers: device pointers, [0] the lower side, [1] the upper side."""
    _fields_ = [("send_claim", ctypes.c_void_p * 2), ("recv_claim", ctypes.c_void_p * 2),
                ("send_commit", ctypes.c_void_p * 2), ("recv_commit", ctypes.c_void_p * 2)]


class KernelTimes(ctypes.Structure):
    _fields_ = [("claim_ms", ctypes.c_double), ("commit_ms", ctypes.c_double),
                ("reconcile_ms", ctypes.c_double), ("resort_ms", ctypes.c_double),
                ("claim_launches", ctypes.c_int64), ("commit_launches", ctypes.c_int64),
                ("reconcile_events", ctypes.c_int64), ("resorts", ctypes.c_int64),
                ("run_ms", ctypes.c_double), ("run_launches", ctypes.c_int64), ("run_events", ctypes.c_int64),
                ("tile_launches", ctypes.c_int64), ("tile_events", ctypes.c_int64),
                ("tile_lean_events", ctypes.c_int64)]

    def as_dict(self):
        return {n: (float(getattr(self, n)) if t is ctypes.c_double else int(getattr(self, n)))
                for n, t in self._fields_}


class TuneResult(ctypes.Structure):
    _fields_ = [("persistent", ctypes.c_int32), ("run_per_thread", ctypes.c_int32),
                ("block_threads", ctypes.c_int32), ("blocks_per_sm", ctypes.c_int32),
                ("resort_period", ctypes.c_int32), ("tiles", ctypes.c_int32), ("graph_events", ctypes.c_int32),
                ("trials", ctypes.c_int32),
                ("events", ctypes.c_int64),
                ("us_per_event", ctypes.c_double), ("us_per_event_before", ctypes.c_double)]

    def as_dict(self):
        return {n: (float(getattr(self, n)) if t is ctypes.c_double else int(getattr(self, n)))
                for n, t in self._fields_}


class BatchTuneResult(ctypes.Structure):
    _fields_ = [("threads", ctypes.c_int32), ("blocks_per_member", ctypes.c_int32), ("trials", ctypes.c_int32),
                ("rounds", ctypes.c_int64), ("us_per_round", ctypes.c_double),
                ("us_per_round_before", ctypes.c_double), ("resort_period", ctypes.c_int32)]

    def as_dict(self):
        return {n: (float(getattr(self, n)) if t is ctypes.c_double else int(getattr(self, n)))
                for n, t in self._fields_}


class Request(ctypes.Structure):
    _fields_ = [("ni", ctypes.c_int32), ("nj", ctypes.c_int32), ("nk", ctypes.c_int32),
                ("boundary_flags", ctypes.c_uint32), ("voxel_radius_m", ctypes.c_double),
                ("n_species", ctypes.c_int32), ("D", ctypes.c_void_p), ("initial_count", ctypes.c_void_p),
                ("n_reactions", ctypes.c_int32), ("n_reactants", ctypes.c_void_p), ("reactants", ctypes.c_void_p),
                ("n_products", ctypes.c_void_p), ("products", ctypes.c_void_p), ("k", ctypes.c_void_p),
                ("seed", ctypes.c_uint64), ("t_end", ctypes.c_double)]


ALLOC_FN = ctypes.CFUNCTYPE(ctypes.c_void_p, ctypes.c_size_t, ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p)
FREE_FN = ctypes.CFUNCTYPE(None, ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p)


def lib():
    """The loaded libpsc.so (built in-tree on first use if sources changed)."""
    global _lib
    if _lib is None:
        path = _build()
        if not os.path.exists(path):
            raise ImportError("libpsc.so missing at %s" % path)
        L = ctypes.CDLL(path)
        P, i32, i64, u32, u64, dbl = (ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64, ctypes.c_uint32,
                                      ctypes.c_uint64, ctypes.c_double)
        sig = {
            "psc_lattice_create": (ctypes.c_int, [ctypes.POINTER(P), i32, i32, i32, dbl, u32, ctypes.c_int, P]),
            "psc_add_species": (ctypes.c_int, [P, dbl, i64, ctypes.POINTER(i32)]),
            "psc_add_reaction": (ctypes.c_int, [P, ctypes.POINTER(i32), i32, ctypes.POINTER(i32), i32, dbl,
                                                ctypes.POINTER(i32)]),
            "psc_set_compartments": (ctypes.c_int, [P, P, i32]),
            "psc_species_compartment": (ctypes.c_int, [P, i32, i32]),
            "psc_populate": (ctypes.c_int, [P, u64]),
            "psc_run": (ctypes.c_int, [P, dbl]),
            "psc_run_events": (ctypes.c_int, [P, i64]),
            "psc_synchronize": (ctypes.c_int, [P]),
            "psc_counts": (ctypes.c_int, [P, P, i32]),
            "psc_coords": (ctypes.c_int, [P, i32, P, P, i64, ctypes.POINTER(i64)]),
            "psc_unwrapped": (ctypes.c_int, [P, i32, P, P, i64, ctypes.POINTER(i64)]),
            "psc_grid": (ctypes.c_int, [P, P]),
            "psc_time": (ctypes.c_int, [P, ctypes.POINTER(dbl)]),
            "psc_event_index": (ctypes.c_int, [P, ctypes.POINTER(u32)]),
            "psc_stats_get": (ctypes.c_int, [P, ctypes.POINTER(Stats)]),
            "psc_set_options": (ctypes.c_int, [P, ctypes.POINTER(Options)]),
            "psc_kernel_times_get": (ctypes.c_int, [P, ctypes.POINTER(KernelTimes)]),
            "psc_autotune": (ctypes.c_int, [P, i64, ctypes.POINTER(TuneResult)]),
            "psc_batch_autotune": (ctypes.c_int, [P, i64, ctypes.POINTER(BatchTuneResult)]),
            "psc_tau": (dbl, [P, i32]),
            "psc_p_ab": (dbl, [P, i32]),
            "psc_device_bytes": (ctypes.c_int, [P, ctypes.POINTER(i64)]),
            "psc_lattice_destroy": (None, [P]),
            "psc_status_string": (ctypes.c_char_p, [ctypes.c_int]),
            "psc_set_allocator": (ctypes.c_int, [ALLOC_FN, FREE_FN, P]),
            "psc_hop_events_static": (ctypes.c_int, [i32, i32, i32, u32, u64, i32, u32, i32, P, P, P, i32, P]),
            "psc_batch_create": (ctypes.c_int, [ctypes.POINTER(P), ctypes.c_int, P]),
            "psc_batch_add": (ctypes.c_int, [P, P]),
            "psc_batch_remove": (ctypes.c_int, [P, P]),
            "psc_batch_size": (ctypes.c_int, [P, ctypes.POINTER(i32)]),
            "psc_batch_run_events": (ctypes.c_int, [P, i64]),
            "psc_batch_run": (ctypes.c_int, [P, dbl]),
            "psc_batch_launches": (i64, [P]),
            "psc_batch_destroy": (None, [P]),
            "psc_server_create": (ctypes.c_int, [ctypes.POINTER(P), ctypes.c_int, P, i64, i32]),
            "psc_server_submit": (ctypes.c_int, [P, ctypes.POINTER(Request), ctypes.POINTER(i64)]),
            "psc_server_step": (ctypes.c_int, [P, i32, ctypes.POINTER(i32), ctypes.POINTER(i32)]),
            "psc_server_result": (ctypes.c_int, [P, i64, P, i32, ctypes.POINTER(dbl)]),
            "psc_server_memory": (ctypes.c_int, [P, ctypes.POINTER(i64), ctypes.POINTER(i64)]),
            "psc_server_destroy": (None, [P]),
            "psc_slab_create": (ctypes.c_int, [ctypes.POINTER(P), P, i32, i32, i32, ctypes.c_int, P]),
            "psc_slab_buffers_get": (ctypes.c_int, [P, ctypes.POINTER(SlabBuffers), ctypes.POINTER(i64),
                                                    ctypes.POINTER(i64)]),
            "psc_slab_buffers_set": (ctypes.c_int, [P, ctypes.POINTER(SlabBuffers)]),
            "psc_slab_claim": (ctypes.c_int, [P]),
            "psc_slab_commit": (ctypes.c_int, [P]),
            "psc_slab_apply": (ctypes.c_int, [P]),
            "psc_slabs_run_events": (ctypes.c_int, [ctypes.POINTER(P), i32, i64]),
            "psc_slab_synchronize": (ctypes.c_int, [P]),
            "psc_slab_coords": (ctypes.c_int, [P, P, P, P, i64, ctypes.POINTER(i64)]),
            "psc_slab_event_index": (ctypes.c_int, [P, ctypes.POINTER(u32)]),
            "psc_slab_destroy": (None, [P]),
        }
        for name, (res, args) in sig.items():
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _lib = L
    return _lib


EXPORTED = ("psc_lattice_create", "psc_add_species", "psc_add_reaction", "psc_set_compartments",
            "psc_species_compartment", "psc_populate", "psc_run",
            "psc_run_events", "psc_synchronize", "psc_counts", "psc_coords", "psc_unwrapped", "psc_grid",
            "psc_time", "psc_event_index", "psc_stats_get", "psc_set_options", "psc_kernel_times_get",
            "psc_autotune", "psc_batch_autotune", "psc_tau", "psc_p_ab",
            "psc_device_bytes", "psc_lattice_destroy", "psc_status_string", "psc_set_allocator",
            "psc_hop_events_static", "psc_batch_create", "psc_batch_add", "psc_batch_remove", "psc_batch_size",
            "psc_batch_run_events", "psc_batch_run", "psc_batch_launches", "psc_batch_destroy",
            "psc_server_create", "psc_server_submit", "psc_server_step", "psc_server_result", "psc_server_memory",
            "psc_server_destroy", "psc_slab_create", "psc_slab_buffers_get", "psc_slab_buffers_set",
            "psc_slab_claim", "psc_slab_commit", "psc_slab_apply", "psc_slabs_run_events", "psc_slab_synchronize",
            "psc_slab_coords", "psc_slab_event_index", "psc_slab_destroy")


class EngineError(RuntimeError):
    def __init__(self, fn, rc):
        name = lib().psc_status_string(rc).decode()
        super().__init__("%s failed: %s (%d)" % (fn, name, rc))
        self.rc = rc


def _check(fn, rc, allow=(OK,)):
    if rc not in allow:
        raise EngineError(fn, rc)
    return rc


def _ptr(a):
    return a.ctypes.data_as(ctypes.c_void_p)


_torch_hooks = None


def use_torch_allocator():
    """Route the engine's device allocations through PyTorch's caching allocator."""
    global _torch_hooks
    import torch

    def alloc(nbytes, device, stream, ctx):
        try:
            return torch.cuda.caching_allocator_alloc(int(nbytes), device, stream or 0)
        except Exception:
            return None

    def free(ptr, device, stream, ctx):
        torch.cuda.caching_allocator_delete(ptr)

    _torch_hooks = (ALLOC_FN(alloc), FREE_FN(free))
    _check("psc_set_allocator", lib().psc_set_allocator(_torch_hooks[0], _torch_hooks[1], None))


def use_cuda_malloc():
    global _torch_hooks
    _check("psc_set_allocator", lib().psc_set_allocator(ALLOC_FN(), FREE_FN(), None))
    _torch_hooks = None


class Lattice:
    """One lattice on one GPU; methods mirror the psc_* entry points."""

    def __init__(self, ni, nj, nk, voxel_radius=10e-9, boundary=PERIODIC_ALL, device=0, stream=None):
        self._h = ctypes.c_void_p()
        _check("psc_lattice_create", lib().psc_lattice_create(
            ctypes.byref(self._h), ni, nj, nk, voxel_radius, boundary, device,
            ctypes.c_void_p(stream) if stream else None))
        self.shape = (ni, nj, nk)
        self.n_species = 0

    def close(self):
        if self._h:
            lib().psc_lattice_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def add_species(self, D, count, compartment=None):
        s = ctypes.c_int32()
        _check("psc_add_species", lib().psc_add_species(self._h, float(D), int(count), ctypes.byref(s)))
        self.n_species += 1
        if compartment is not None:
            self.species_compartment(s.value, compartment)
        return s.value

    def set_compartments(self, labels, n):
        """labels: uint8 per voxel, flat (v = i + ni (j + nj k)) or shaped (nk, nj, ni)."""
        lab = np.ascontiguousarray(np.asarray(labels, dtype=np.uint8).reshape(-1))
        if lab.size != self.shape[0] * self.shape[1] * self.shape[2]:
            raise ValueError("labels: one byte per voxel")
        _check("psc_set_compartments", lib().psc_set_compartments(self._h, _ptr(lab), int(n)))

    def species_compartment(self, species, c):
        _check("psc_species_compartment", lib().psc_species_compartment(self._h, int(species), int(c)))

    def add_reaction(self, reactants, products, k):
        r = (ctypes.c_int32 * max(1, len(reactants)))(*reactants)
        p = (ctypes.c_int32 * max(1, len(products)))(*products)
        out = ctypes.c_int32()
        _check("psc_add_reaction", lib().psc_add_reaction(
            self._h, r, len(reactants), p, len(products), float(k), ctypes.byref(out)))
        return out.value

    def populate(self, seed):
        return _check("psc_populate", lib().psc_populate(self._h, int(seed)), (OK, W_PCLAMP))

    def run(self, t_end):
        _check("psc_run", lib().psc_run(self._h, float(t_end)))

    def run_events(self, n):
        _check("psc_run_events", lib().psc_run_events(self._h, int(n)))

    def synchronize(self):
        _check("psc_synchronize", lib().psc_synchronize(self._h))

    def set_options(self, **kw):
        o = Options(**kw)
        _check("psc_set_options", lib().psc_set_options(self._h, ctypes.byref(o)))

    def counts(self):
        c = np.zeros(max(1, self.n_species), dtype=np.int64)
        _check("psc_counts", lib().psc_counts(self._h, _ptr(c), max(1, self.n_species)))
        return c[: self.n_species]

    def coords(self, species):
        n = ctypes.c_int64()
        _check("psc_coords", lib().psc_coords(self._h, species, None, None, 0, ctypes.byref(n)), (OK, E_ARG))
        ijk = np.empty((max(1, n.value), 3), dtype=np.int32)     # every entry is written
        ids = np.empty(max(1, n.value), dtype=np.uint32)
        _check("psc_coords", lib().psc_coords(self._h, species, _ptr(ijk), _ptr(ids), n.value, ctypes.byref(n)))
        return ijk[: n.value], ids[: n.value]

    def unwrapped(self, species):
        n = ctypes.c_int64()
        _check("psc_unwrapped", lib().psc_unwrapped(self._h, species, None, None, 0, ctypes.byref(n)), (OK, E_ARG))
        xyz = np.empty((max(1, n.value), 3), dtype=np.int32)     # every entry is written
        ids = np.empty(max(1, n.value), dtype=np.uint32)
        _check("psc_unwrapped", lib().psc_unwrapped(self._h, species, _ptr(xyz), _ptr(ids), n.value,
                                                    ctypes.byref(n)))
        return xyz[: n.value], ids[: n.value]

    def grid(self):
        ni, nj, nk = self.shape
        g = np.zeros(ni * nj * nk, dtype=np.uint16)
        _check("psc_grid", lib().psc_grid(self._h, _ptr(g)))
        return g

    def time(self):
        t = ctypes.c_double()
        _check("psc_time", lib().psc_time(self._h, ctypes.byref(t)))
        return t.value

    def event_index(self):
        g = ctypes.c_uint32()
        _check("psc_event_index", lib().psc_event_index(self._h, ctypes.byref(g)))
        return g.value

    def stats(self):
        s = Stats()
        _check("psc_stats_get", lib().psc_stats_get(self._h, ctypes.byref(s)))
        return s.as_dict()

    def kernel_times(self):
        k = KernelTimes()
        _check("psc_kernel_times_get", lib().psc_kernel_times_get(self._h, ctypes.byref(k)))
        return k.as_dict()

    def autotune(self, max_events=3000):
        """Pick launch options by timing real events (psc_autotune); returns the choice."""
        r = TuneResult()
        _check("psc_autotune", lib().psc_autotune(self._h, int(max_events), ctypes.byref(r)))
        return r.as_dict()

    def tau(self, species):
        return lib().psc_tau(self._h, species)

    def p_ab(self, reaction):
        return lib().psc_p_ab(self._h, reaction)

    def device_bytes(self):
        b = ctypes.c_int64()
        _check("psc_device_bytes", lib().psc_device_bytes(self._h, ctypes.byref(b)))
        return b.value


class Batch:
    """Lattices advanced together by shared launches (psc_batch_*)."""

    def __init__(self, device=0, stream=None):
        self._h = ctypes.c_void_p()
        _check("psc_batch_create", lib().psc_batch_create(ctypes.byref(self._h), device,
                                                          ctypes.c_void_p(stream) if stream else None))
        self.members = []

    def add(self, lattice):
        _check("psc_batch_add", lib().psc_batch_add(self._h, lattice._h))
        self.members.append(lattice)

    def remove(self, lattice):
        _check("psc_batch_remove", lib().psc_batch_remove(self._h, lattice._h))
        self.members.remove(lattice)

    def run_events(self, n):
        _check("psc_batch_run_events", lib().psc_batch_run_events(self._h, int(n)))

    def run(self, t_end):
        _check("psc_batch_run", lib().psc_batch_run(self._h, float(t_end)))

    def launches(self):
        return int(lib().psc_batch_launches(self._h))

    def autotune(self, max_rounds=200):
        """Pick the batched launches' block shape by timing real batched events."""
        r = BatchTuneResult()
        _check("psc_batch_autotune", lib().psc_batch_autotune(self._h, int(max_rounds), ctypes.byref(r)))
        return r.as_dict()

    def close(self):
        if self._h:
            lib().psc_batch_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Server:
    """Serving loop with continuous batching (psc_server_*)."""

    def __init__(self, max_device_bytes, max_active=512, device=0, stream=None):
        self._h = ctypes.c_void_p()
        _check("psc_server_create", lib().psc_server_create(
            ctypes.byref(self._h), device, ctypes.c_void_p(stream) if stream else None, int(max_device_bytes),
            int(max_active)))
        self._keep = {}

    def submit(self, shape, D, counts, reactions, seed, t_end, voxel_radius=10e-9, boundary=PERIODIC_ALL):
        """reactions: list of (reactants, products, k)."""
        D = np.ascontiguousarray(D, dtype=np.float64)
        n0 = np.ascontiguousarray(counts, dtype=np.int64)
        nr = len(reactions)
        nre = np.array([len(r[0]) for r in reactions] or [0], dtype=np.int32)
        npr = np.array([len(r[1]) for r in reactions] or [0], dtype=np.int32)
        re = np.zeros(2 * max(1, nr), dtype=np.int32)
        pr = np.zeros(2 * max(1, nr), dtype=np.int32)
        kk = np.array([r[2] for r in reactions] or [0.0], dtype=np.float64)
        for x, (a, b, _) in enumerate(reactions):
            re[2 * x: 2 * x + len(a)] = a
            pr[2 * x: 2 * x + len(b)] = b
        req = Request(shape[0], shape[1], shape[2], boundary, voxel_radius, len(D), _ptr(D), _ptr(n0), nr,
                      _ptr(nre), _ptr(re), _ptr(npr), _ptr(pr), _ptr(kk), int(seed), float(t_end))
        t = ctypes.c_int64()
        _check("psc_server_submit", lib().psc_server_submit(self._h, ctypes.byref(req), ctypes.byref(t)))
        self._keep[t.value] = len(D)
        return t.value

    def step(self, n_events):
        a, w = ctypes.c_int32(), ctypes.c_int32()
        _check("psc_server_step", lib().psc_server_step(self._h, int(n_events), ctypes.byref(a), ctypes.byref(w)))
        return a.value, w.value

    def result(self, ticket):
        """(counts, seconds_to_result), or None while the request runs."""
        n = self._keep[ticket]
        c = np.zeros(n, dtype=np.int64)
        sec = ctypes.c_double()
        rc = lib().psc_server_result(self._h, ticket, _ptr(c), n, ctypes.byref(sec))
        if rc == E_ORDER:
            return None
        _check("psc_server_result", rc)
        return c, sec.value

    def memory(self):
        a, b = ctypes.c_int64(), ctypes.c_int64()
        _check("psc_server_memory", lib().psc_server_memory(self._h, ctypes.byref(a), ctypes.byref(b)))
        return a.value, b.value

    def close(self):
        if self._h:
            lib().psc_server_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Slab:
    """One slab of a lattice split along k (psc_slab_*): created from a
    populated Lattice, advanced either together with the other slabs of the
    split in this process (run_slabs) or one per rank through claim / commit /
    apply with the exchanges in between (SlabRanks)."""

    def __init__(self, lattice, species, index, count, device=0, stream=None):
        self._h = ctypes.c_void_p()
        _check("psc_slab_create", lib().psc_slab_create(ctypes.byref(self._h), lattice._h, species, index, count,
                                                        device, ctypes.c_void_p(stream) if stream else None))
        self.index, self.count = index, count

    def close(self):
        if self._h:
            lib().psc_slab_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def buffers(self):
        b = SlabBuffers()
        cb, mb = ctypes.c_int64(), ctypes.c_int64()
        _check("psc_slab_buffers_get", lib().psc_slab_buffers_get(self._h, ctypes.byref(b), ctypes.byref(cb),
                                                                  ctypes.byref(mb)))
        return b, cb.value, mb.value

    def set_buffers(self, send_claim, recv_claim, send_commit, recv_commit):
        """Exchange buffers the caller owns (device pointers, two each: lower, upper side)."""
        b = SlabBuffers()
        for name, ptrs in (("send_claim", send_claim), ("recv_claim", recv_claim),
                           ("send_commit", send_commit), ("recv_commit", recv_commit)):
            arr = getattr(b, name)
            arr[0], arr[1] = int(ptrs[0]), int(ptrs[1])
        _check("psc_slab_buffers_set", lib().psc_slab_buffers_set(self._h, ctypes.byref(b)))

    def claim(self):
        _check("psc_slab_claim", lib().psc_slab_claim(self._h))

    def commit(self):
        _check("psc_slab_commit", lib().psc_slab_commit(self._h))

    def apply(self):
        _check("psc_slab_apply", lib().psc_slab_apply(self._h))

    def synchronize(self):
        _check("psc_slab_synchronize", lib().psc_slab_synchronize(self._h))

    def event_index(self):
        g = ctypes.c_uint32()
        _check("psc_slab_event_index", lib().psc_slab_event_index(self._h, ctypes.byref(g)))
        return g.value

    def coords(self):
        """(ijk, ids, xyz) of the slab's molecules: global coordinates, ids and
        unwrapped positions, in list order."""
        n = ctypes.c_int64()
        _check("psc_slab_coords", lib().psc_slab_coords(self._h, None, None, None, 0, ctypes.byref(n)))
        m = max(1, n.value)
        ijk = np.zeros((m, 3), dtype=np.int32)
        ids = np.zeros(m, dtype=np.uint32)
        xyz = np.zeros((m, 3), dtype=np.int32)
        _check("psc_slab_coords", lib().psc_slab_coords(self._h, _ptr(ijk), _ptr(ids), _ptr(xyz), m,
                                                        ctypes.byref(n)))
        return ijk[: n.value], ids[: n.value], xyz[: n.value]


def run_slabs(slabs, n_events):
    """n_events events of all slabs of a split held by this process."""
    arr = (ctypes.c_void_p * len(slabs))(*[s._h.value for s in slabs])
    _check("psc_slabs_run_events", lib().psc_slabs_run_events(arr, len(slabs), int(n_events)))


def slab_neighbour(rank, world, side, periodic_k):
    """Rank holding the neighbouring slab on `side` (0 below, 1 above), None at a wall."""
    q = rank - 1 if side == 0 else rank + 1
    if 0 <= q < world:
        return q
    return (q % world) if periodic_k else None


class SlabRanks:
    """Host side of a split with one slab per rank: the neighbour ranks and the
    two exchanges of every event as point-to-point sends and receives of whole
    buffers through torch.distributed.  A slab's send[1] (its upper face) goes
    to the upper neighbour's recv[0]; its send[0] to the lower neighbour's
    recv[1].  Every rank posts the upward traffic first, then the downward
    traffic, so that messages between one pair of ranks match in order (as
    NCCL requires) even when the two neighbours are the same rank."""

    UP, DOWN = 0, 1

    def __init__(self, rank, world, periodic_k):
        self.rank, self.world, self.periodic_k = rank, world, bool(periodic_k)
        self.nb = [slab_neighbour(rank, world, s, periodic_k) for s in (0, 1)]

    def exchange(self, send, recv):
        """send[side] to the neighbour on that side, recv[side] from it (tensors)."""
        import torch.distributed as dist
        if self.world == 1:
            if self.periodic_k:
                recv[0].copy_(send[1])
                recv[1].copy_(send[0])
            return
        ops = []
        if self.nb[1] is not None:
            ops.append(dist.P2POp(dist.isend, send[1], self.nb[1], tag=self.UP))
        if self.nb[0] is not None:
            ops.append(dist.P2POp(dist.irecv, recv[0], self.nb[0], tag=self.UP))
        if self.nb[0] is not None:
            ops.append(dist.P2POp(dist.isend, send[0], self.nb[0], tag=self.DOWN))
        if self.nb[1] is not None:
            ops.append(dist.P2POp(dist.irecv, recv[1], self.nb[1], tag=self.DOWN))
        if ops:
            for req in dist.batch_isend_irecv(ops):
                req.wait()

    def run_events(self, slab, bufs, n_events):
        """n_events events of this rank's slab; bufs = dict of the slab's
        exchange tensors (send_claim, recv_claim, send_commit, recv_commit,
        each a pair) already set with Slab.set_buffers."""
        for _ in range(int(n_events)):
            slab.claim()
            self.exchange(bufs["send_claim"], bufs["recv_claim"])
            slab.commit()
            self.exchange(bufs["send_commit"], bufs["recv_commit"])
            slab.apply()
