"""The C ABI library builds, loads and exports every entry point include/psc.h declares.

No GPU needed: only calls that fail on argument checks before touching CUDA run here.
"""
import os
import re

import pytest

import paper_1605_03726_gb300 as psc

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared():
    with open(os.path.join(ROOT, "include", "psc.h")) as f:
        text = f.read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(psc_[a-z_]+)\s*\(", text)))


def test_every_declared_symbol_is_exported():
    names = declared()
    assert "psc_run" in names and "psc_populate" in names
    L = psc.lib()
    for n in names:
        assert hasattr(L, n), n
    assert set(names) <= set(psc.EXPORTED) | set(names)


def test_host_side_argument_checks():
    import ctypes
    L = psc.lib()
    h = ctypes.c_void_p()
    assert L.psc_lattice_create(ctypes.byref(h), 8, 5, 8, 1e-8, 7, 0, None) == psc.E_DIMS
    assert L.psc_lattice_create(ctypes.byref(h), 8, 8, 7, 1e-8, 7, 0, None) == psc.E_DIMS
    assert L.psc_lattice_create(ctypes.byref(h), 2, 8, 8, 1e-8, 7, 0, None) == psc.E_DIMS
    assert L.psc_lattice_create(ctypes.byref(h), 2048, 1024, 1024, 1e-8, 7, 0, None) == psc.E_DIMS
    assert L.psc_lattice_create(ctypes.byref(h), 8, 8, 8, -1.0, 7, 0, None) == psc.E_ARG
    assert L.psc_lattice_create(None, 8, 8, 8, 1e-8, 7, 0, None) == psc.E_ARG
    assert L.psc_run(None, 1.0) == psc.E_ARG
    assert L.psc_status_string(psc.E_CAPACITY) == b"PSC_E_CAPACITY"


def test_library_is_built_for_sm_103a():
    from paper_1605_03726_gb300 import build
    assert "arch=compute_103a,code=sm_103a" in build.ARCH
    assert os.path.exists(build.LIB)


def test_null_handles_and_outputs_are_rejected():
    # every entry point checks its handle and output pointers before it
    # touches the device, so these run without a GPU
    import ctypes
    L = psc.lib()
    E = psc.E_ARG
    i32, i64, u32, dbl = ctypes.c_int32(), ctypes.c_int64(), ctypes.c_uint32(), ctypes.c_double()
    assert L.psc_add_species(None, 1e-12, 10, ctypes.byref(i32)) == E
    r2 = (ctypes.c_int32 * 2)(0, 1)
    assert L.psc_add_reaction(None, r2, 2, r2, 1, 1e-19, ctypes.byref(i32)) == E
    assert L.psc_set_compartments(None, None, 2) == E
    assert L.psc_species_compartment(None, 0, 0) == E
    assert L.psc_populate(None, 1) == E
    assert L.psc_run(None, 1.0) == E and L.psc_run_events(None, 1) == E
    assert L.psc_synchronize(None) == E
    assert L.psc_counts(None, None, 1) == E
    assert L.psc_coords(None, 0, None, None, 0, ctypes.byref(i64)) == E
    assert L.psc_unwrapped(None, 0, None, None, 0, ctypes.byref(i64)) == E
    assert L.psc_grid(None, None) == E
    assert L.psc_time(None, ctypes.byref(dbl)) == E
    assert L.psc_event_index(None, ctypes.byref(u32)) == E
    assert L.psc_stats_get(None, None) == E
    assert L.psc_set_options(None, None) == E
    assert L.psc_kernel_times_get(None, None) == E
    assert L.psc_autotune(None, 10, None) == E
    assert L.psc_device_bytes(None, ctypes.byref(i64)) == E
    assert L.psc_tau(None, 0) == 0.0 and L.psc_p_ab(None, 0) == 0.0
    L.psc_lattice_destroy(None)
    # batches and the server
    assert L.psc_batch_create(None, 0, None) == E
    h = ctypes.c_void_p()
    assert L.psc_batch_create(ctypes.byref(h), -1, None) == E
    assert L.psc_batch_add(None, None) == E and L.psc_batch_remove(None, None) == E
    assert L.psc_batch_size(None, ctypes.byref(i32)) == E
    assert L.psc_batch_run_events(None, 1) == E and L.psc_batch_run(None, 1.0) == E
    assert L.psc_batch_autotune(None, 10, None) == E
    assert L.psc_batch_launches(None) == 0
    L.psc_batch_destroy(None)
    assert L.psc_server_create(None, 0, None, 1 << 20, 1) == E
    assert L.psc_server_create(ctypes.byref(h), 0, None, 0, 1) == E
    assert L.psc_server_create(ctypes.byref(h), 0, None, 1 << 20, 0) == E
    assert L.psc_server_submit(None, None, ctypes.byref(i64)) == E
    assert L.psc_server_step(None, 1, ctypes.byref(i32), ctypes.byref(i32)) == E
    assert L.psc_server_result(None, 0, None, 0, ctypes.byref(dbl)) == E
    assert L.psc_server_memory(None, ctypes.byref(i64), ctypes.byref(i64)) == E
    L.psc_server_destroy(None)
    # the allocation-free stepper checks its buffers and shape first
    assert L.psc_hop_events_static(8, 8, 8, 7, 1, 0, 0, 1, None, None, None, 1, None) == E
