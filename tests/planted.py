"""Build a copy of the oracle with one planted mistake (CPU only).

A pin is only worth something if a plausible mistake in the oracle breaks it.
`planted_oracle` copies oracle/psco.c and psco.h into a temporary folder,
replaces one exact piece of source text, compiles the copy with the oracle's
own flags and returns the loaded library; `using` makes the oracle binding
route every call to it for the duration of a `with` block.
"""
import contextlib
import os
import shutil

import oracle
from oracle import build as obuild


def planted_oracle(tmp_path, old, new):
    src_dir = os.path.dirname(obuild.SOURCES[0])
    with open(os.path.join(src_dir, "psco.c")) as f:
        text = f.read()
    assert text.count(old) == 1, "planted mistake: the text to replace must occur exactly once"
    d = str(tmp_path)
    shutil.copy(os.path.join(src_dir, "psco.h"), os.path.join(d, "psco.h"))
    c_path = os.path.join(d, "psco.c")
    with open(c_path, "w") as f:
        f.write(text.replace(old, new))
    return oracle.load(obuild.compile_library([c_path], os.path.join(d, "libplanted.so")))


@contextlib.contextmanager
def using(lib):
    saved = oracle.lib()
    oracle._lib = lib
    try:
        yield
    finally:
        oracle._lib = saved
