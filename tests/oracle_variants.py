"""Planted mistakes: the oracle compiled with a text substitution into a temporary
library, swapped in for the duration of a ``with`` block, so that a pin can show that it
fails on a plausible error in the arithmetic it guards (a wrong index, a swapped
component, a dropped term). CPU only; the product library is never touched."""
import contextlib
import ctypes as C
import os
import subprocess
import tempfile

import oracle


@contextlib.contextmanager
def planted(*subs):
    """Runs the block with the oracle built from its source with each (old, new)
    substitution applied (every ``old`` must occur in the source)."""
    with open(oracle._SRC) as f:
        src = f.read()
    for old, new in subs:
        assert old in src, f"planted mistake does not apply: {old!r}"
        src = src.replace(old, new)
    with tempfile.TemporaryDirectory() as d:
        c_path = os.path.join(d, "variant.c")
        so_path = os.path.join(d, "variant.so")
        with open(c_path, "w") as f:
            f.write(src)
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-o", so_path,
                               c_path, "-lm"])
        saved = oracle.lib()
        oracle._lib = oracle.configure(C.CDLL(so_path))
        try:
            yield
        finally:
            oracle._lib = saved


def fails(check, *subs) -> bool:
    """Whether ``check()`` raises an AssertionError under the planted mistake."""
    with planted(*subs):
        try:
            check()
        except AssertionError:
            return True
    return False
