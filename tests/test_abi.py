"""The C-ABI library loads and exports every entry point include/*.h declares (no GPU
needed: nothing is called)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    import glob
    src = "".join(open(h).read() for h in sorted(glob.glob(os.path.join(ROOT, "include", "*.h"))))
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    names = re.findall(r"^\s*(?:const\s+)?[a-z_][a-z0-9_]*\s*\**\s+\**([a-z_][a-z0-9_]*)\s*\(",
                       src, flags=re.M)
    return sorted(set(names))


def test_header_declares_the_boundary():
    names = _declared()
    for required in ("mp_init", "mp_init_batch", "mp_step", "mp_vacf", "mp_mass", "mp_info",
                     "mp_get_field", "mp_set_field", "mp_free", "mp_last_error",
                     "mp_default_options", "lb_steady"):
        assert required in names


def test_library_exports_every_declared_symbol():
    from paper_1303_2470_gb300 import build as b
    path = b.build()
    lib = ctypes.CDLL(path)
    for name in _declared():
        assert hasattr(lib, name), f"{name} not exported by {path}"


def test_options_defaults_without_gpu():
    from paper_1303_2470_gb300 import build as b
    b.build()
    from paper_1303_2470_gb300 import mp
    o = mp.mp_default_options()
    assert o.precision == mp.MP_FP32 and o.directions == 1 and o.capacity == 131072
    assert o.init_density == mp.MP_INIT_EQUILIBRIUM and not o.allow_negative
