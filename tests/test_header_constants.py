"""The binding's constants equal the C header's (include/s2gb.h): return codes, samplings,
precisions, plan flags and the no-allocation scratch size, read from the header text."""
import os
import re

from paper_2311_14670_gb300 import _native as nat

HEADER = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "include", "s2gb.h")


def _header_values():
    text = open(HEADER).read()
    vals = {}
    for name, val in re.findall(r"\b(S2GB_[A-Z0-9_]+)\s*=\s*(-?\d+)", text):       # enum members
        vals[name] = int(val)
    for name, val in re.findall(r"#define\s+(S2GB_[A-Z0-9_]+)\s+\(?(\d+)u?", text):  # flag macros
        vals.setdefault(name, int(val))
    return vals


def test_binding_constants_match_header():
    vals = _header_values()
    names = [n for n in dir(nat) if n.startswith("S2GB_") and isinstance(getattr(nat, n), int)]
    assert names
    for n in names:
        assert n in vals, f"{n} is not declared in include/s2gb.h"
        assert getattr(nat, n) == vals[n], n
    for n in ("S2GB_MW", "S2GB_MWSS", "S2GB_DH", "S2GB_FP64", "S2GB_FP32", "S2GB_PLAN_REAL",
              "S2GB_PLAN_PRECOMPUTE", "S2GB_PLAN_MRECURSION", "S2GB_EWORKSPACE"):
        assert n in names, f"{n} missing from the binding"


def test_sampling_shapes_of_the_python_plan_helper():
    from paper_2311_14670_gb300.transforms import sampling_shape
    for L in (1, 2, 7, 64):
        assert sampling_shape(L, "mw") == (L, 2 * L - 1)
        assert sampling_shape(L, "mwss") == (L + 1, 2 * L)
        assert sampling_shape(L, "dh") == (2 * L, 2 * L - 1)
