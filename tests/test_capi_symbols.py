"""The C-ABI library builds for sm_103a and exports every function that
include/qaoa.h declares (no GPU needed: nothing is called)."""

import ctypes
import os
import re

from conftest import ROOT


def declared_functions():
    src = open(os.path.join(ROOT, "include", "qaoa.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(qaoa_[a-z_0-9]+)\s*\(", src)))


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ["qaoa_cost_precompute", "qaoa_expectation", "qaoa_gradient",
                     "qaoa_expectation_batched", "qaoa_create", "qaoa_destroy"]:
        assert required in names


def test_library_builds_and_exports_every_symbol():
    from paper_2312_06451_gb300 import _binding, build

    path = build.build()
    assert os.path.exists(path)
    lib = ctypes.CDLL(path)
    for name in declared_functions():
        assert hasattr(lib, name), name
    # the ctypes mirror covers exactly the declared functions
    assert sorted(_binding.SIGNATURES) == declared_functions()


def test_oracle_is_independent_of_the_library():
    """The oracle shares no code with the CUDA path: neither side includes or
    imports the other."""
    osrc = open(os.path.join(ROOT, "oracle", "qaoa_oracle.c")).read()
    assert "#include \"" not in osrc
    opy = open(os.path.join(ROOT, "oracle", "__init__.py")).read()
    assert "paper_2312_06451_gb300" not in opy
    pkg = os.path.join(ROOT, "paper_2312_06451_gb300")
    for dp, _, files in os.walk(pkg):
        for f in files:
            if f.endswith((".py", ".cu", ".cuh", ".h")):
                txt = open(os.path.join(dp, f)).read()
                assert "import oracle" not in txt and "from oracle" not in txt, f
                assert "qaoa_oracle" not in txt, f
