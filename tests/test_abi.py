"""The C-ABI library builds for sm_103a, loads, and exports every entry
point that include/qmc.h declares (no compute calls: no GPU needed)."""
import ctypes
import os
import re

from paper_2504_07948_gb300 import build as B

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_symbols():
    names = set()
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if fn.endswith(".h"):
            txt = open(os.path.join(ROOT, "include", fn)).read()
            txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
            names |= set(re.findall(r"^\s*(?:const\s+)?\w+\s*\*?\s*(qmc_\w+)\s*\(", txt, flags=re.M))
    return names


def test_library_exports_every_declared_symbol():
    lib = ctypes.CDLL(B.build())
    names = declared_symbols()
    assert len(names) >= 20
    missing = [n for n in sorted(names) if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_covers_header():
    from paper_2504_07948_gb300 import qmc as Q
    for n in declared_symbols():
        assert hasattr(Q, n), n


def test_create_without_device_fails_cleanly():
    """On a machine without a GPU the handle cannot be created; the error is
    a status code and a message, never a crash or a silent CPU path."""
    import torch
    if torch.cuda.is_available():
        return
    from paper_2504_07948_gb300 import qmc as Q
    try:
        Q.qmc_create(0)
    except Q.QmcError as e:
        assert e.code in (-1, -2)
    else:
        raise AssertionError("handle created without a CUDA device")
