"""The C-ABI library loads and exports every function include/ibdl.h
declares; argument validation rejects bad descriptions before touching the
GPU.  CPU only (no compute calls)."""
import os
import re
import subprocess

import numpy as np
import pytest

import paper_2203_12126_gb300 as pkg
from paper_2203_12126_gb300 import ibdl

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "ibdl.h")


def _declared():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(ibdl_[a-z0-9_]+)\s*\(", src)))


@pytest.fixture(scope="module")
def lib():
    if not os.path.exists(ibdl.LIB_PATH):
        import __graft_entry__
        __graft_entry__.build()
    return pkg.load()


def test_header_and_binding_agree():
    assert _declared() == sorted(ibdl.EXPORTS)


def test_library_exports_every_declared_symbol(lib):
    out = subprocess.run(["nm", "-D", "--defined-only", ibdl.LIB_PATH], capture_output=True,
                         text=True, check=True).stdout
    exported = set(re.findall(r"\bT (ibdl_[a-z0-9_]+)\b", out))
    missing = [s for s in _declared() if s not in exported]
    assert not missing, missing
    for s in _declared():
        assert hasattr(lib, s)


def test_version_and_status_strings(lib):
    assert lib.ibdl_version() == 1
    assert lib.ibdl_status_string(0) == b"ok"
    assert lib.ibdl_status_string(4) == b"not converged"


def _desc_args(**over):
    m = 8
    a = dict(dim=2, n=64, box_len=1.0, origin=(0.0, 0.0), x=np.full(m, 0.5),
             y=np.full(m, 0.5), nx=np.ones(m), ny=np.zeros(m), w=np.ones(m), kappa=1e-2)
    a.update(over)
    return a


@pytest.mark.parametrize("bad", [
    dict(dim=4), dict(n=48), dict(n=8), dict(n=8192), dict(kappa=0.0),
    dict(kappa=float("nan")), dict(box_len=-1.0), dict(delta=7), dict(bc=3),
    dict(precision=5), dict(dim=3, n=1024),
])
def test_invalid_descriptions_are_rejected(lib, bad):
    with pytest.raises(ibdl.IbdlError) as e:
        ibdl.Geometry(**_desc_args(**bad))
    assert e.value.status == ibdl.ERR_INVALID_ARG


def test_missing_3d_arrays_rejected(lib):
    with pytest.raises(ibdl.IbdlError) as e:
        ibdl.Geometry(**_desc_args(dim=3, n=32))
    assert e.value.status == ibdl.ERR_INVALID_ARG
    assert "NULL" in str(e.value)


@pytest.mark.parametrize("args", [
    (4, 64, 0, 8), (1, 64, 0, 8), (2, 100, 0, 8), (2, 8, 0, 2), (2, 8192, 0, 2),
    (2, 64, 2, 8), (2, 64, -1, 8), (2, 64, 0, 6), (2, 64, 0, 32), (2, 64, 0, -2),
    (2, 64, 0, 1), (2, 1024, 1, 8), (3, 32, 0, 16), (3, 256, 0, 64),
])
def test_inadmissible_tiling_pins_are_rejected(lib, args):
    """ibdl_tuning_set checks dim, n, precision and the tiling (an even power
    of two R with n/R >= 4, R <= n - 5, float64 row tiles within 100 KB)
    before it reads the device."""
    with pytest.raises(ibdl.IbdlError) as e:
        ibdl.tuning_set(*args)
    assert e.value.status == ibdl.ERR_INVALID_ARG
