"""The C-ABI library loads and exports every entry point declared in include/*.h
(CPU only: no compute call is made)."""
import ctypes
import glob
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        text = open(h).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        for m in re.finditer(r"^\s*(?:const\s+)?[A-Za-z_][\w\s\*]*?\b(bccb_\w+)\s*\(", text, flags=re.M):
            names.add(m.group(1))
    return names


@pytest.fixture(scope="module")
def so_path():
    from paper_2509_13592_gb300 import build as b

    if not os.path.exists(b.LIB):
        b.build()
    return b.LIB


def test_header_declares_the_boundary():
    names = _declared()
    for n in ("bccb_batch_create", "bccb_batch_solve", "bccb_batch_solve_host", "bccb_batch_results",
              "bccb_create", "bccb_solve", "bccb_destroy", "bccb_status_string"):
        assert n in names


def test_library_exports_every_declared_symbol(so_path):
    lib = ctypes.CDLL(so_path)
    missing = [n for n in sorted(_declared()) if not hasattr(lib, n)]
    assert not missing, missing


def test_status_strings_without_gpu(so_path):
    lib = ctypes.CDLL(so_path)
    lib.bccb_status_string.restype = ctypes.c_char_p
    assert lib.bccb_status_string(0) == b"ok"
    assert lib.bccb_status_string(2) == b"unsupported size"


def test_binding_rejects_bad_sizes_before_any_device_call(so_path):
    import numpy as np

    import paper_2509_13592_gb300 as bccb

    q = bccb.bccb_inst_t(4, 4, 48, 16, 0, 0, 0, 0.1, 0, 0)
    with pytest.raises(bccb.BccbError) as e:
        bccb.bccb_batch_create([q], np.ones(16, np.uint8), bccb.FISTA, 1.0, stream=0)
    assert e.value.status == bccb.ERR_UNSUPPORTED
