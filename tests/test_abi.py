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


@pytest.mark.parametrize("field,value,status", [
    ("L1", 4, "ERR_UNSUPPORTED"),       # below the smallest grid side (8)
    ("L2", 2048, "ERR_UNSUPPORTED"),    # above the largest (1024)
    ("L1", 96, "ERR_UNSUPPORTED"),      # not a power of two
    ("M1", 0, "ERR_INVALID_ARG"),
    ("lam", -0.5, "ERR_INVALID_ARG"),
    ("lam", float("nan"), "ERR_INVALID_ARG"),
    ("reserved", 1, "ERR_INVALID_ARG"),
    ("c_off", -1, "ERR_INVALID_ARG"),
])
def test_create_rejects_bad_instances_on_the_host(so_path, field, value, status):
    """Every instance is validated before any device work, with the documented status and a message."""
    import numpy as np

    import paper_2509_13592_gb300 as bccb

    q = bccb.bccb_inst_t(4, 4, 16, 16, 0, 0, 0, 0.1, 0, 0)
    setattr(q, field, value)
    with pytest.raises(bccb.BccbError) as e:
        bccb.bccb_batch_create([q], np.ones(16, np.uint8), bccb.FISTA, 1.0, stream=0)
    assert e.value.status == getattr(bccb, status)
    assert len(str(e.value)) > len(bccb.bccb_status_string(e.value.status))  # a message came with it


def test_create_rejects_bad_solver_arguments_on_the_host(so_path):
    import numpy as np

    import paper_2509_13592_gb300 as bccb

    q = bccb.bccb_inst_t(4, 4, 16, 16, 0, 0, 0, 0.1, 0, 0)
    ones = np.ones(16, np.uint8)
    for kw, status in ((dict(algo=7), bccb.ERR_INVALID_ARG), (dict(algo=bccb.ADMM, rho=0.0), bccb.ERR_INVALID_ARG),
                       (dict(algo=bccb.FISTA, prec=5), bccb.ERR_INVALID_ARG)):
        args = dict(algo=bccb.FISTA, rho=1.0, prec=bccb.F32)
        args.update(kw)
        with pytest.raises(bccb.BccbError) as e:
            bccb.bccb_batch_create([q], ones, args["algo"], args["rho"], stream=0, prec=args["prec"])
        assert e.value.status == status
    with pytest.raises(bccb.BccbError) as e:  # a mask that keeps no element
        bccb.bccb_batch_create([q], np.zeros(16, np.uint8), bccb.FISTA, 1.0, stream=0)
    assert e.value.status == bccb.ERR_INVALID_ARG
    assert b"empty mask" in bccb._lib.bccb_last_error(None)
