"""CPU checks of the C ABI: the library loads, exports every declared entry
point, and its host-side FC-Gram table builder agrees with the oracle's."""
import ctypes
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "fcsdnn.h")


@pytest.fixture(scope="module")
def lib():
    from paper_2506_19370_gb300 import build, fcsdnn
    if not os.path.exists(fcsdnn.LIB_PATH):
        build.build()
    return fcsdnn.lib()


def declared_functions():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    names = re.findall(r"^\s*(?:const\s+)?[a-z_]+\s*\**\s*([a-z_][a-z0-9_]*)\s*\(", src, flags=re.M)
    return sorted(set(names))


def test_header_declares_the_entry_points():
    names = declared_functions()
    for n in ("fc_setup", "fc_derivative", "sdnn_classify", "av_assemble", "euler_rhs", "rk_stage",
              "patch_exchange"):
        assert n in names


def test_library_exports_every_declared_symbol(lib):
    from paper_2506_19370_gb300 import fcsdnn
    names = declared_functions()
    for n in names:
        assert hasattr(lib, n), n
    assert sorted(fcsdnn.EXPORTS) == names


@pytest.mark.parametrize("d,C", [(5, 25), (2, 25), (5, 24), (5, 26), (5, 27), (5, 32), (5, 48)])
def test_table_builder_matches_oracle(lib, d, C):
    # the library builds its tables in double-double (Lagrange basis,
    # Householder QR); the oracle at 40 digits (Gram basis, mpmath QR)
    from oracle import fcgram
    from paper_2506_19370_gb300 import fcsdnn
    A_lib = fcsdnn.build_table(d, C)
    A_or, _ = fcgram.continuation_tables(d, C)
    scale = np.abs(A_or).max()
    assert np.abs(A_lib - A_or).max() <= 4e-16 * scale


def test_errors_are_reported(lib):
    from paper_2506_19370_gb300 import fcsdnn
    assert lib.fcs_strerror(-2) == b"fringe point without a donor outside the donor's own fringe"
    out = np.zeros(5, dtype=np.float64)
    assert lib.fcs_build_table(1, 25, out.ctypes.data_as(ctypes.POINTER(ctypes.c_double))) == -1
    h = ctypes.c_void_p()
    assert lib.fc_setup(ctypes.byref(h), 5, 25, None, 0, None) == -1


def _setup_rc(lib, bc, lcut=(0, 0), op_form=0):
    """fc_setup return code for one 40 x 40 Cartesian patch; every case here is
    refused by the host-side validation, before any CUDA call."""
    from paper_2506_19370_gb300 import fcsdnn
    desc = (fcsdnn.PatchDesc * 1)()
    desc[0].n1 = desc[0].n2 = 40
    desc[0].cartesian = 1
    desc[0].lcut[0], desc[0].lcut[1] = lcut
    for k in range(4):
        desc[0].bc[k] = bc[k]
    desc[0].box[0], desc[0].box[1], desc[0].box[2], desc[0].box[3] = 0.0, 1.0, 0.0, 1.0
    opt = fcsdnn.Options()
    lib.fcs_default_options(ctypes.byref(opt))
    opt.op_form = op_form
    h = ctypes.c_void_p()
    rc = lib.fc_setup(ctypes.byref(h), 5, 25, desc, 1, ctypes.byref(opt))
    assert not h.value
    return rc


def test_setup_refuses_unsupported_wall_layouts_on_the_host(lib):
    NOSLIP, WALL, FREE = 5, 1, 4
    assert _setup_rc(lib, (NOSLIP, WALL, NOSLIP, WALL)) == -3         # adjacent no-slip sides
    assert _setup_rc(lib, (WALL, NOSLIP, WALL, NOSLIP)) == -3
    assert _setup_rc(lib, (NOSLIP, WALL, WALL, WALL), lcut=(20, 20)) == -3   # no-slip side on an L-shaped patch
    assert _setup_rc(lib, (6, WALL, WALL, WALL)) == -1                 # unknown side code
    assert _setup_rc(lib, (FREE, FREE, FREE, FREE), op_form=2) == -1   # unknown operator form
