"""CPU checks of the C ABI library: it builds, loads and exports every symbol
declared in include/geneo.h (no compute calls: there is no GPU here)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = set()
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if not fn.endswith(".h"):
            continue
        src = open(os.path.join(ROOT, "include", fn)).read()
        src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
        for m in re.finditer(r"^\s*(?:const\s+)?(?:long\s+)?\w+\s*\*?\s*(geneo_\w+)\s*\(", src, flags=re.M):
            names.add(m.group(1))
    return sorted(names)


@pytest.fixture(scope="module")
def lib():
    from paper_1901_05188_gb300 import build
    path = build.build()
    return ctypes.CDLL(path)


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ("geneo_create", "geneo_assemble", "geneo_setup", "geneo_solve",
                     "geneo_destroy", "geneo_apply_preconditioner", "geneo_spmv"):
        assert required in names


def test_library_exports_every_declared_symbol(lib):
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_covers_every_declared_symbol():
    import paper_1901_05188_gb300 as pkg
    assert set(declared_functions()) <= set(pkg.EXPORTED)


def test_status_strings_without_gpu(lib):
    lib.geneo_status_string.restype = ctypes.c_char_p
    assert lib.geneo_status_string(0) == b"ok"
    assert lib.geneo_status_string(4) == b"matrix not positive definite"


def test_workspace_size_query_is_host_only(lib):
    import paper_1901_05188_gb300 as pkg
    pkg.load()
    import numpy as np
    x = np.arange(9, dtype=np.float64)
    m = pkg.geneo_mesh(8, 8, 8, x.ctypes.data, x.ctypes.data, x.ctypes.data)
    n = pkg.geneo_assemble_workspace_bytes(m)
    # BSR values alone take 27 * 729 * 9 doubles
    assert n > 27 * 729 * 9 * 8


def test_binding_refuses_other_elements():
    # the library meshes with trilinear hexahedra only: a 20-node problem (which
    # the oracle can build) is refused before anything reaches the GPU
    import paper_1901_05188_gb300 as pkg
    from workloads.laminate import make_block
    p = make_block(2, 2, 2, [0.0, 90.0], partition=(1, 1, 1, 1))
    pkg.GeneoSolver.check_element(p)
    q = dict(p, element="serendipity")
    with pytest.raises(ValueError, match="trilinear"):
        pkg.GeneoSolver.check_element(q)
