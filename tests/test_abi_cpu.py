"""The C-ABI library builds for sm_103a, loads without a GPU, and exports every
entry point include/md_gb300.h declares.  No compute calls (CPU only)."""
import ctypes
import os
import re
import shutil

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "md_gb300.h")


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    names = re.findall(r"^\s*(?:md_status|void|const char\s*\*)\s*(md_\w+)\s*\(", text, flags=re.M)
    return sorted(set(names))


@pytest.fixture(scope="module")
def libpath():
    if shutil.which("nvcc") is None and not os.path.exists("/usr/local/cuda/bin/nvcc"):
        pytest.skip("nvcc not available")
    from paper_1611_00075_gb300 import build
    return build.build()


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ("md_create", "md_bin_cells", "md_build_neighbors", "md_forces", "md_step",
                     "md_energy", "md_get_state", "md_set_state", "md_get_neighbors",
                     "md_get_cells", "md_cost_model", "md_stats", "md_last_error",
                     "md_destroy"):
        assert required in names


def test_library_exports_every_declared_symbol(libpath):
    lib = ctypes.CDLL(libpath)
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, missing


def test_null_handle_errors_without_gpu(libpath):
    # argument checks run before any CUDA call
    from paper_1611_00075_gb300 import md
    L = md.lib()
    assert L.md_step(None, 1) == md.MD_ERR_INVALID
    assert L.md_forces(None) == md.MD_ERR_INVALID
    assert b"null handle" in L.md_last_error(None)
    h = ctypes.c_void_p()
    p = md.make_params()
    box = (ctypes.c_double * 3)(8.0, 8.0, 8.0)
    # box too small for 3 list radii -> rejected before touching the device
    st = L.md_create(ctypes.byref(h), ctypes.byref(p), 10, ctypes.cast(box, ctypes.c_void_p),
                     ctypes.c_void_p(1), None, None)
    assert st == md.MD_ERR_INVALID
    assert b"3 list radii" in L.md_last_error(None)


def test_python_binding_names_match_c_abi(libpath):
    from paper_1611_00075_gb300 import md
    for n in declared_functions():
        if n == "md_last_error":
            continue
        assert hasattr(md, n), n


@pytest.mark.parametrize("ncell", [(3, 3, 3), (4, 5, 6), (7, 3, 8), (9, 10, 11), (5, 5, 5)])
def test_cell_colouring_is_conflict_free(libpath, ncell):
    """Race check of MD_FORCE_HALF_COLOR on the host: two distinct cells of one
    colour must have disjoint (periodic) 27-cell neighbourhoods, since a cell's
    force task writes to every atom of its neighbourhood."""
    import numpy as np
    from paper_1611_00075_gb300 import md
    col, k = md.md_color_cells(ncell)
    nx, ny, nz = ncell
    col = np.array(col).reshape(nz, ny, nx)
    assert len(np.unique(col)) == k
    def neigh(c):
        x, y, z = c
        return {((x + a) % nx, (y + b) % ny, (z + d) % nz)
                for a in (-1, 0, 1) for b in (-1, 0, 1) for d in (-1, 0, 1)}
    cells = [(x, y, z) for z in range(nz) for y in range(ny) for x in range(nx)]
    by_colour = {}
    for c in cells:
        by_colour.setdefault(int(col[c[2], c[1], c[0]]), []).append(c)
    for group in by_colour.values():
        seen = set()
        for c in group:
            nb = neigh(c)
            assert not (nb & seen), (ncell, c)
            seen |= nb


@pytest.mark.parametrize("fn", ["md_partition", "md_partition_noalloc"])
def test_partition_binding_refuses_bad_tensors(fn):
    """The binding refuses, before any call into the library, cost or
    bounds tensors the C call would read or write out of bounds."""
    torch = pytest.importorskip("torch")
    from paper_1611_00075_gb300 import md
    call = getattr(md, fn)
    good = torch.zeros(8, dtype=torch.int64)  # a host tensor: refused as well
    for cost, bounds in ((torch.zeros(8, dtype=torch.int32), good),
                         (good, torch.zeros(3, dtype=torch.int64)),
                         (good, good[::2]),
                         (good, good)):
        with pytest.raises(md.MDError) as e:
            call(cost, 4, bounds)
        assert e.value.status == md.MD_ERR_INVALID
