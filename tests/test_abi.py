"""The C ABI: the library loads, exports every entry point include/wf.h
declares, its structs match the binding, and argument checks that need no
GPU reject bad input with WF_EINVAL."""
import ctypes
import os
import re
import subprocess
import tempfile

import numpy as np
import pytest

from paper_1211_0585_gb300 import build as B
from paper_1211_0585_gb300 import wf

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "wf.h")


@pytest.fixture(scope="module")
def lib():
    B.build()
    return wf.load()


def declared_functions():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(wf_[a-z_0-9]+)\s*\(", src)))


def test_exports_every_declared_symbol(lib):
    names = declared_functions()
    assert "wf_solve" in names and "wf_plan_create" in names and len(names) >= 18
    for n in names:
        assert hasattr(lib, n), n
    assert sorted(names) == sorted(wf.EXPORTED)


def test_struct_layouts_match_header():
    """Every field of the binding's structs sits where the C compiler puts it
    (the header is compiled by gcc, offsets printed per field)."""
    structs = {"wf_options": wf.Options, "wf_stats": wf.Stats, "wf_iter_record": wf.IterRecord}
    lines = []
    want = []
    for cname, py in structs.items():
        lines.append(f'printf("%zu\\n", sizeof({cname}));')
        want.append(ctypes.sizeof(py))
        for fname, _ in py._fields_:
            cfield = fname[:-1] if fname.endswith("_") else fname  # lambda_: a Python keyword in C's name
            lines.append(f'printf("%zu\\n", offsetof({cname}, {cfield}));')
            want.append(getattr(py, fname).offset)
    code = "#include <stdio.h>\n#include <stddef.h>\n#include \"wf.h\"\nint main(void) {\n" + \
        "\n".join(lines) + "\nreturn 0;\n}\n"
    with tempfile.TemporaryDirectory() as td:
        c = os.path.join(td, "t.c")
        exe = os.path.join(td, "t")
        open(c, "w").write(code)
        subprocess.check_call(["gcc", "-I", os.path.join(ROOT, "include"), c, "-o", exe])
        got = [int(x) for x in subprocess.check_output([exe]).split()]
    assert got == want


def test_defaults(lib):
    o = wf.options()
    assert (o.tol, o.max_iter, o.l_iter0, o.lmax_margin, o.cooling, o.band_limit) == (1e-6, 10000, 20, 100, 1, 1)


@pytest.mark.parametrize("nside,lmax", [(0, 4), (3, 4), (4096, 10), (4, -1), (4, 17), (2048, 4097)])
def test_bad_sizes_rejected(lib, nside, lmax):
    # sizes are checked before any per-pixel array is read: the large cases pass a short one
    npix = max(12 * nside * nside, 1) if nside <= 64 else 1
    h = ctypes.c_void_p()
    cl = np.ones(max(lmax + 1, 1))
    nv = np.ones(npix)
    st = lib.wf_plan_create(nside, lmax, cl.ctypes.data_as(ctypes.c_void_p), nv.ctypes.data_as(ctypes.c_void_p),
                            None, None, ctypes.byref(h))
    assert st == wf.WF_EINVAL
    assert wf.last_error()


BAD_OPTIONS = {"bad_opt": dict(max_iter=0), "synthesis_table_high": dict(synthesis_table=3),
               "synthesis_table_low": dict(synthesis_table=-2), "slots_high": dict(batch_slots=65),
               "slots_low": dict(batch_slots=0), "graph_iters": dict(graph_iters=0), "precision": dict(precision=3)}


@pytest.mark.parametrize("bad", ["nan_var", "neg_var", "all_masked", "neg_cl"] + list(BAD_OPTIONS))
def test_bad_values_rejected(lib, bad):
    nside, lmax = 4, 8
    npix = 12 * nside * nside
    cl, nv, mask = np.ones(lmax + 1), np.ones(npix), np.ones(npix, np.uint8)
    opt = None
    if bad == "nan_var":
        nv[5] = np.nan
    elif bad == "neg_var":
        nv[7] = -1.0
    elif bad == "all_masked":
        mask[:] = 0
    elif bad == "neg_cl":
        cl[3] = -1.0
    else:
        opt = wf.options(**BAD_OPTIONS[bad])
    h = ctypes.c_void_p()
    st = lib.wf_plan_create(nside, lmax, cl.ctypes.data_as(ctypes.c_void_p), nv.ctypes.data_as(ctypes.c_void_p),
                            mask.ctypes.data_as(ctypes.c_void_p), ctypes.byref(opt) if opt else None,
                            ctypes.byref(h))
    assert st == wf.WF_EINVAL, wf.last_error()


def test_masked_pixels_may_hold_anything(lib):
    """A masked pixel's variance is never read (N^-1 = 0 there)."""
    nside, lmax = 2, 4
    npix = 12 * nside * nside
    nv = np.ones(npix)
    mask = np.ones(npix, np.uint8)
    nv[3], mask[3] = np.nan, 0
    h = ctypes.c_void_p()
    st = lib.wf_plan_create(nside, lmax, np.ones(lmax + 1).ctypes.data_as(ctypes.c_void_p),
                            nv.ctypes.data_as(ctypes.c_void_p), mask.ctypes.data_as(ctypes.c_void_p), None,
                            ctypes.byref(h))
    assert st != wf.WF_EINVAL
    if st == wf.WF_OK:
        lib.wf_plan_destroy(h)


def test_null_arguments(lib):
    assert lib.wf_solve(None, None, 0, None, 0, None, None) == wf.WF_EINVAL
    assert lib.wf_alm2map(None, 0, None, None) == wf.WF_EINVAL
    assert lib.wf_plan_kernels_per_iteration(None, None) == wf.WF_EINVAL
    assert lib.wf_plan_destroy(None) == wf.WF_OK
