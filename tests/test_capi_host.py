"""Host-side checks of the C ABI (no GPU): exported symbols, argument
validation, and bit-exact agreement of the host planner with the oracle's
layout definitions."""
import ctypes
import glob
import os
import re
import shutil
import subprocess

import numpy as np
import pytest

import fegen
from oracle import layout
import paper_1501_00324_gb300 as fs

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = []
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        text = open(h).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        text = re.sub(r"//[^\n]*", "", text)
        for m in re.finditer(r"^[A-Za-z_][\w \t\*]*?\b([A-Za-z_]\w*)\s*\([^;{]*\)\s*;", text, re.M):
            if not m.group(0).lstrip().startswith(("typedef", "#")):
                names.append(m.group(1))
    return sorted(set(names))


def test_library_exports_every_declared_symbol():
    names = declared_functions()
    assert {"spmv_create", "spmv_apply", "spmv_destroy", "spmv_plan"} <= set(names)
    lib = ctypes.CDLL(fs.LIB_PATH)
    missing = [n for n in names if not hasattr(lib, n)]
    assert not missing, missing


def test_library_exports_only_the_declared_symbols():
    """Hidden visibility and the link's version script leave the header's C functions
    as the library's whole dynamic interface: no internal or template symbol leaks."""
    nm = shutil.which("nm")
    if nm is None:
        pytest.skip("nm is not installed")
    out = subprocess.run([nm, "-D", "--defined-only", fs.LIB_PATH], capture_output=True, text=True,
                         check=True).stdout
    exported = {ln.split()[-1] for ln in out.splitlines() if ln.strip()}
    assert exported == set(declared_functions())


def test_status_strings():
    lib = fs.lib()
    assert lib.fespmv_status_string(0) == b"ok"
    assert lib.fespmv_status_string(fs.FESPMV_ERR_BAD_CSR) == b"malformed CSR"


def _expect(status, fn, *a, **k):
    with pytest.raises(fs.FespmvError) as e:
        fn(*a, **k)
    assert e.value.status == status


def test_create_rejects_bad_arguments_before_touching_the_device():
    p = fegen.cube_laplace(3, 1)
    rp, ci, v = p.rowptr, p.colind, p.values
    _expect(fs.FESPMV_ERR_INVALID_ARG, fs.spmv_create, rp, ci, v, format=7)
    _expect(fs.FESPMV_ERR_INVALID_ARG, fs.spmv_create, rp, ci, v, vec=3)
    _expect(fs.FESPMV_ERR_INVALID_ARG, fs.spmv_create, rp, ci, v, format=0, csr_lanes=3)
    _expect(fs.FESPMV_ERR_INVALID_ARG, fs.spmv_create, rp, ci, v, block=100)
    _expect(fs.FESPMV_ERR_INVALID_ARG, fs.spmv_create, rp, ci, v,
            reorder=fs.FESPMV_REORDER_MORTON)                     # Morton without coordinates
    bad = ci.copy()
    bad[5] = p.n_rows                                             # column out of range
    _expect(fs.FESPMV_ERR_BAD_CSR, fs.spmv_create, rp, bad, v)
    bad[5] = -1
    _expect(fs.FESPMV_ERR_BAD_CSR, fs.spmv_create, rp, bad, v)
    rp2 = rp.copy()
    rp2[3] = rp2[4] + 1                                           # offsets decrease
    _expect(fs.FESPMV_ERR_BAD_CSR, fs.spmv_create, rp2, ci, v)
    rp3 = rp.copy()
    rp3[0] = 1
    _expect(fs.FESPMV_ERR_BAD_CSR, fs.spmv_create, rp3, ci, v)
    h = ctypes.c_void_p()
    assert fs.lib().spmv_create(None, 0, None, None, None, None, None, None) == fs.FESPMV_ERR_INVALID_ARG
    assert fs.lib().spmv_create(ctypes.byref(h), -1, None, None, None, None, None, None) \
        == fs.FESPMV_ERR_INVALID_ARG


def test_plan_rejects_duplicates_and_bad_dofs():
    rowptr = np.array([0, 2, 3])
    _expect(fs.FESPMV_ERR_BAD_CSR, fs.spmv_plan, rowptr, np.array([1, 1, 0]))
    _expect(fs.FESPMV_ERR_INVALID_ARG, fs.spmv_plan, np.array([0, 1, 2, 3]), np.array([0, 1, 2]),
            dofs_per_node=2)


def oracle_plan(p, reorder, sigma, threshold, V, use_xyz=True):
    P = layout.row_permutation(p.rowptr, p.dofs_per_node, p.node_xyz if use_xyz else None,
                               reorder, sigma)
    rp2, ci2, v2, vmap = layout.permute_csr(p.rowptr, p.colind, p.values, P)
    meta, col, val, pmap = layout.pack(rp2, ci2, v2, threshold, V)
    src = np.full(len(col), -1, dtype=np.int64)
    src[pmap[vmap]] = np.arange(p.nnz)
    return P, meta, col, src


CASES = [
    (lambda: fegen.cube_laplace(7, 31), "morton", 0, 0, 1),
    (lambda: fegen.cube_laplace(7, 32), "morton", 64, 0, 2),
    (lambda: fegen.cube_laplace(8, 33, dirichlet=False), "morton", 10**9, 4, 2),
    (lambda: fegen.cube_elasticity(5, 34), "morton", 96, 0, 2),
    (lambda: fegen.cube_elasticity(4, 35), "none", 32, 8, 4),
    (lambda: fegen.shell_laplace(4, 8, 12, 36), "morton", 128, 3, 1),
    (lambda: fegen.shell_laplace(3, 6, 10, 37), "none", 0, 0, 4),
]


@pytest.mark.parametrize("case", range(len(CASES)))
def test_host_planner_matches_oracle_bit_exactly(case):
    make, reorder, sigma, threshold, V = CASES[case]
    p = make()
    P, meta, col, src = oracle_plan(p, reorder, sigma, threshold, V)
    got = fs.spmv_plan(p.rowptr, p.colind, p.node_xyz if reorder == "morton" else None,
                       p.dofs_per_node, fs.FESPMV_REORDER_MORTON if reorder == "morton"
                       else fs.FESPMV_REORDER_NONE, sigma, threshold, V)
    assert np.array_equal(got["perm"], P.astype(np.int32))
    assert np.array_equal(got["meta"], meta)
    assert np.array_equal(got["cols"], col)
    assert np.array_equal(got["srcmap"], src)


def test_planner_edge_cases():
    # empty matrix
    g = fs.spmv_plan(np.array([0]), np.array([], dtype=np.int32))
    assert g["perm"].size == 0 and g["meta"].size == 0 and g["cols"].size == 0
    # empty rows and a ragged tail (n not a multiple of 32)
    n = 37
    lens = np.array([0 if i % 5 == 0 else 1 + i % 4 for i in range(n)])
    rowptr = np.concatenate([[0], np.cumsum(lens)])
    cols = np.concatenate([np.sort(np.random.default_rng(i).choice(n, lens[i], replace=False))
                           for i in range(n)]).astype(np.int32)
    for thr, V in ((0, 1), (1, 2), (2, 4)):
        got = fs.spmv_plan(rowptr, cols, None, 1, fs.FESPMV_REORDER_NONE, 8, thr, V)
        P = layout.row_permutation(rowptr, 1, None, "none", 8)
        rp2, ci2, v2, vmap = layout.permute_csr(rowptr, cols, np.ones(len(cols)), P)
        meta, col, _, pmap = layout.pack(rp2, ci2, v2, thr, V)
        assert np.array_equal(got["meta"], meta) and np.array_equal(got["cols"], col)


@pytest.mark.parametrize("case", range(len(CASES)))
def test_host_tiles_match_oracle_bit_exactly(case):
    """The tile builder (x staging) against oracle.layout.tiles, on spmv_plan's layout."""
    make, reorder, sigma, threshold, V = CASES[case]
    p = make()
    got = fs.spmv_plan(p.rowptr, p.colind, p.node_xyz if reorder == "morton" else None,
                       p.dofs_per_node, fs.FESPMV_REORDER_MORTON if reorder == "morton"
                       else fs.FESPMV_REORDER_NONE, sigma, threshold, V)
    t = fs.spmv_plan_tiles(p.n_rows, got["meta"], got["cols"])
    o = layout.tiles(got["meta"], got["cols"], 8, 4096)
    assert np.array_equal(t[0], o[0]) and np.array_equal(t[1], o[1]) and np.array_equal(t[2], o[2])


def test_host_tiles_wide_slice_and_bad_input():
    n = 20000
    rng = np.random.default_rng(61)
    rows = [np.sort(rng.choice(n, 200, replace=False)) if i < 32 else np.array([i]) for i in range(n)]
    rowptr = np.concatenate([[0], np.cumsum([len(r) for r in rows])])
    cols = np.concatenate(rows).astype(np.int32)
    got = fs.spmv_plan(rowptr, cols, sigma=0)
    assert fs.spmv_plan_tiles(n, got["meta"], got["cols"]) is None
    assert layout.tiles(got["meta"], got["cols"], 8, 4096) is None
    bad = got["cols"].copy()
    bad[3] = n
    _expect(fs.FESPMV_ERR_INVALID_ARG, fs.spmv_plan_tiles, n, got["meta"], bad)
    _expect(fs.FESPMV_ERR_INVALID_ARG, fs.spmv_plan_tiles, n, got["meta"], got["cols"][:10])
