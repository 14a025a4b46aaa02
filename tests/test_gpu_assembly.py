"""Assembly as a sparse product (assembly_*, Sec. 4) on the GPU.

The element matrices come from the generator; the oracle's assembly of them
equals the generator's CSR values bit for bit (tests/test_oracle_pins.py).  A
handle whose values the GPU assembles must therefore hold exactly the values,
diagonal, scale and low-precision copies of a handle created from those CSR
values: every comparison below is bitwise.
"""
import numpy as np
import pytest

import fegen
import oracle

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_1501_00324_gb300 as fs  # noqa: E402

MESHES = {"cube_laplace_10": lambda: fegen.cube_laplace(10, 501, elements=True),
          "elasticity_7": lambda: fegen.cube_elasticity(7, 502, elements=True),
          "shell_4x12x16": lambda: fegen.shell_laplace(4, 12, 16, 503, elements=True),
          "elasticity_6_neumann": lambda: fegen.cube_elasticity(6, 504, dirichlet=False, elements=True)}

FORMATS = {"tiled": dict(sigma=256), "untiled_v1": dict(sigma=256, tiles=-1, vec=1),
           "k2": dict(sigma=64, threshold=3, vec=4), "csr": dict(format=fs.FESPMV_FMT_CSR, csr_lanes=4),
           "float_pairs": dict(sigma=256, prec=fs.FESPMV_PREC_DF64)}


def handle(p, values, fmt):
    kw = dict(FORMATS[fmt])
    prec = fs.FESPMV_PREC_F32 | fs.FESPMV_PREC_BF16 | kw.pop("prec", 0)
    return fs.spmv_create(p.rowptr, p.colind, values, p.node_xyz, p.dofs_per_node, precisions=prec, **kw)


EXPORTS = (fs.FESPMV_EXPORT_VALUES, fs.FESPMV_EXPORT_DIAG, fs.FESPMV_EXPORT_SCALE,
           fs.FESPMV_EXPORT_VALUES_F32, fs.FESPMV_EXPORT_VALUES_BF16)


def same_handles(R, Z, exports=EXPORTS):
    for what in exports:
        a, b = fs.spmv_export(R, what), fs.spmv_export(Z, what)
        assert len(a) > 0 and np.array_equal(a.view(np.uint8), b.view(np.uint8)), what


def dirichlet_of(p):
    return p.dirichlet if p.dirichlet.any() else None


@pytest.mark.parametrize("fmt", list(FORMATS))
@pytest.mark.parametrize("mesh", list(MESHES))
def test_assembled_values_equal_a_handle_of_the_assembled_csr(mesh, fmt):
    p = MESHES[mesh]()
    assert np.array_equal(oracle.assemble_matrix(p.rowptr, p.colind, p.elem_nodes, p.elem_mats,
                                                 p.dofs_per_node, dirichlet_of(p)), p.values)
    R = handle(p, p.values, fmt)
    Z = handle(p, 2.0 * p.values, fmt)                 # other values, same pattern
    P = fs.assembly_create(Z, p.rowptr, p.colind, p.elem_nodes, p.dofs_per_node, dirichlet_of(p))
    assert fs.assembly_get_info(P)["contributions"] > 0
    fs.assembly_matrix(P, torch.from_numpy(p.elem_mats).cuda())
    torch.cuda.synchronize()
    same_handles(R, Z)
    # the products agree bit for bit as well
    x = torch.from_numpy(fegen.random_vector(p.n_rows, 505)).cuda()
    yr, yz = torch.empty_like(x), torch.empty_like(x)
    fs.spmv_apply(R, x, yr)
    fs.spmv_apply(Z, x, yz)
    torch.cuda.synchronize()
    assert torch.equal(yr, yz)


def test_host_element_matrices_and_repeated_assembly():
    """Element matrices from host memory; a second assembly of doubled element
    matrices gives exactly doubled values (a Newton step's refresh), and the
    solve on the assembled handle equals the solve on a handle of the CSR."""
    p = MESHES["elasticity_7"]()
    Z = handle(p, 3.0 * p.values, "tiled")
    P = fs.assembly_create(Z, p.rowptr, p.colind, p.elem_nodes, 3, p.dirichlet)
    fs.assembly_matrix(P, p.elem_mats)
    R = handle(p, p.values, "tiled")
    same_handles(R, Z)
    b = torch.from_numpy(fegen.random_vector(p.n_rows, 506)).cuda()
    xr, xz = torch.zeros_like(b), torch.zeros_like(b)
    rr = fs.cg_solve(R, b, xr, tol=1e-10)
    rz = fs.cg_solve(Z, b, xz, tol=1e-10)
    torch.cuda.synchronize()
    assert rr["status"] == rz["status"] == 0 and rr["iters"] == rz["iters"] and torch.equal(xr, xz)
    fs.assembly_matrix(P, 2.0 * p.elem_mats)
    R2 = handle(p, np.where(p.dirichlet[np.repeat(np.arange(p.n_rows), np.diff(p.rowptr))] == 1,
                            p.values, 2.0 * p.values), "tiled")
    same_handles(R2, Z)


@pytest.mark.parametrize("permuted", [False, True])
@pytest.mark.parametrize("mesh", ["elasticity_7", "shell_4x12x16"])
def test_assembled_vectors_equal_the_oracle(mesh, permuted):
    p = MESHES[mesh]()
    dpn = p.dofs_per_node
    u = fegen.random_vector(p.n_rows, 507)
    idx = (dpn * p.elem_nodes[:, :, None] + np.arange(dpn)[None, None, :]).reshape(p.n_elems, -1)
    re = np.einsum("eij,ej->ei", p.elem_mats, u[idx])
    ro = oracle.assemble_vector(p.n_rows, p.elem_nodes, re, dpn, dirichlet_of(p))
    A = handle(p, p.values, "tiled")
    P = fs.assembly_create(A, p.rowptr, p.colind, p.elem_nodes, dpn, dirichlet_of(p))
    r = torch.full((p.n_rows,), float("nan"), dtype=torch.float64, device="cuda")
    fs.assembly_vector(P, torch.from_numpy(re).cuda(), r, fs.FESPMV_IO_PERMUTED if permuted else 0)
    torch.cuda.synchronize()
    got = r.cpu().numpy()
    if permuted:
        perm = fs.spmv_export(A, fs.FESPMV_EXPORT_PERM)
        unp = np.empty_like(got)
        unp[perm] = got
        got = unp
    assert np.array_equal(got.view(np.uint64), ro.view(np.uint64))


def test_assembly_errors():
    p = MESHES["cube_laplace_10"]()
    A = handle(p, p.values, "tiled")
    bad_nodes = p.elem_nodes.copy()
    bad_nodes[3, 2] = p.n_rows                          # outside the node range
    with pytest.raises(fs.FespmvError) as e:
        fs.assembly_create(A, p.rowptr, p.colind, bad_nodes, 1, p.dirichlet)
    assert e.value.status == fs.FESPMV_ERR_INVALID_ARG
    with pytest.raises(fs.FespmvError) as e:            # the mask left out: contributions to dropped entries
        fs.assembly_create(A, p.rowptr, p.colind, p.elem_nodes, 1, None)
    assert e.value.status == fs.FESPMV_ERR_BAD_CSR
    rp = p.rowptr.copy()                                # a pattern with another nnz (one entry short)
    rp[-1] -= 1
    with pytest.raises(fs.FespmvError) as e:
        fs.assembly_create(A, rp, p.colind[:-1], p.elem_nodes, 1, p.dirichlet)
    assert e.value.status == fs.FESPMV_ERR_INVALID_ARG


def test_assembly_full_size_elasticity_64():
    """The 64^3 elasticity matrix (1.5 M tetrahedra, 214 M contributions): the
    assembled handle equals the handle of the generator's CSR, bit for bit."""
    p = fegen.cube_elasticity(64, 1502, elements=True)
    R = fs.spmv_create(p.rowptr, p.colind, p.values, p.node_xyz, 3, sigma=1024, vec=1,
                       precisions=fs.FESPMV_PREC_F32)
    Z = fs.spmv_create(p.rowptr, p.colind, 2.0 * p.values, p.node_xyz, 3, sigma=1024, vec=1,
                       precisions=fs.FESPMV_PREC_F32)
    P = fs.assembly_create(Z, p.rowptr, p.colind, p.elem_nodes, 3, p.dirichlet)
    Ke = torch.from_numpy(p.elem_mats).cuda()
    fs.assembly_matrix(P, Ke)
    torch.cuda.synchronize()
    same_handles(R, Z, (fs.FESPMV_EXPORT_VALUES, fs.FESPMV_EXPORT_DIAG, fs.FESPMV_EXPORT_VALUES_F32))


def test_assembly_edge_cases():
    """No elements at all (every row constrained: the identity), permuted vectors on a
    CSR handle rejected, and a second map on the same handle giving the same values."""
    n = 40
    rowptr = np.arange(n + 1, dtype=np.int64)
    colind = np.arange(n, dtype=np.int32)
    A = fs.spmv_create(rowptr, colind, np.full(n, 3.0), sigma=8, precisions=fs.FESPMV_PREC_F32)
    P = fs.assembly_create(A, rowptr, colind, np.zeros((0, 4), dtype=np.int32), 1, np.ones(n, dtype=np.uint8))
    assert fs.assembly_get_info(P)["contributions"] == 0
    fs.assembly_matrix(P, torch.zeros(1, dtype=torch.float64, device="cuda"))
    torch.cuda.synchronize()
    info = fs.spmv_get_info(A)
    vals = fs.spmv_export(A, fs.FESPMV_EXPORT_VALUES)
    assert np.array_equal(np.sort(vals)[-n:], np.ones(n)) and np.count_nonzero(vals) == n
    assert np.array_equal(fs.spmv_export(A, fs.FESPMV_EXPORT_DIAG), np.ones(n))
    assert info["packed_len"] >= n
    p = MESHES["elasticity_7"]()
    C = handle(p, 2.0 * p.values, "csr")
    Q = fs.assembly_create(C, p.rowptr, p.colind, p.elem_nodes, 3, p.dirichlet)
    r = torch.zeros(p.n_rows, dtype=torch.float64, device="cuda")
    re = torch.zeros((p.n_elems, 12), dtype=torch.float64, device="cuda")
    with pytest.raises(fs.FespmvError) as e:
        fs.assembly_vector(Q, re, r, fs.FESPMV_IO_PERMUTED)
    assert e.value.status == fs.FESPMV_ERR_INVALID_ARG
    Z = handle(p, 2.0 * p.values, "tiled")
    P1 = fs.assembly_create(Z, p.rowptr, p.colind, p.elem_nodes, 3, p.dirichlet)
    P2 = fs.assembly_create(Z, p.rowptr, p.colind, p.elem_nodes, 3, p.dirichlet)
    Ke = torch.from_numpy(p.elem_mats).cuda()
    fs.assembly_matrix(P1, Ke)
    v1 = fs.spmv_export(Z, fs.FESPMV_EXPORT_VALUES).copy()
    fs.assembly_matrix(P2, 3.0 * Ke)
    fs.assembly_matrix(P2, Ke)
    assert np.array_equal(v1, fs.spmv_export(Z, fs.FESPMV_EXPORT_VALUES))


@pytest.mark.parametrize("fmt", ["tiled", "csr"])
def test_assembly_partial_node_masks_and_uncontributed_entries(fmt):
    """Three dofs per node with single dofs marked (nodes partly constrained) on a
    pattern that keeps every entry, plus one stored entry no element touches: the
    assembled handle equals the handle of the oracle's assembly, bit for bit
    (marked rows: unit diagonal and zeros; entries with a marked column: zero; the
    untouched entry: zero)."""
    p = MESHES["elasticity_6_neumann"]()
    rng = np.random.default_rng(508)
    mask = (rng.random(p.n_rows) < 0.1).astype(np.uint8)
    # one more stored entry in row 0, at a column no element couples to it
    row0 = set(p.colind[p.rowptr[0]:p.rowptr[1]].tolist())
    extra = next(c for c in range(p.n_rows - 1, 0, -1) if c not in row0)
    cols0 = np.sort(np.array(sorted(row0) + [extra], dtype=np.int32))
    colind = np.concatenate([cols0, p.colind[p.rowptr[1]:]]).astype(np.int32)
    rowptr = p.rowptr.copy()
    rowptr[1:] += 1
    vals = oracle.assemble_matrix(rowptr, colind, p.elem_nodes, p.elem_mats, 3, mask)
    kw = dict(FORMATS[fmt])
    R = fs.spmv_create(rowptr, colind, vals, p.node_xyz, 3, precisions=fs.FESPMV_PREC_F32, **kw)
    Z = fs.spmv_create(rowptr, colind, 2.0 * vals + 1.0, p.node_xyz, 3, precisions=fs.FESPMV_PREC_F32, **kw)
    P = fs.assembly_create(Z, rowptr, colind, p.elem_nodes, 3, mask)
    fs.assembly_matrix(P, torch.from_numpy(p.elem_mats).cuda())
    torch.cuda.synchronize()
    same_handles(R, Z, (fs.FESPMV_EXPORT_VALUES, fs.FESPMV_EXPORT_DIAG, fs.FESPMV_EXPORT_VALUES_F32))


@pytest.mark.parametrize("fmt", list(FORMATS))
def test_assembly_on_the_smallest_mesh(fmt):
    """2^3 nodes, 6 tets, half the nodes clamped: the assembled handle equals a handle
    of the generator's CSR bit for bit, products included."""
    p = fegen.cube_elasticity(2, 506, elements=True)
    assert np.array_equal(oracle.assemble_matrix(p.rowptr, p.colind, p.elem_nodes, p.elem_mats,
                                                 p.dofs_per_node, dirichlet_of(p)), p.values)
    R = handle(p, p.values, fmt)
    Z = handle(p, 2.0 * p.values, fmt)
    P = fs.assembly_create(Z, p.rowptr, p.colind, p.elem_nodes, p.dofs_per_node, dirichlet_of(p))
    assert fs.assembly_get_info(P)["contributions"] > 0
    fs.assembly_matrix(P, torch.from_numpy(p.elem_mats).cuda())
    torch.cuda.synchronize()
    same_handles(R, Z)
    x = torch.from_numpy(fegen.random_vector(p.n_rows, 507)).cuda()
    yr, yz = torch.empty_like(x), torch.empty_like(x)
    fs.spmv_apply(R, x, yr)
    fs.spmv_apply(Z, x, yz)
    torch.cuda.synchronize()
    assert torch.equal(yr, yz)
