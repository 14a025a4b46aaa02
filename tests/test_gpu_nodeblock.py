"""3x3 node blocks (spmv_create with node_blocks = 3) on the GPU.

- Layout (integer work, bit-exact): the handle's permutation, slice metadata,
  block columns and value map equal oracle/layout.py's node_row_permutation /
  node_blocks; the FP32 / BF16 block values are the oracle's S A S values at
  the mapped entries (zero elsewhere), bit for bit.
- Products y = B x: within 2 L 2^-24 (|B||x|)_i of the oracle's float product
  (as the scalar float products), in both numberings, every row at full size.
- The refined CG on such a handle reaches the FP64 tolerance on the true
  residual and takes a step count close to the oracle's reliable-update
  refinement; values assembled on the GPU refresh the blocks bit for bit.
"""
import numpy as np
import pytest

import fegen
import oracle
from oracle import layout

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_1501_00324_gb300 as fs  # noqa: E402

PREC = {"f32": fs.FESPMV_PREC_F32, "bf16": fs.FESPMV_PREC_BF16}
BOTH = fs.FESPMV_PREC_F32 | fs.FESPMV_PREC_BF16


def make(p, sigma=96, **kw):
    return fs.spmv_create(p.rowptr, p.colind, p.values, p.node_xyz, 3, sigma=sigma, node_blocks=3, **kw)


@pytest.mark.parametrize("sigma,vec", [(96, 1), (1024, 2), (0, 4)])
def test_layout_bit_exact(sigma, vec):
    p = fegen.cube_elasticity(7, 91)
    A = make(p, sigma, vec=vec, precisions=BOTH)
    info = fs.spmv_get_info(A)
    assert info["node_blocks"] == 3
    P = layout.node_row_permutation(p.rowptr, p.node_xyz, "morton", sigma)
    assert np.array_equal(fs.spmv_export(A, fs.FESPMV_EXPORT_PERM), P)
    rp2, c2, _, vmap = layout.permute_csr(p.rowptr, p.colind, p.values, P)
    meta, col, vidx = layout.node_blocks(rp2, c2)
    assert np.array_equal(fs.spmv_export(A, fs.FESPMV_EXPORT_NB_META), meta)
    assert np.array_equal(fs.spmv_export(A, fs.FESPMV_EXPORT_NB_COLS), col)
    # tiles of node-block slices: the generic tiling of the oracle over block columns
    tl, td, ti = layout.tiles(meta, col, 8, 2048)
    assert info["nb_tiles"] == len(tl) > 0
    assert np.array_equal(fs.spmv_export(A, fs.FESPMV_EXPORT_NB_TILES), tl)
    assert np.array_equal(fs.spmv_export(A, fs.FESPMV_EXPORT_NB_TILE_NODES), td)
    assert np.array_equal(fs.spmv_export(A, fs.FESPMV_EXPORT_NB_TILE_INDEX), ti)
    # the map points at the packed scalar positions of the same entries
    _, _, _, pmap = layout.pack(rp2, c2, np.zeros(len(c2)), 0, vec)
    want = np.where(vidx >= 0, pmap[np.maximum(vidx, 0)], -1)
    assert np.array_equal(fs.spmv_export(A, fs.FESPMV_EXPORT_NB_MAP), want)
    # block values: the oracle's S A S at those entries (input position = inverse of vmap)
    inp = np.empty_like(vmap)
    inp[vmap] = np.arange(len(vmap))
    live = vidx >= 0
    b32 = oracle.scaled_values(p.rowptr, p.colind, p.values, "f32")
    b16 = oracle.scaled_values(p.rowptr, p.colind, p.values, "bf16")
    g32 = fs.spmv_export(A, fs.FESPMV_EXPORT_NB_VALUES_F32)
    g16 = fs.spmv_export(A, fs.FESPMV_EXPORT_NB_VALUES_BF16)
    assert np.array_equal(g32[live].view(np.uint32), b32[inp[vidx[live]]].view(np.uint32))
    assert np.array_equal(g16[live], (b16[inp[vidx[live]]].view(np.uint32) >> 16).astype(np.uint16))
    assert not g32[~live].any() and not g16[~live].any()


def check_product(p, A, storage, x, permuted):
    bv = oracle.scaled_values(p.rowptr, p.colind, p.values, storage)
    xd = torch.from_numpy(x).cuda()
    yd = torch.full_like(xd, float("nan"))
    if permuted:
        perm = torch.from_numpy(fs.spmv_export(A, fs.FESPMV_EXPORT_PERM).astype(np.int64)).cuda()
        xp = xd[perm].contiguous()
        yp = torch.full_like(xp, float("nan"))
        fs.spmv_apply_scaled(A, xp, yp, PREC[storage], fs.FESPMV_IO_PERMUTED)
        yd[perm] = yp
    else:
        fs.spmv_apply_scaled(A, xd, yd, PREC[storage])
    torch.cuda.synchronize()
    y = yd.cpu().numpy()
    yo = oracle.csr_spmv_f32(p.rowptr, p.colind, bv, x)
    bound = oracle.csr_spmv(p.rowptr, p.colind, np.abs(bv).astype(np.float64), np.abs(x).astype(np.float64))
    L = np.diff(p.rowptr).max()
    assert np.all(np.abs(y.astype(np.float64) - yo) <= 2 * L * 2.0 ** -24 * bound)


@pytest.mark.parametrize("tiles", [0, -1])
@pytest.mark.parametrize("permuted", [False, True])
@pytest.mark.parametrize("storage", ["f32", "bf16"])
@pytest.mark.parametrize("mesh", ["elasticity_9", "elasticity_4_ragged"])
def test_product_parity(mesh, storage, permuted, tiles):
    # 9^3 nodes: 23 slices of 32 node rows and a ragged last slice; 4^3 nodes: two
    # slices of 32 node rows with the clamped face's identity blocks; x staged per
    # tile, or gathered from L1/L2 (tiles = -1)
    p = {"elasticity_9": lambda: fegen.cube_elasticity(9, 92),
         "elasticity_4_ragged": lambda: fegen.cube_elasticity(4, 93)}[mesh]()
    A = make(p, 96, precisions=PREC[storage], tiles=tiles)
    assert (fs.spmv_get_info(A)["nb_tiles"] > 0) == (tiles == 0)
    x = fegen.random_vector(p.n_rows, 94).astype(np.float32)
    check_product(p, A, storage, x, permuted)


def test_full_size_elasticity_64_products():
    """The benchmark's matrix, every row, FP32 and BF16 node-block products."""
    p = fegen.cube_elasticity(64, 1502)
    A = make(p, 1024, vec=4, precisions=BOTH)
    x = fegen.random_vector(p.n_rows, 1504).astype(np.float32)
    for storage in ("f32", "bf16"):
        check_product(p, A, storage, x, False)


@pytest.mark.parametrize("tiles", [0, -1])
@pytest.mark.parametrize("storage", ["f32"])
def test_refined_cg_on_node_blocks(storage, tiles):
    p = fegen.cube_elasticity(10, 95)
    A = make(p, 256, precisions=PREC[storage], tiles=tiles)
    u = fegen.manufactured_solution(p)
    b = oracle.csr_spmv(p.rowptr, p.colind, p.values, u)
    bd = torch.from_numpy(b).cuda()
    for flags in (0, fs.FESPMV_CG_RELIABLE):
        xd = torch.zeros_like(bd)
        res = fs.cg_solve(A, bd, xd, tol=1e-10, precision=fs.FESPMV_CG_F32_REFINE, flags=flags)
        torch.cuda.synchronize()
        assert res["status"] == 0, (res, fs.last_error())
        x = xd.cpu().numpy()
        r = b - oracle.csr_spmv(p.rowptr, p.colind, p.values, x)
        assert np.linalg.norm(r) <= 1.01e-10 * np.linalg.norm(b)
        if flags:
            _, info = oracle.refine_reliable(p.rowptr, p.colind, p.values, b, tol=1e-10)
            assert info["status"] == "converged"
            assert abs(res["iters"] - info["iters"]) <= 0.1 * info["iters"] + 5


def test_assembly_refreshes_the_blocks():
    p = fegen.cube_elasticity(6, 96, elements=True)
    R = make(p, 96, precisions=BOTH)
    Z = fs.spmv_create(p.rowptr, p.colind, 2.0 * p.values, p.node_xyz, 3, sigma=96, node_blocks=3, precisions=BOTH)
    P = fs.assembly_create(Z, p.rowptr, p.colind, p.elem_nodes, 3, p.dirichlet)
    fs.assembly_matrix(P, torch.from_numpy(p.elem_mats).cuda())
    torch.cuda.synchronize()
    for what in (fs.FESPMV_EXPORT_NB_VALUES_F32, fs.FESPMV_EXPORT_NB_VALUES_BF16):
        assert np.array_equal(fs.spmv_export(R, what).view(np.uint8), fs.spmv_export(Z, what).view(np.uint8))


def test_node_blocks_rejected_without_three_dofs():
    p = fegen.cube_laplace(6, 97)
    with pytest.raises(fs.FespmvError):
        fs.spmv_create(p.rowptr, p.colind, p.values, p.node_xyz, 1, node_blocks=3, precisions=fs.FESPMV_PREC_F32)
    q = fegen.cube_elasticity(4, 98)
    with pytest.raises(fs.FespmvError):     # nothing to store in blocks without FP32 / BF16 values
        fs.spmv_create(q.rowptr, q.colind, q.values, q.node_xyz, 3, node_blocks=3)


@pytest.mark.parametrize("k", [1, 4, 7, 16, 32])
def test_multi_rhs_product_on_node_blocks(k):
    """Y = B X with FP32 node blocks, every column against the oracle's float product
    (bound of the single products), host-side padding of k to 4/8/16/32 included."""
    p = fegen.cube_elasticity(9, 99)
    A = make(p, 96, precisions=fs.FESPMV_PREC_F32)
    bv = oracle.scaled_values(p.rowptr, p.colind, p.values, "f32")
    X = np.stack([fegen.random_vector(p.n_rows, 200 + j) for j in range(k)], axis=1).astype(np.float32)
    Xd = torch.from_numpy(np.ascontiguousarray(X)).cuda()
    Yd = torch.full_like(Xd, float("nan"))
    fs.spmv_apply_multi(A, Xd, Yd, fs.FESPMV_PREC_F32)
    torch.cuda.synchronize()
    Y = Yd.cpu().numpy()
    L = np.diff(p.rowptr).max()
    for j in range(k):
        x = np.ascontiguousarray(X[:, j])
        yo = oracle.csr_spmv_f32(p.rowptr, p.colind, bv, x)
        bound = oracle.csr_spmv(p.rowptr, p.colind, np.abs(bv).astype(np.float64), np.abs(x).astype(np.float64))
        assert np.all(np.abs(Y[:, j].astype(np.float64) - yo) <= 2 * L * 2.0 ** -24 * bound), j


@pytest.mark.parametrize("tiles", [0, -1])
def test_smallest_mesh_on_node_blocks(tiles):
    """2^3 nodes: one slice holding 8 node rows of its 32, half of them the clamped
    face's identity blocks.  The layout is bit-exact.  Both storages' products are
    checked in both numberings.  The refined CG on the blocks reaches the tolerance,
    through the cluster path and through the graphs."""
    p = fegen.cube_elasticity(2, 97)
    A = make(p, 96, precisions=BOTH, tiles=tiles)
    P = layout.node_row_permutation(p.rowptr, p.node_xyz, "morton", 96)
    assert np.array_equal(fs.spmv_export(A, fs.FESPMV_EXPORT_PERM), P)
    rp2, c2, _, _ = layout.permute_csr(p.rowptr, p.colind, p.values, P)
    meta, col, _ = layout.node_blocks(rp2, c2)
    assert np.array_equal(fs.spmv_export(A, fs.FESPMV_EXPORT_NB_META), meta)
    assert np.array_equal(fs.spmv_export(A, fs.FESPMV_EXPORT_NB_COLS), col)
    x = fegen.random_vector(p.n_rows, 98).astype(np.float32)
    for storage in ("f32", "bf16"):
        for permuted in (False, True):
            check_product(p, A, storage, x, permuted)
    u = fegen.manufactured_solution(p)
    b = oracle.csr_spmv(p.rowptr, p.colind, p.values, u)
    assert np.linalg.norm(b) > 0
    bd = torch.from_numpy(b).cuda()
    for flags in (fs.FESPMV_CG_RELIABLE, fs.FESPMV_CG_RELIABLE | fs.FESPMV_CG_NO_CLUSTER, 0):
        xd = torch.zeros_like(bd)
        res = fs.cg_solve(A, bd, xd, tol=1e-10, precision=fs.FESPMV_CG_F32_REFINE, flags=flags)
        torch.cuda.synchronize()
        assert res["status"] == 0, (flags, res, fs.last_error())
        r = b - oracle.csr_spmv(p.rowptr, p.colind, p.values, xd.cpu().numpy())
        assert np.linalg.norm(r) <= 1.01e-10 * np.linalg.norm(b)
