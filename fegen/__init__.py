"""Seeded synthetic finite-element inputs (shared by the oracle and the CUDA path).

This module generates the stiffness matrices and vectors that the tests, the
benchmark and the CPU oracle consume.  It holds none of the arithmetic of the
method under test (no sparse product, no conjugate gradient): random numbers are
drawn here with numpy's PCG64 generator and handed to ``fegen.c``, which only
computes P1 element matrices and assembles them (paper Sec. 2: linear
tetrahedra, one integration point, D = d_iso I + d_ani n (x) n).

Workloads (all sizes are node grids, hex cells split into 6 Kuhn tetrahedra):

* ``cube_laplace``      unit cube, D = I, interior nodes jittered +-0.2h,
                        random node numbering, Dirichlet on the z=0 face.
                        (+-0.2h almost never inverts a Kuhn tetrahedron -- its
                        smallest height is h/sqrt(2) = 0.707h -- but a tilted
                        face can; the generator then raises, and the pools
                        below redraw with the next seed, see valid_seed.)
* ``cube_elasticity``   unit cube, 3 dof/node (dof = 3*node + c), per-tet
                        Young's modulus log-uniform in [0.5, 2], nu = 0.3,
                        clamped (all 3 dof) on the z=0 face.
* ``shell_laplace``     thick truncated prolate-spheroidal shell on an
                        (r, theta, phi) grid, phi periodic, fibre direction
                        rotating from +60 deg (inner wall) to -60 deg (outer
                        wall), D = I + 8 n n^T (9:1 anisotropy), Dirichlet on
                        the base (theta = theta_base) face.  Jitter is +-0.15
                        cell in (r, theta, phi) index space: the curved map
                        eats into the 0.707 - 0.69 margin that +-0.2 leaves.
"""
from __future__ import annotations

import ctypes
import dataclasses
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "fegen.c")
_BUILD = os.path.join(_HERE, "_build")
_SO = os.path.join(_BUILD, "libfegen.so")
_lib_handle = None


def build(force: bool = False) -> str:
    """Compile fegen.c into fegen/_build/libfegen.so (gcc, portable flags)."""
    os.makedirs(_BUILD, exist_ok=True)
    if force or not os.path.exists(_SO) or os.path.getmtime(_SO) < os.path.getmtime(_SRC):
        tmp = _SO + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-fPIC", "-shared", "-ffp-contract=off", "-fopenmp",
                               "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _SO)
    return _SO


def _lib():
    global _lib_handle
    if _lib_handle is None:
        lib = ctypes.CDLL(build())
        P = ctypes.c_void_p
        i32, i64, dbl = ctypes.c_int, ctypes.c_int64, ctypes.c_double
        lib.fegen_node_degrees.argtypes = [i32, i32, i32, i32, P, P]
        lib.fegen_node_degrees.restype = i32
        lib.fegen_assemble.argtypes = [i32, i32, i32, i32, i32, P, P, P, dbl, dbl, dbl,
                                       P, P, P, P]
        lib.fegen_assemble.restype = i32
        lib.fegen_dirichlet.argtypes = [i64, P, P, P, P]
        lib.fegen_dirichlet.restype = i64
        lib.fegen_elements.argtypes = [i32, i32, i32, i32, i32, P, P, P, dbl, dbl, dbl, P, P, P]
        lib.fegen_elements.restype = i32
        _lib_handle = lib
    return _lib_handle


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


@dataclasses.dataclass
class FEProblem:
    """A stiffness matrix in CSR form with its mesh metadata (new numbering)."""
    name: str
    n_rows: int
    rowptr: np.ndarray          # int64 [n_rows+1]
    colind: np.ndarray          # int32 [nnz], ascending within each row
    values: np.ndarray          # float64 [nnz]
    node_xyz: np.ndarray        # float64 [n_nodes, 3], indexed by node number
    dofs_per_node: int
    dirichlet: np.ndarray       # uint8 [n_rows], 1 = constrained (identity row)
    n_elems: int
    grid: tuple                 # node grid dims
    seed: int
    # with elements=True: the element quantities the matrix is the sum of (tet order)
    elem_nodes: np.ndarray = None   # int32 [n_elems, 4], node numbers (new numbering)
    elem_mats: np.ndarray = None    # float64 [n_elems, 4*dpn, 4*dpn], row/col dpn*vertex + comp

    @property
    def nnz(self) -> int:
        return int(self.rowptr[-1])

    @property
    def n_nodes(self) -> int:
        return self.node_xyz.shape[0]


def _assemble(name, kind, dims, periodic2, xyz_grid, rng_perm, coef, d_iso, d_ani, nu,
              dir_grid_mask, seed, dirichlet=True, elements=False):
    n0, n1, n2 = dims
    nn = n0 * n1 * n2
    lib = _lib()
    newid = np.ascontiguousarray(rng_perm.astype(np.int32))
    deg = np.zeros(nn, dtype=np.int32)
    rc = lib.fegen_node_degrees(n0, n1, n2, periodic2, _ptr(newid), _ptr(deg))
    if rc != 0:
        raise RuntimeError(f"fegen_node_degrees failed ({rc})")
    dpn = 3 if kind == 2 else 1
    nnz = int(deg.astype(np.int64).sum()) * dpn * dpn
    n_rows = nn * dpn
    rowptr = np.zeros(n_rows + 1, dtype=np.int64)
    colind = np.zeros(nnz, dtype=np.int32)
    values = np.zeros(nnz, dtype=np.float64)
    bad = np.zeros(1, dtype=np.int64)
    xyz_c = np.ascontiguousarray(xyz_grid, dtype=np.float64)
    coef_c = np.ascontiguousarray(coef if coef is not None else np.zeros(1), dtype=np.float64)
    rc = lib.fegen_assemble(kind, n0, n1, n2, periodic2, _ptr(xyz_c), _ptr(newid), _ptr(coef_c),
                            d_iso, d_ani, nu, _ptr(rowptr), _ptr(colind), _ptr(values), _ptr(bad))
    if rc == -3:
        raise ValueError(f"{name}: tetrahedron {int(bad[0])} is inverted or degenerate "
                         "(jitter too large for this seed)")
    if rc != 0:
        raise RuntimeError(f"fegen_assemble failed ({rc})")
    node_xyz = np.empty((nn, 3), dtype=np.float64)
    node_xyz[newid] = xyz_c
    node_mask = np.zeros(nn, dtype=np.uint8)
    node_mask[newid] = dir_grid_mask.astype(np.uint8)
    row_mask = np.repeat(node_mask, dpn)
    if dirichlet and row_mask.any():
        new_nnz = lib.fegen_dirichlet(n_rows, _ptr(rowptr), _ptr(colind), _ptr(values),
                                      _ptr(row_mask))
        colind = colind[:new_nnz].copy()
        values = values[:new_nnz].copy()
    if not dirichlet:
        row_mask = np.zeros_like(row_mask)
    n_elems = 6 * (n0 - 1) * (n1 - 1) * (n2 if periodic2 else n2 - 1)
    elem_nodes = elem_mats = None
    if elements:
        ne = 4 * dpn
        elem_nodes = np.zeros((n_elems, 4), dtype=np.int32)
        elem_mats = np.zeros((n_elems, ne, ne), dtype=np.float64)
        rc = lib.fegen_elements(kind, n0, n1, n2, periodic2, _ptr(xyz_c), _ptr(newid), _ptr(coef_c),
                                d_iso, d_ani, nu, _ptr(elem_nodes), _ptr(elem_mats), _ptr(bad))
        if rc != 0:
            raise RuntimeError(f"fegen_elements failed ({rc})")
    return FEProblem(name=name, n_rows=n_rows, rowptr=rowptr, colind=colind, values=values,
                     node_xyz=node_xyz, dofs_per_node=dpn, dirichlet=row_mask,
                     n_elems=n_elems, grid=tuple(dims), seed=seed, elem_nodes=elem_nodes,
                     elem_mats=elem_mats)


def _cube_grid(n, rng, jitter):
    """Node coordinates of an n^3 grid on [0,1]^3, interior nodes jittered by
    U[-jitter*h, jitter*h] per coordinate (draw order: jitter then permutation)."""
    h = 1.0 / (n - 1)
    i = np.arange(n, dtype=np.float64)
    X, Y, Z = np.meshgrid(i, i, i, indexing="ij")
    idx = np.stack([X.ravel(), Y.ravel(), Z.ravel()], axis=1)
    jit = rng.uniform(-jitter, jitter, size=idx.shape)
    interior = np.all((idx > 0) & (idx < n - 1), axis=1)
    idx = idx + jit * interior[:, None]
    return idx * h, idx


def cube_laplace(n: int = 20, seed: int = 1501, jitter: float = 0.2, permute: bool = True,
                 dirichlet: bool = True, elements: bool = False) -> FEProblem:
    """P1 Laplace stiffness on the unit cube (n^3 nodes), Dirichlet on z=0."""
    rng = np.random.default_rng(seed)
    xyz, idx = _cube_grid(n, rng, jitter)
    perm = rng.permutation(n ** 3) if permute else np.arange(n ** 3)
    zmask = np.round(idx[:, 2]) == 0
    return _assemble(f"cube_laplace_{n}", 0, (n, n, n), 0, xyz, perm, None, 1.0, 0.0, 0.0,
                     zmask, seed, dirichlet, elements)


def cube_elasticity(n: int = 64, seed: int = 1502, jitter: float = 0.2, nu: float = 0.3,
                    permute: bool = True, dirichlet: bool = True, elements: bool = False) -> FEProblem:
    """P1 linear elasticity (3 dof/node) on the unit cube, clamped on z=0."""
    rng = np.random.default_rng(seed)
    xyz, idx = _cube_grid(n, rng, jitter)
    perm = rng.permutation(n ** 3) if permute else np.arange(n ** 3)
    n_tets = 6 * (n - 1) ** 3
    E = np.exp(rng.uniform(np.log(0.5), np.log(2.0), size=n_tets))
    zmask = np.round(idx[:, 2]) == 0
    return _assemble(f"cube_elasticity_{n}", 2, (n, n, n), 0, xyz, perm, E, 0.0, 0.0, nu,
                     zmask, seed, dirichlet, elements)


# shell geometry (cm): inner and outer semi-axes of the prolate spheroid, theta range
SHELL_A = (4.0, 5.0)     # long semi-axis at r=0 (inner) and r=1 (outer)
SHELL_B = (2.0, 3.0)     # short semi-axis at r=0 and r=1
SHELL_THETA = (0.30 * np.pi, 0.95 * np.pi)   # base .. near-apex (pole excluded)


def _shell_map(r, th, ph):
    a = SHELL_A[0] + (SHELL_A[1] - SHELL_A[0]) * r
    b = SHELL_B[0] + (SHELL_B[1] - SHELL_B[0]) * r
    return np.stack([b * np.sin(th) * np.cos(ph), b * np.sin(th) * np.sin(ph), a * np.cos(th)],
                    axis=-1)


def shell_laplace(nr: int = 24, nt: int = 256, nph: int = 512, seed: int = 1503,
                  jitter: float = 0.15, permute: bool = True, dirichlet: bool = True,
                  d_iso: float = 1.0, d_ani: float = 8.0, elements: bool = False) -> FEProblem:
    """Anisotropic P1 Laplace on a heart-like thick prolate-spheroidal shell."""
    rng = np.random.default_rng(seed)
    ir, it, ip = np.meshgrid(np.arange(nr, dtype=np.float64), np.arange(nt, dtype=np.float64),
                             np.arange(nph, dtype=np.float64), indexing="ij")
    idx = np.stack([ir.ravel(), it.ravel(), ip.ravel()], axis=1)
    jit = rng.uniform(-jitter, jitter, size=idx.shape)
    interior = (idx[:, 0] > 0) & (idx[:, 0] < nr - 1) & (idx[:, 1] > 0) & (idx[:, 1] < nt - 1)
    idx = idx + jit * interior[:, None]
    r = idx[:, 0] / (nr - 1)
    th = SHELL_THETA[0] + (SHELL_THETA[1] - SHELL_THETA[0]) * idx[:, 1] / (nt - 1)
    ph = 2.0 * np.pi * idx[:, 2] / nph
    xyz = _shell_map(r, th, ph)
    perm = rng.permutation(nr * nt * nph) if permute else np.arange(nr * nt * nph)
    # fibre direction per hex cell, from the un-jittered cell centre
    cr, ct, cp = np.meshgrid(np.arange(nr - 1) + 0.5, np.arange(nt - 1) + 0.5,
                             np.arange(nph) + 0.5, indexing="ij")
    rc = (cr / (nr - 1)).ravel()
    thc = (SHELL_THETA[0] + (SHELL_THETA[1] - SHELL_THETA[0]) * ct / (nt - 1)).ravel()
    phc = (2.0 * np.pi * cp / nph).ravel()
    a = SHELL_A[0] + (SHELL_A[1] - SHELL_A[0]) * rc
    b = SHELL_B[0] + (SHELL_B[1] - SHELL_B[0]) * rc
    e_ph = np.stack([-np.sin(phc), np.cos(phc), np.zeros_like(phc)], axis=1)
    e_th = np.stack([b * np.cos(thc) * np.cos(phc), b * np.cos(thc) * np.sin(phc),
                     -a * np.sin(thc)], axis=1)
    e_th /= np.linalg.norm(e_th, axis=1, keepdims=True)
    helix = np.deg2rad(60.0) * (1.0 - 2.0 * rc)
    fib = np.cos(helix)[:, None] * e_ph + np.sin(helix)[:, None] * e_th
    fib /= np.linalg.norm(fib, axis=1, keepdims=True)
    base = np.round(idx[:, 1]) == 0
    return _assemble(f"shell_laplace_{nr}x{nt}x{nph}", 1, (nr, nt, nph), 1, xyz, perm,
                     fib.ravel(), d_iso, d_ani, 0.0, base, seed, dirichlet, elements)


def valid_seed(maker, seed: int, tries: int = 16):
    """maker(seed) for seed, seed + 100003, seed + 2*100003, ... until no tetrahedron
    is inverted by the jitter; returns the problem (its .seed says which draw)."""
    last = None
    for k in range(tries):
        try:
            return maker(seed + 100003 * k)
        except ValueError as e:
            last = e
    raise last


def random_vector(n: int, seed: int, lo: float = -1.0, hi: float = 1.0) -> np.ndarray:
    """x ~ U[lo, hi], float64, from numpy PCG64(seed)."""
    return np.random.default_rng(seed).uniform(lo, hi, size=n)


def manufactured_solution(p: FEProblem) -> np.ndarray:
    """A smooth field u*(x,y,z) on the dofs, zero on constrained rows.

    Scalar problems use sin(pi x) sin(pi y) + z^2 + 0.5; elasticity uses one
    such field per component with different phases.  b = A u* is left to the
    caller (the generator computes no matrix products).
    """
    xyz = p.node_xyz
    s = xyz / max(1e-300, float(np.abs(xyz).max()))
    comps = []
    for c in range(p.dofs_per_node):
        comps.append(np.sin(np.pi * (s[:, 0] + 0.1 * c)) * np.sin(np.pi * (s[:, 1] - 0.2 * c))
                     + s[:, 2] ** 2 + 0.5)
    u = np.stack(comps, axis=1).ravel()
    u[p.dirichlet.astype(bool)] = 0.0
    return u


# Named workloads (node grids and seeds) used by the tests and the benchmark.
WORKLOADS = {
    "cube_laplace_20": lambda: cube_laplace(20, 1501),
    "cube_elasticity_64": lambda: cube_elasticity(64, 1502),
    "shell_laplace_24x256x512": lambda: shell_laplace(24, 256, 512, 1503),
}
