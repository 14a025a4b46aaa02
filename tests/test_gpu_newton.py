"""Newton updates on a fixed pattern (fe_newton_step, fe_newton_solve; Sec. 2).

The caller's physics here is a backward-Euler step of a reaction-diffusion
equation of the monodomain form of Sec. 2 with the recovery variable frozen:
  (phi - phi_n) / dt = div(D grad phi) + f(phi),   f(phi) = c phi (phi - a) (1 - phi)
on P1 tetrahedra with one integration point and a lumped mass m_e = V_e / 4 per
element vertex.  Element residual and tangent (computed by the test in numpy,
the caller's side of the boundary):
  R_e = m_e ((phi_e - phi_n,e) / dt - f(phi_e)) + K_e phi_e
  T_e = K_e + diag(m_e (1 / dt - f'(phi_e)))
Every update is checked against the oracle on the same element quantities:
the assembled residual and values bit for bit (oracle_assemble_vector /
_matrix), dx within cond(T) * 2e-10 of the oracle's PCG solution with a true
residual <= 1.01e-10, and phi - dx exact.  The Newton loop must converge
quadratically, and the callback-driven loop must reproduce the update sequence
bit for bit.
"""
import numpy as np
import pytest

import fegen
import oracle

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_1501_00324_gb300 as fs  # noqa: E402

C, A_TH, DT = 8.0, 0.1, 0.05


def volumes(p):
    x = p.node_xyz[p.elem_nodes]                     # (E, 4, 3)
    d = x[:, 1:, :] - x[:, :1, :]
    return np.abs(np.linalg.det(d)) / 6.0


def element_quantities(p, vol, phi, phi_n):
    """(T_e, R_e) of the backward-Euler reaction-diffusion step at phi."""
    pe = phi[p.elem_nodes]                            # (E, 4)
    pn = phi_n[p.elem_nodes]
    m = (vol / 4.0)[:, None]
    f = C * pe * (pe - A_TH) * (1.0 - pe)
    df = C * (-3.0 * pe * pe + 2.0 * (1.0 + A_TH) * pe - A_TH)
    Ke = p.elem_mats
    Re = m * ((pe - pn) / DT - f) + np.einsum("eij,ej->ei", Ke, pe)
    Te = Ke.copy()
    idx = np.arange(4)
    Te[:, idx, idx] += m * (1.0 / DT - df)
    return np.ascontiguousarray(Te), np.ascontiguousarray(Re)


def dense(rowptr, colind, values, n):
    D = np.zeros((n, n))
    for i in range(n):
        D[i, colind[rowptr[i]:rowptr[i + 1]]] = values[rowptr[i]:rowptr[i + 1]]
    return D


def setup(n=12, seed=81):
    p = fegen.cube_laplace(n, seed, elements=True)
    vol = volumes(p)
    phi_n = np.where(p.node_xyz[:, 0] < 0.3, 1.0, 0.0)
    phi_n[p.dirichlet == 1] = 0.0
    A = fs.spmv_create(p.rowptr, p.colind, p.values, p.node_xyz, 1, sigma=256)
    P = fs.assembly_create(A, p.rowptr, p.colind, p.elem_nodes, 1, p.dirichlet)
    return p, vol, phi_n, A, P


def test_newton_steps_match_the_oracle_step_by_step():
    p, vol, phi_n, A, P = setup()
    n = p.n_rows
    phi_d = torch.from_numpy(phi_n.copy()).cuda()
    R_d, dx_d = torch.empty_like(phi_d), torch.zeros_like(phi_d)
    norms = []
    for k in range(6):
        phi = phi_d.cpu().numpy()
        Te, Re = element_quantities(p, vol, phi, phi_n)
        out = fs.fe_newton_step(P, torch.from_numpy(Te).cuda(), torch.from_numpy(Re).cuda(), R_d, dx_d,
                                phi_d, tol=1e-10)
        torch.cuda.synchronize()
        # the residual and the tangent, bit for bit as the oracle assembles them
        Ro = oracle.assemble_vector(n, p.elem_nodes, Re, 1, p.dirichlet)
        assert np.array_equal(R_d.cpu().numpy().view(np.uint64), Ro.view(np.uint64))
        To = oracle.assemble_matrix(p.rowptr, p.colind, p.elem_nodes, Te, 1, p.dirichlet)
        ref = fs.spmv_create(p.rowptr, p.colind, To, p.node_xyz, 1, sigma=256)
        for what in (fs.FESPMV_EXPORT_VALUES, fs.FESPMV_EXPORT_DIAG):
            assert np.array_equal(fs.spmv_export(A, what).view(np.uint8), fs.spmv_export(ref, what).view(np.uint8))
        assert abs(out["res_norm"] - np.linalg.norm(Ro)) <= 1e-12 * np.linalg.norm(Ro)
        norms.append(out["res_norm"])
        if out["res_norm"] <= 1e-12 * norms[0]:   # at the rounding floor of the residual
            break
        assert out["status"] == 0 and out["steps"] == 1, out
        # the update against the oracle's PCG on the same system
        dx = dx_d.cpu().numpy()
        xo, info = oracle.pcg(p.rowptr, p.colind, To, Ro, tol=1e-10)
        assert info["status"] == "converged"
        r = Ro - oracle.csr_spmv(p.rowptr, p.colind, To, dx)
        assert np.linalg.norm(r) <= 1.01e-10 * np.linalg.norm(Ro)
        cond = np.linalg.cond(dense(p.rowptr, p.colind, To, n))
        assert np.linalg.norm(dx - xo) <= cond * 2e-10 * np.linalg.norm(xo)
        assert abs(out["last_cg"]["iters"] - info["iters"]) <= 0.02 * info["iters"] + 2
        assert abs(out["dx_norm"] - np.linalg.norm(dx)) <= 1e-12 * np.linalg.norm(dx)
        assert np.array_equal(phi_d.cpu().numpy().view(np.uint64), (phi - dx).view(np.uint64))
    # Newton converges, and fast: each residual well below the previous one
    assert len(norms) >= 3
    assert all(b < 0.5 * a for a, b in zip(norms, norms[1:]))
    assert norms[-1] <= 1e-9 * norms[0]


def test_newton_loop_with_callback_reproduces_the_steps():
    p, vol, phi_n, A, P = setup(10, 82)
    E = p.n_elems
    Ke_d = torch.empty((E, 4, 4), dtype=torch.float64, device="cuda")
    Re_d = torch.empty((E, 4), dtype=torch.float64, device="cuda")
    calls = []

    def element_fn(phi_t, Ke_t, Re_t):
        Te, Re = element_quantities(p, vol, phi_t.cpu().numpy(), phi_n)
        Ke_t.copy_(torch.from_numpy(Te))
        Re_t.copy_(torch.from_numpy(Re))
        calls.append(1)

    phi_d = torch.from_numpy(phi_n.copy()).cuda()
    R_d, dx_d = torch.empty_like(phi_d), torch.zeros_like(phi_d)
    out = fs.fe_newton_solve(P, phi_d, element_fn, Ke_d, Re_d, R_d, dx_d, newton_tol=1e-10, max_steps=12,
                             tol=1e-11)
    torch.cuda.synchronize()
    assert out["status"] == 0 and 2 <= out["steps"] <= 8, out
    assert len(calls) == out["steps"] + 1
    assert out["res_norm"] <= 1e-10 * out["res_norm0"]
    # the same updates one by one give the same phi, bit for bit
    q_d = torch.from_numpy(phi_n.copy()).cuda()
    R2, dx2 = torch.empty_like(q_d), torch.zeros_like(q_d)
    for _ in range(out["steps"]):
        Te, Re = element_quantities(p, vol, q_d.cpu().numpy(), phi_n)
        fs.fe_newton_step(P, torch.from_numpy(Te).cuda(), torch.from_numpy(Re).cuda(), R2, dx2, q_d, tol=1e-11)
    torch.cuda.synchronize()
    assert torch.equal(phi_d, q_d)
    # the update limit is reported, and a failing callback stops the loop with an error
    phi2 = torch.from_numpy(phi_n.copy()).cuda()
    lim = fs.fe_newton_solve(P, phi2, element_fn, Ke_d, Re_d, R_d, dx_d, newton_tol=0.0, max_steps=1,
                             tol=1e-11)
    assert lim["status"] == fs.FESPMV_ERR_NOT_CONVERGED and lim["steps"] == 1

    def failing(phi_t, Ke_t, Re_t):
        raise RuntimeError("element routine failed")

    with pytest.raises(fs.FespmvError):
        fs.fe_newton_solve(P, phi2, failing, Ke_d, Re_d, R_d, dx_d)
