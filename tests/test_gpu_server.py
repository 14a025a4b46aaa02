"""The solve server (continuous batching) through the C ABI.

Each result in the mix must equal, bit for bit, the result of cg_solve on the
same handle alone (the server runs the same kernels, grids and fixed-order
reductions on its own workspace), and must meet its tolerance on the true
residual recomputed by the oracle.
"""
import time

import numpy as np
import pytest

import fegen
import oracle

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_1501_00324_gb300 as fs  # noqa: E402


def problems():
    return [fegen.cube_laplace(12, 81), fegen.cube_elasticity(8, 82), fegen.shell_laplace(5, 16, 24, 83),
            fegen.cube_laplace(16, 84)]


def alone(A, b, **kw):
    bd = torch.from_numpy(b).cuda()
    xd = torch.zeros_like(bd)
    res = fs.cg_solve(A, bd, xd, **kw)
    torch.cuda.synchronize()
    return xd.cpu().numpy(), res


def test_results_in_the_mix_equal_results_alone():
    ps = problems()
    mats = [fs.spmv_create(p.rowptr, p.colind, p.values, p.node_xyz, p.dofs_per_node, sigma=256,
                           precisions=fs.FESPMV_PREC_F32) for p in ps]
    S = fs.srv_create(1 << 30, 6)
    ids = [fs.srv_register(S, A) for A in mats]
    rng = np.random.default_rng(85)
    reqs = []
    for k in range(24):
        m = int(rng.integers(len(ps)))
        b = fegen.random_vector(ps[m].n_rows, 1000 + k)
        tol = [1e-8, 1e-10][k % 2]
        # FP64, restarted FP32 refinement, FP32 with reliable updates, single-reduction FP64
        prec, fl = [(fs.FESPMV_CG_F64, 0), (fs.FESPMV_CG_F32_REFINE, 0),
                    (fs.FESPMV_CG_F32_REFINE, fs.FESPMV_CG_RELIABLE),
                    (fs.FESPMV_CG_F64, fs.FESPMV_CG_SINGLE_REDUCTION)][(k // 2) % 4]
        reqs.append((m, b, tol, prec, fl))
    tickets = [fs.srv_submit(S, ids[m], b, tol=tol, precision=prec, flags=fl) for (m, b, tol, prec, fl) in reqs]
    results = [fs.srv_poll(S, t, ps[m].n_rows) for t, (m, *_rest) in zip(tickets, reqs)]
    st = fs.srv_get_stats(S)
    assert st["completed"] == 24 and st["peak_active"] > 1
    for (m, b, tol, prec, fl), (rc, x, res, tm) in zip(reqs, results):
        assert rc == 0, res
        p = ps[m]
        r = b - oracle.csr_spmv(p.rowptr, p.colind, p.values, x)
        assert np.linalg.norm(r) <= tol * 1.01 * np.linalg.norm(b)
        xa, ra = alone(mats[m], b, tol=tol, precision=prec, flags=fl)
        assert np.array_equal(x.view(np.uint64), xa.view(np.uint64))
        assert res["iters"] == ra["iters"] and res["outer"] == ra["outer"]
        assert tm["t_total_s"] >= tm["t_solve_s"] > 0
    fs.srv_destroy(S)


def test_budget_admission_and_late_arrivals():
    ps = problems()[:2]
    mats = [fs.spmv_create(p.rowptr, p.colind, p.values, p.node_xyz, p.dofs_per_node, sigma=256)
            for p in ps]
    # a budget that holds one workspace of the larger matrix, and a few small ones
    n_big = max(p.n_rows for p in ps)
    budget = 80 * n_big + (1 << 20)
    S = fs.srv_create(budget, 8)
    ids = [fs.srv_register(S, A) for A in mats]
    tickets = []
    for k in range(6):
        m = k % 2
        tickets.append((m, fs.srv_submit(S, ids[m], fegen.random_vector(ps[m].n_rows, 2000 + k))))
    time.sleep(0.01)
    for k in range(6, 12):                 # arrive while the first wave runs
        m = k % 2
        tickets.append((m, fs.srv_submit(S, ids[m], fegen.random_vector(ps[m].n_rows, 2000 + k))))
    for m, t in tickets:
        rc, x, res, tm = fs.srv_poll(S, t, ps[m].n_rows)
        assert rc == 0
    st = fs.srv_get_stats(S)
    assert st["completed"] == 12 and st["peak_workspace_bytes"] <= budget
    fs.srv_destroy(S)


def test_errors_are_per_request():
    p = fegen.cube_laplace(10, 86)
    A = fs.spmv_create(p.rowptr, p.colind, p.values, p.node_xyz, 1, sigma=128)
    bad = fs.spmv_create(np.array([0, 1, 2]), np.array([0, 1]), np.array([1.0, -1.0]),
                         format=fs.FESPMV_FMT_CSR)
    S = fs.srv_create(1 << 28, 4)
    ia, ib = fs.srv_register(S, A), fs.srv_register(S, bad)
    with pytest.raises(fs.FespmvError):
        fs.srv_submit(S, 99, np.zeros(3))
    with pytest.raises(fs.FespmvError):
        fs.srv_submit(S, ia, np.zeros(p.n_rows), flags=fs.FESPMV_CG_X0)
    with pytest.raises(fs.FespmvError):       # the handle holds no FP32 copy
        fs.srv_submit(S, ia, np.zeros(p.n_rows), precision=fs.FESPMV_CG_F32_REFINE)
    t1 = fs.srv_submit(S, ib, np.array([1.0, 1.0]))
    t2 = fs.srv_submit(S, ia, fegen.random_vector(p.n_rows, 3))
    assert fs.srv_poll(S, t1, 2)[0] == fs.FESPMV_ERR_BREAKDOWN
    rc, x, res, tm = fs.srv_poll(S, t2, p.n_rows)
    assert rc == 0
    t3 = fs.srv_submit(S, ia, fegen.random_vector(p.n_rows, 4), tol=1e-12, max_iter=3,
                       max_restarts=-1)
    assert fs.srv_poll(S, t3, p.n_rows)[0] == fs.FESPMV_ERR_NOT_CONVERGED
    with pytest.raises(fs.FespmvError):       # a collected ticket is gone
        fs.srv_poll(S, t3, p.n_rows)
    fs.srv_destroy(S)


def test_cancel_queued():
    p = fegen.cube_laplace(16, 87)
    A = fs.spmv_create(p.rowptr, p.colind, p.values, p.node_xyz, 1, sigma=256)
    S = fs.srv_create(1 << 28, 1)                   # one slot: the rest wait in the queue
    mid = fs.srv_register(S, A)
    tickets = [fs.srv_submit(S, mid, fegen.random_vector(p.n_rows, 50 + k)) for k in range(20)]
    n = fs.srv_cancel_queued(S)
    assert 1 <= n <= 19
    codes = [fs.srv_poll(S, t, p.n_rows)[0] for t in tickets]
    assert codes.count(fs.FESPMV_ERR_CANCELLED) == n and codes.count(0) == 20 - n
    fs.srv_destroy(S)


def multi_alone(A, b, width, **kw):
    """cg_solve_multi of b alone with `width` columns (the others zero)."""
    B = np.zeros((len(b), width))
    B[:, 0] = b
    Bd = torch.from_numpy(B).cuda()
    Xd = torch.zeros_like(Bd)
    rc, res = fs.cg_solve_multi(A, Bd, Xd, **kw)
    torch.cuda.synchronize()
    return Xd.cpu().numpy()[:, 0].copy(), res[0]


def same(x, res, xa, ra):
    return (np.array_equal(x.view(np.uint64), xa.view(np.uint64)) and res["iters"] == ra["iters"]
            and res["outer"] == ra["outer"])


@pytest.mark.parametrize("width", [8, -1])
def test_grouped_results_equal_the_lockstep_solve_alone(width):
    """With grouping on, requests on one matrix share lockstep groups; each result
    equals (bit for bit) cg_solve_multi of that right-hand side alone with the
    group's width, or cg_solve alone when it took the single path (a lone request,
    or the single-reduction flag, which groups do not take)."""
    ps = problems()
    mats = [fs.spmv_create(p.rowptr, p.colind, p.values, p.node_xyz, p.dofs_per_node, sigma=256,
                           precisions=fs.FESPMV_PREC_F32) for p in ps]
    S = fs.srv_create(1 << 30, 6)
    fs.srv_set_grouping(S, width)
    ids = [fs.srv_register(S, A) for A in mats]
    rng = np.random.default_rng(91)
    reqs = []
    for k in range(40):
        m = int(rng.integers(len(ps)))
        b = fegen.random_vector(ps[m].n_rows, 3000 + k)
        tol = [1e-8, 1e-10][k % 2]
        single = k % 5 == 4
        prec, fl = ((fs.FESPMV_CG_F64, fs.FESPMV_CG_SINGLE_REDUCTION) if single else
                    (fs.FESPMV_CG_F32_REFINE, fs.FESPMV_CG_RELIABLE))
        reqs.append((m, b, tol, prec, fl, single))
    tickets = [fs.srv_submit(S, ids[m], b, tol=tol, precision=prec, flags=fl)
               for (m, b, tol, prec, fl, _) in reqs]
    results = [fs.srv_poll(S, t, ps[r[0]].n_rows) for t, r in zip(tickets, reqs)]
    st = fs.srv_get_stats(S)
    assert st["completed"] == 40 and st["grouped"] >= 8
    n_grouped = 0
    for (m, b, tol, prec, fl, single), (rc, x, res, tm) in zip(reqs, results):
        assert rc == 0, res
        p = ps[m]
        r = b - oracle.csr_spmv(p.rowptr, p.colind, p.values, x)
        assert np.linalg.norm(r) <= tol * 1.01 * np.linalg.norm(b)
        xa, ra = alone(mats[m], b, tol=tol, precision=prec, flags=fl)
        if single:
            assert same(x, res, xa, ra)
            continue
        kw = width if width > 0 else 32          # these matrices are small: 32 columns
        xm, rm = multi_alone(mats[m], b, kw, tol=tol, precision=prec, flags=fl)
        assert same(x, res, xm, rm) or same(x, res, xa, ra)
        n_grouped += same(x, res, xm, rm)
    assert n_grouped == st["grouped"]
    fs.srv_destroy(S)


@pytest.mark.parametrize("precision,flags", [(fs.FESPMV_CG_F64, 0), (fs.FESPMV_CG_F32_REFINE, 0),
                                             (fs.FESPMV_CG_F32_REFINE, fs.FESPMV_CG_RELIABLE)])
def test_late_arrivals_join_running_groups(precision, flags):
    """Requests that arrive while a group runs take the columns that finished
    solves free, at the group's outer steps (every 8 * check_every = 32 inner
    iterations here): more requests than columns, results as alone."""
    p = fegen.cube_elasticity(9, 92)
    A = fs.spmv_create(p.rowptr, p.colind, p.values, p.node_xyz, 3, sigma=256, precisions=fs.FESPMV_PREC_F32)
    S = fs.srv_create(1 << 30, 4)
    fs.srv_set_grouping(S, 4)
    mid = fs.srv_register(S, A)
    bs = [fegen.random_vector(p.n_rows, 4000 + k) for k in range(14)]
    tols = [[1e-8, 1e-10, 1e-6][k % 3] for k in range(14)]
    kw = dict(precision=precision, flags=flags, check_every=4)
    tickets = [fs.srv_submit(S, mid, bs[k], tol=tols[k], **kw) for k in range(7)]
    time.sleep(0.005)
    tickets += [fs.srv_submit(S, mid, bs[k], tol=tols[k], **kw) for k in range(7, 14)]
    n_grouped = 0
    for k, t in enumerate(tickets):
        rc, x, res, tm = fs.srv_poll(S, t, p.n_rows)
        assert rc == 0, res
        xm, rm = multi_alone(A, bs[k], 4, tol=tols[k], **kw)
        xa, ra = alone(A, bs[k], tol=tols[k], **kw)
        assert same(x, res, xm, rm) or same(x, res, xa, ra), k
        n_grouped += same(x, res, xm, rm)
    st = fs.srv_get_stats(S)
    assert st["completed"] == 14 and n_grouped == st["grouped"] >= 8   # more than one group's worth
    fs.srv_destroy(S)


def test_grouping_falls_back_to_the_single_path():
    """A budget too small for a group, and a width of 0 again: the requests take the
    single path and equal cg_solve alone; a bad width is rejected."""
    p = fegen.cube_laplace(12, 93)
    A = fs.spmv_create(p.rowptr, p.colind, p.values, p.node_xyz, 1, sigma=256)
    S = fs.srv_create(80 * p.n_rows + (1 << 20), 4)   # room for one single workspace only
    with pytest.raises(fs.FespmvError):
        fs.srv_set_grouping(S, 12)
    fs.srv_set_grouping(S, 32)
    mid = fs.srv_register(S, A)
    bs = [fegen.random_vector(p.n_rows, 5000 + k) for k in range(5)]
    tickets = [fs.srv_submit(S, mid, b) for b in bs]
    for b, t in zip(bs, tickets):
        rc, x, res, tm = fs.srv_poll(S, t, p.n_rows)
        assert rc == 0
        xa, ra = alone(A, b)
        assert np.array_equal(x.view(np.uint64), xa.view(np.uint64))
    fs.srv_destroy(S)


def test_grouped_cancel_and_errors_are_per_request():
    """With grouping on: cancelling the queue leaves the requests already in groups
    to finish; a matrix whose diagonal is not positive fails its requests (the
    group cannot be built), the others are served."""
    p = fegen.cube_laplace(14, 94)
    A = fs.spmv_create(p.rowptr, p.colind, p.values, p.node_xyz, 1, sigma=256, precisions=fs.FESPMV_PREC_F32)
    vals = p.values.copy()
    rows = np.repeat(np.arange(p.n_rows), np.diff(p.rowptr))
    vals[(rows == 5) & (p.colind == 5)] = -2.0
    Bad = fs.spmv_create(p.rowptr, p.colind, vals, p.node_xyz, 1, sigma=256)
    S = fs.srv_create(1 << 30, 2)
    fs.srv_set_grouping(S, 4)
    ia, ib = fs.srv_register(S, A), fs.srv_register(S, Bad)
    bad_tickets = [fs.srv_submit(S, ib, fegen.random_vector(p.n_rows, 6000 + k)) for k in range(3)]
    tickets = [fs.srv_submit(S, ia, fegen.random_vector(p.n_rows, 6100 + k), precision=fs.FESPMV_CG_F32_REFINE,
                             flags=fs.FESPMV_CG_RELIABLE) for k in range(40)]
    n = fs.srv_cancel_queued(S)
    codes = [fs.srv_poll(S, t, p.n_rows)[0] for t in tickets]
    assert codes.count(fs.FESPMV_ERR_CANCELLED) == n and codes.count(0) == 40 - n
    assert all(fs.srv_poll(S, t, p.n_rows)[0] in (fs.FESPMV_ERR_BREAKDOWN, fs.FESPMV_ERR_CANCELLED)
               for t in bad_tickets)
    # the server keeps serving after the cancellation and the failures
    t = fs.srv_submit(S, ia, fegen.random_vector(p.n_rows, 6200))
    assert fs.srv_poll(S, t, p.n_rows)[0] == 0
    fs.srv_destroy(S)


@pytest.mark.parametrize("width", [0, -1])
def test_tiny_problems_in_the_mix(width):
    """Matrices of 1, 2 and 33 rows and the smallest elasticity mesh served together
    (without and with lockstep groups): every result meets its tolerance on the true
    residual and equals the solve alone bit for bit (cg_solve, or cg_solve_multi of
    the right-hand side alone at the group's width when it was grouped)."""
    from test_gpu_cg import tridiagonal_problem
    ps = [tridiagonal_problem(1), tridiagonal_problem(2), tridiagonal_problem(33), fegen.cube_elasticity(2, 88)]
    mats = [fs.spmv_create(p.rowptr, p.colind, p.values, p.node_xyz, p.dofs_per_node, sigma=256,
                           precisions=fs.FESPMV_PREC_F32) for p in ps]
    S = fs.srv_create(1 << 28, 4)
    if width:
        fs.srv_set_grouping(S, width)
    ids = [fs.srv_register(S, A) for A in mats]
    reqs = []
    for k in range(12):
        m = k % len(ps)
        prec, fl = [(fs.FESPMV_CG_F64, 0), (fs.FESPMV_CG_F32_REFINE, fs.FESPMV_CG_RELIABLE)][(k // 4) % 2]
        reqs.append((m, fegen.random_vector(ps[m].n_rows, 1100 + k), [1e-8, 1e-10][k % 2], prec, fl))
    tickets = [fs.srv_submit(S, ids[m], b, tol=tol, precision=prec, flags=fl) for (m, b, tol, prec, fl) in reqs]
    results = [fs.srv_poll(S, t, ps[m].n_rows) for t, (m, *_rest) in zip(tickets, reqs)]
    assert fs.srv_get_stats(S)["completed"] == 12
    for (m, b, tol, prec, fl), (rc, x, res, tm) in zip(reqs, results):
        assert rc == 0, res
        p = ps[m]
        r = b - oracle.csr_spmv(p.rowptr, p.colind, p.values, x)
        assert np.linalg.norm(r) <= tol * 1.01 * np.linalg.norm(b)
        xa, ra = alone(mats[m], b, tol=tol, precision=prec, flags=fl)
        if width:                                 # these matrices are small: groups of 32
            xm, rm = multi_alone(mats[m], b, 32, tol=tol, precision=prec, flags=fl)
            assert same(x, res, xm, rm) or same(x, res, xa, ra), (m, res)
        else:
            assert same(x, res, xa, ra), (m, res, ra)
    fs.srv_destroy(S)
