"""One-pass conjugate gradients (pf_solve_opts.method = PF_CG_SYMMETRIC / PF_CG_ALL, the OpCG stencil kernel on the
TMA plane pipeline) against the oracle's pfo_pcg: converged solutions in FP64 and in mixed precision (FP32 inner CG
under FP64 refinement) on cubic and ragged grids, the k-th FP64 iterate, PF1 and PF2, the nonlinear solve with CG
for PF1 against the oracle's solver = 1 solve, the 257^3 PF1 system (edge nodes), and the refused uses."""
import numpy as np
import pytest

from paper_1711_04060_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def api():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1711_04060_gb300 import build
    build.build()
    from paper_1711_04060_gb300 import api as A
    return A


def _rel(a, b):
    return np.abs(a - b).max() / np.abs(b).max()


def _linear_case(n, seed, shape=None):
    if shape is None:
        return W.linear_problem(n=n, seed=seed, n_spheres=6)
    nx, ny, nz = shape
    g = W.Grid(nx, ny, nz, 1.0, (-(nx - 1) / 2, -(ny - 1) / 2, -(nz - 1) / 2))
    eps = W.to_f32_exact(40.0 * np.exp(0.5 * W.normal(W.substream(seed, 1), g.n)))
    b = W.uniform(W.substream(seed, 4), g.n, -1.0, 1.0).reshape(g.shape_zyx)
    b[0] = b[-1] = 0.0
    return W.LinearProblem(g, eps, b.ravel().copy())


def _grid(api, p):
    g = p.grid
    grid = api.Grid(g.nx, g.ny, g.nz, g.h, g.origin)
    grid.set_coeffs(p.eps, np.ones(g.n, np.uint8), np.zeros((0, 4)), 0.0, 0.0, [W.NA, W.CL, W.WATER], 78.5, 1.2)
    return grid


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
@pytest.mark.parametrize("n,shape", [(9, None), (33, None), (0, (45, 11, 20)), (0, (33, 40, 5)), (0, (65, 17, 34))])
def test_poisson_cg_pass_matches_oracle(api, orc, precision, n, shape):
    p = _linear_case(n, seed=31 + n, shape=shape)
    g = p.grid
    A = orc.assemble_eps(g.nx, g.ny, g.nz, g.h, p.eps)
    ref = orc.pcg(g.nx, g.ny, g.nz, A, p.b, tol=1e-13, max_it=20000)
    assert ref["status"] == 0
    grid = _grid(api, p)
    x = np.zeros(g.n)
    prec = api.PF_FP64 if precision == "fp64" else api.PF_MIXED
    rep = grid.linear_solve(api.PF_OP_POISSON, p.b, x,
                            api.solve_opts(tol=1e-13, precision=prec, method=api.PF_CG_SYMMETRIC))
    grid.close()
    assert rep["status"] == 0 and rep["residual"] <= 1e-13
    assert _rel(x, ref["x"]) < (1e-10 if precision == "fp64" else 1e-9)
    if precision == "fp64":  # the single-reduction recurrence takes the same iterations up to rounding
        assert abs(rep["iterations"] - ref["iters"]) <= 0.1 * ref["iters"] + 3, (rep["iterations"], ref["iters"])


@pytest.mark.parametrize("k", [1, 3, 10])
def test_cg_pass_kth_iterate_matches_oracle(api, orc, k):
    """Chronopoulos-Gear and the oracle's two-reduction CG have the same iterates in exact arithmetic."""
    p = _linear_case(33, seed=5)
    g = p.grid
    A = orc.assemble_eps(g.nx, g.ny, g.nz, g.h, p.eps)
    x0 = W.uniform(77, g.n, -0.1, 0.1)
    ref = orc.pcg(g.nx, g.ny, g.nz, A, p.b, x0=x0, tol=1e-30, max_it=k)
    grid = _grid(api, p)
    x = x0.copy()
    rep = grid.linear_solve(api.PF_OP_POISSON, p.b, x,
                            api.solve_opts(tol=1e-30, max_iter=k, method=api.PF_CG_ALL), allow=(3,))
    grid.close()
    assert rep["status"] == 3 and rep["iterations"] == k
    assert _rel(x, ref["x"]) < 1e-10


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_pf1_and_pf2_cg_pass(api, orc, precision):
    prob = W.channel_problem(37, box_half=9.0, slab_half=3.0, pores=((0.5, 0.0, 3.0),), n_charges=0)
    g = prob.grid
    prec = api.PF_FP64 if precision == "fp64" else api.PF_MIXED
    bar = 1e-10 if precision == "fp64" else 1e-9
    grid = api.Grid.for_problem(prob)
    A1 = orc.assemble_pf1(g.nx, g.ny, g.nz, g.h, prob.solvent, prob.eps_s, prob.lc_A)
    b1 = np.where(prob.solvent == 1, W.uniform(21, g.n, -1, 1), 0.0).reshape(g.shape_zyx)
    b1[0] = b1[-1] = 0.0
    b1 = b1.ravel().copy()
    ref = orc.pcg(g.nx, g.ny, g.nz, A1, b1, tol=1e-13)
    x = np.zeros(g.n)
    rep = grid.linear_solve(api.PF_OP_PF1, b1, x, api.solve_opts(tol=1e-13, precision=prec,
                                                                  method=api.PF_CG_SYMMETRIC))
    assert rep["status"] == 0
    assert _rel(x, ref["x"]) < bar
    kappa = W.uniform(22, g.n, 0.0, 2.0)
    grid.set_kappa(kappa)
    A2 = orc.assemble_eps(g.nx, g.ny, g.nz, g.h, prob.eps, kappa * prob.solvent)
    b2 = W.uniform(23, g.n, -1, 1)
    ref = orc.pcg(g.nx, g.ny, g.nz, A2, b2, tol=1e-13)
    x = np.zeros(g.n)
    rep = grid.linear_solve(api.PF_OP_PF2, b2, x, api.solve_opts(tol=1e-13, precision=prec, method=api.PF_CG_ALL))
    assert rep["status"] == 0
    assert _rel(x, ref["x"]) < bar
    # PF_CG_SYMMETRIC leaves PF2 to BiCGSTAB, which reaches the same solution
    y = np.zeros(g.n)
    rep = grid.linear_solve(api.PF_OP_PF2, b2, y, api.solve_opts(tol=1e-13, precision=prec,
                                                                  method=api.PF_CG_SYMMETRIC))
    assert rep["status"] == 0 and _rel(y, ref["x"]) < bar
    grid.close()


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_nonlinear_solve_with_cg_for_pf1(api, orc, precision):
    """The PF fixed point with CG for the Poisson start and PF1 is the oracle's (solver = 1) to the parity bars."""
    prob = W.channel_problem(33)
    g = prob.grid
    ref = orc.pf_solve_problem(prob, tol_outer=1e-11, lin_tol=1e-12, solver=1)
    assert ref["status"] == 0
    grid = api.Grid.for_problem(prob)
    prec = api.PF_FP64 if precision == "fp64" else api.PF_MIXED
    out, rep = grid.nonlinear_solve(api.nl_opts(tol_outer=1e-11, tol=1e-12, precision=prec,
                                                method=api.PF_CG_SYMMETRIC))
    grid.close()
    assert rep["status"] == 0
    assert _rel(out["phi_V"], ref["phi_V"]) < (1e-8 if precision == "fp64" else 1e-6)
    C = out["C_M"].reshape(len(prob.species), g.n)
    for i in range(len(prob.species)):
        assert _rel(C[i], ref["C_M"][i]) < 1e-6, i


def test_pf1_257_cg_pass_edge_nodes(api):
    """The 257^3 PF1 system (tiles with edge nodes): mixed-precision CG converges to the FP64 true residual and
    agrees with BiCGSTAB."""
    prob = W.config2(n=257)
    g = prob.grid
    grid = api.Grid.for_problem(prob)
    b1 = np.where(prob.solvent == 1, W.uniform(41, g.n, -1, 1), 0.0).reshape(g.shape_zyx)
    b1[0] = b1[-1] = 0.0
    b1 = b1.ravel().copy()
    x = np.zeros(g.n)
    rep = grid.linear_solve(api.PF_OP_PF1, b1, x, api.solve_opts(tol=1e-10, precision=api.PF_MIXED,
                                                                  method=api.PF_CG_SYMMETRIC))
    assert rep["status"] == 0 and rep["residual"] <= 1e-10
    y = np.zeros(g.n)
    rep = grid.linear_solve(api.PF_OP_PF1, b1, y, api.solve_opts(tol=1e-10, precision=api.PF_MIXED))
    grid.close()
    assert rep["status"] == 0
    assert _rel(x, y) < 1e-7


def test_cg_pass_refusals(api):
    p = _linear_case(9, seed=3)
    g = p.grid
    grid = _grid(api, p)
    x = np.zeros(g.n)
    with pytest.raises(RuntimeError):  # not a method
        grid.linear_solve(api.PF_OP_POISSON, p.b, x, api.solve_opts(method=3))
    # b = 0 from x = 0: converged before the first iteration
    rep = grid.linear_solve(api.PF_OP_POISSON, np.zeros(g.n), x, api.solve_opts(tol=1e-12, method=api.PF_CG_ALL))
    assert rep["status"] == 0 and rep["iterations"] == 0 and np.all(x == 0)
    # a negative kappa makes the PF2 operator indefinite: reported as a breakdown
    grid.set_kappa(np.full(g.n, -1e6))
    rep = grid.linear_solve(api.PF_OP_PF2, p.b, x, api.solve_opts(tol=1e-12, method=api.PF_CG_ALL), allow=(4,))
    assert rep["status"] == 4
    grid.close()
    # batches solve with BiCGSTAB only
    probs = W.batch_instances(2)
    grids = [api.Grid.for_problem(q) for q in probs]
    batch = api.Batch(grids)
    with pytest.raises(RuntimeError):
        batch.nonlinear_solve(api.nl_opts(tol_outer=1e-2, method=api.PF_CG_SYMMETRIC))
    batch.close()
    for gr in grids:
        gr.close()
