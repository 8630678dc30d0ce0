"""Conjugate gradients through pf_linear_solve_cg (GPU) against the oracle's pfo_pcg: converged solutions, the
k-th iterate, both stop tests with device memory, the three operators on ragged grids, and the error reports."""
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


@pytest.mark.parametrize("n,shape", [(9, None), (33, None), (0, (45, 11, 20)), (0, (33, 40, 5))])
def test_poisson_cg_matches_oracle(api, orc, n, shape):
    p = _linear_case(n, seed=11 + n, shape=shape)
    g = p.grid
    A = orc.assemble_eps(g.nx, g.ny, g.nz, g.h, p.eps)
    ref = orc.pcg(g.nx, g.ny, g.nz, A, p.b, tol=1e-13, max_it=20000)
    assert ref["status"] == 0
    grid = _grid(api, p)
    x = np.zeros(g.n)
    rep = grid.linear_solve(api.PF_OP_POISSON, p.b, x, api.solve_opts(tol=1e-13), method="cg")
    grid.close()
    assert rep["status"] == 0 and rep["residual"] <= 1e-13
    assert _rel(x, ref["x"]) < 1e-10
    assert abs(rep["iterations"] - ref["iters"]) <= 0.1 * ref["iters"] + 3, (rep["iterations"], ref["iters"])


@pytest.mark.parametrize("k", [1, 3, 10])
def test_cg_kth_iterate_matches_oracle(api, orc, k):
    p = _linear_case(33, seed=5)
    g = p.grid
    A = orc.assemble_eps(g.nx, g.ny, g.nz, g.h, p.eps)
    x0 = W.uniform(77, g.n, -0.1, 0.1)
    ref = orc.pcg(g.nx, g.ny, g.nz, A, p.b, x0=x0, tol=1e-30, max_it=k)
    grid = _grid(api, p)
    x = x0.copy()
    rep = grid.linear_solve(api.PF_OP_POISSON, p.b, x, api.solve_opts(tol=1e-30, max_iter=k), allow=(3,),
                            method="cg")
    grid.close()
    assert rep["status"] == 3 and rep["iterations"] == k
    assert _rel(x, ref["x"]) < 1e-11


def test_pf1_and_pf2_cg(api, orc):
    prob = W.channel_problem(37, box_half=9.0, slab_half=3.0, pores=((0.5, 0.0, 3.0),), n_charges=0)
    g = prob.grid
    grid = api.Grid.for_problem(prob)
    A1 = orc.assemble_pf1(g.nx, g.ny, g.nz, g.h, prob.solvent, prob.eps_s, prob.lc_A)
    b1 = np.where(prob.solvent == 1, W.uniform(21, g.n, -1, 1), 0.0).reshape(g.shape_zyx)
    b1[0] = b1[-1] = 0.0
    b1 = b1.ravel().copy()
    ref = orc.pcg(g.nx, g.ny, g.nz, A1, b1, tol=1e-13)
    x = np.zeros(g.n)
    rep = grid.linear_solve(api.PF_OP_PF1, b1, x, api.solve_opts(tol=1e-13), method="cg")
    assert rep["status"] == 0 and abs(rep["iterations"] - ref["iters"]) <= 2
    assert _rel(x, ref["x"]) < 1e-10
    kappa = W.uniform(22, g.n, 0.0, 2.0)
    grid.set_kappa(kappa)
    A2 = orc.assemble_eps(g.nx, g.ny, g.nz, g.h, prob.eps, kappa * prob.solvent)
    b2 = W.uniform(23, g.n, -1, 1)
    ref = orc.pcg(g.nx, g.ny, g.nz, A2, b2, tol=1e-13)
    x = np.zeros(g.n)
    rep = grid.linear_solve(api.PF_OP_PF2, b2, x, api.solve_opts(tol=1e-13), method="cg")
    assert rep["status"] == 0
    assert _rel(x, ref["x"]) < 1e-10
    # the BiCGSTAB path reaches the same solution
    y = np.zeros(g.n)
    grid.linear_solve(api.PF_OP_PF2, b2, y, api.solve_opts(tol=1e-13))
    assert _rel(x, y) < 1e-10
    grid.close()


def test_cg_absinf_stop_and_device_memory(api, orc):
    import torch
    p = _linear_case(33, seed=8)
    g = p.grid
    A = orc.assemble_eps(g.nx, g.ny, g.nz, g.h, p.eps)
    ref = orc.pcg(g.nx, g.ny, g.nz, A, p.b, tol=1e-10, norm_mode=1, max_it=20000)
    grid = _grid(api, p)
    b = torch.from_numpy(p.b).cuda()
    x = torch.zeros(g.n, dtype=torch.float64, device="cuda")
    rep = grid.linear_solve(api.PF_OP_POISSON, b, x, api.solve_opts(tol=1e-10, norm=api.PF_NORM_ABSINF),
                            method="cg")
    torch.cuda.synchronize()
    grid.close()
    assert rep["status"] == 0 and rep["residual"] < 1e-10
    assert abs(rep["iterations"] - ref["iters"]) <= 0.1 * ref["iters"] + 3
    np.testing.assert_allclose(x.cpu().numpy(), ref["x"], atol=1e-8 * np.abs(ref["x"]).max())


def test_cg_reports(api):
    p = _linear_case(9, seed=3)
    g = p.grid
    grid = _grid(api, p)
    x = np.zeros(g.n)
    with pytest.raises(RuntimeError):  # FP64 only
        grid.linear_solve(api.PF_OP_POISSON, p.b, x, api.solve_opts(precision=api.PF_MIXED), method="cg")
    # b = 0 from x = 0: converged before the first iteration
    rep = grid.linear_solve(api.PF_OP_POISSON, np.zeros(g.n), x, api.solve_opts(tol=1e-12), method="cg")
    assert rep["status"] == 0 and rep["iterations"] == 0 and np.all(x == 0)
    # a negative kappa makes the PF2 diagonal negative: not positive definite, reported as a breakdown
    grid.set_kappa(np.full(g.n, -1e6))
    rep = grid.linear_solve(api.PF_OP_PF2, p.b, x, api.solve_opts(tol=1e-12), allow=(4,), method="cg")
    assert rep["status"] == 4
    grid.close()


def test_cg_129_linear_configuration(api):
    """The 129^3 variable-dielectric configuration: CG and BiCGSTAB reach the same solution; the report
    records the iteration counts and device times of both."""
    p = W.linear_problem(n=129, seed=1, n_spheres=32)
    g = p.grid
    grid = _grid(api, p)
    x = np.zeros(g.n)
    rc = grid.linear_solve(api.PF_OP_POISSON, p.b, x, api.solve_opts(tol=1e-12, max_iter=20000), method="cg")
    y = np.zeros(g.n)
    rb = grid.linear_solve(api.PF_OP_POISSON, p.b, y, api.solve_opts(tol=1e-12, max_iter=20000))
    grid.close()
    print(f"\n129^3 CG: {rc['iterations']} it {rc['time_ms']:.1f} ms; BiCGSTAB: {rb['iterations']} it "
          f"{rb['time_ms']:.1f} ms")
    assert rc["status"] == 0 and rb["status"] == 0
    assert _rel(x, y) < 1e-6
