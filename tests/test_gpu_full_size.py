"""Parity at the bench's full size (257^3 four-pore channel, the launch configuration bench.py times), where the
oracle cannot run the whole solve: (1) the pointwise step of Eq. (1) at sampled solvent nodes, recomputed by the
oracle from the GPU's final potential, equals the GPU's concentrations, steric potential and void fraction;
(2) a GPU linear solve with the full-size operator leaves the residual that the oracle's own assembled operator
measures within the requested tolerance."""
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


@pytest.fixture(scope="module")
def prob():
    return W.config2(257)


def test_fermi_at_sampled_nodes_of_the_full_solve(api, orc, prob):
    g = prob.grid
    grid = api.Grid.for_problem(prob)
    out, rep = grid.nonlinear_solve(api.nl_opts(tol_outer=1e-3, tol=1e-6, precision=api.PF_MIXED))
    grid.close()
    assert rep["status"] == 0
    z = [s.z for s in prob.species]
    sp = orc.species_setup(z, [s.radius_A for s in prob.species], [s.bulk_M for s in prob.species])
    Tv = orc.thermal_voltage(prob.T_K)
    molar = orc.molar_to_per_A3()
    ns = len(z)
    C = out["C_M"].reshape(ns, g.n)
    sol = np.flatnonzero(prob.solvent)
    pick = sol[np.linspace(0, len(sol) - 1, 3000).astype(np.int64)]
    worst = 0.0
    for node in pick:
        ref = orc.fermi_point(sp, z, out["phi_V"][node] / Tv)
        assert ref["status"] == 0
        for i in range(ns):
            cr = ref["C"][i] / molar
            if cr > 0:
                worst = max(worst, abs(C[i, node] - cr) / cr)
        assert abs(out["S"][node] - ref["S"]) < 1e-9
        assert abs(out["Gamma"][node] - ref["Gamma"]) <= 1e-9 * ref["Gamma"]
    assert worst < 1e-9, worst


def test_full_size_linear_solve_against_the_oracle_operator(api, orc, prob):
    g = prob.grid
    A = orc.assemble_eps(g.nx, g.ny, g.nz, g.h, prob.eps)
    b = W.uniform(W.substream(257, 9), g.n, -1.0, 1.0).reshape(g.shape_zyx)
    b[0] = b[-1] = 0.0
    b = b.ravel().copy()
    grid = api.Grid.for_problem(prob)
    x = np.zeros(g.n)
    rep = grid.linear_solve(api.PF_OP_POISSON, b, x, api.solve_opts(tol=1e-9, precision=api.PF_MIXED))
    grid.close()
    assert rep["status"] == 0
    r = b - orc.dia_apply(g.nx, g.ny, g.nz, A, x)
    assert np.linalg.norm(r) <= 2e-9 * np.linalg.norm(b)


@pytest.mark.parametrize("precision,tol", [("fp64", 1e-10), ("mixed", 1e-6)])
def test_config_129_linear_solver(api, orc, precision, tol):
    """The 129^3 lognormal-dielectric linear system with sphere inclusions (2 / 78.5): the GPU solve in each
    precision leaves the residual the oracle's operator measures within the stated tolerance, and (FP64) agrees
    with the oracle's own BiCGSTAB solution as far as the conditioning lets a 1e-10 residual fix the solution."""
    p = W.linear_problem(n=129, seed=1, n_spheres=32)
    g = p.grid
    A = orc.assemble_eps(g.nx, g.ny, g.nz, g.h, p.eps)
    grid = api.Grid(g.nx, g.ny, g.nz, g.h, g.origin)
    grid.set_coeffs(p.eps, np.ones(g.n, np.uint8), np.zeros((0, 4)), 0.0, 0.0, [W.NA, W.CL, W.WATER], 78.5, 1.2)
    x = np.zeros(g.n)
    prec = api.PF_FP64 if precision == "fp64" else api.PF_MIXED
    rep = grid.linear_solve(api.PF_OP_POISSON, p.b, x, api.solve_opts(tol=tol, precision=prec))
    grid.close()
    assert rep["status"] == 0
    r = p.b - orc.dia_apply(g.nx, g.ny, g.nz, A, x)
    assert np.linalg.norm(r) <= 1.5 * tol * np.linalg.norm(p.b)
    if precision == "fp64":
        ref = orc.bicgstab(g.nx, g.ny, g.nz, A, p.b, tol=1e-10, max_it=20000)
        assert ref["status"] == 0
        assert np.abs(x - ref["x"]).max() <= 1e-4 * np.abs(ref["x"]).max()


def test_zero_right_hand_side(api):
    """b = 0 gives x = 0 at once (the degenerate start), in both precisions."""
    p = W.linear_problem(n=17, seed=4, n_spheres=2)
    g = p.grid
    grid = api.Grid(g.nx, g.ny, g.nz, g.h, g.origin)
    grid.set_coeffs(p.eps, np.ones(g.n, np.uint8), np.zeros((0, 4)), 0.0, 0.0, [W.NA, W.CL, W.WATER], 78.5, 1.2)
    for prec in (api.PF_FP64, api.PF_MIXED):
        x = np.full(g.n, 0.0)
        rep = grid.linear_solve(api.PF_OP_POISSON, np.zeros(g.n), x, api.solve_opts(tol=1e-10, precision=prec))
        assert rep["status"] == 0 and rep["iterations"] == 0
        assert not x.any()
    grid.close()
