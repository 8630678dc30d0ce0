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
