"""The potential decomposition of Eqs. (5)-(10) on the GPU (pf_set_charge_mode) against the oracle's pfo_decompose
and its charge_mode = 1 nonlinear solve: G = phi* + phi^L and the interface right-hand side element by element,
the PF solution with decomposed charges in FP64 and mixed precision, switching back to spread charges, and the
inputs the decomposition refuses."""
import numpy as np
import pytest

from paper_1711_04060_gb300 import workloads as W

pytestmark = pytest.mark.gpu

TOL_FP64 = 1e-8
TOL_MIXED = 1e-6
TOL_CONC = 1e-6
CHARGES = np.array([[0.37, -0.21, 0.29, 1.0], [-2.13, 1.41, -1.07, -0.5]])


@pytest.fixture(scope="module")
def api():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1711_04060_gb300 import build
    build.build()
    from paper_1711_04060_gb300 import api as A
    return A


def _rel(a, b, floor=1e-300):
    return np.abs(a - b).max() / max(np.abs(b).max(), floor)


def _slab(h, charges=CHARGES):
    """A membrane slab |z| < 2.5 A (eps 2) across the box in 0.1 M NaCl at 50 mV, charges inside the slab."""
    n = int(round(16.0 / h)) + 1
    g = W.Grid(n, n, n, h, (-8.0, -8.0, -8.0))
    memb = (np.abs(g.coords()[2]) < 2.5).ravel()
    sp = [W.Species(1, 0.95, 0.1), W.Species(-1, 1.81, 0.1), W.Species(0, 1.4, 55.5)]
    return W.PFProblem(g, np.where(memb, 2.0, 78.5), (~memb).astype(np.uint8), np.asarray(charges, float), 0.0, 0.05,
                       sp, 78.5, 1.2, 298.15, "slab")


def _channel():
    return W.channel_problem(21, box_half=10.0, slab_half=4.0, pores=((0.0, 0.0, 3.0),), n_charges=6, charge_seed=4)


@pytest.mark.parametrize("case", ["slab_h1", "slab_h0.5", "channel"])
def test_decomposition_matches_oracle(api, orc, case):
    prob = {"slab_h1": lambda: _slab(1.0), "slab_h0.5": lambda: _slab(0.5), "channel": _channel}[case]()
    g = prob.grid
    ref = orc.decompose(g.nx, g.ny, g.nz, g.h, g.origin, prob.solvent, prob.charges, 2.0, prob.eps_s,
                        orc.lam(prob.T_K))
    assert ref["status"] == 0
    grid = api.Grid.for_problem(prob)
    rep = grid.set_charge_mode(api.PF_CHARGES_DECOMPOSED)
    G = np.zeros(g.n)
    b = np.zeros(g.n)
    grid.get_decomposition(G, b)
    grid.close()
    assert rep["status"] == 0 and rep["residual"] <= 1e-13
    Tv = orc.thermal_voltage(prob.T_K)
    assert _rel(G / Tv, ref["G"]) < 1e-9
    assert np.all(G[prob.solvent == 1] == 0.0)
    assert _rel(b, ref["bif"]) < 1e-9


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
@pytest.mark.parametrize("case", ["slab", "channel"])
def test_nonlinear_solve_with_decomposed_charges(api, orc, precision, case):
    prob = _slab(1.0) if case == "slab" else _channel()
    g = prob.grid
    ref = orc.pf_solve_problem(prob, tol_outer=1e-11, lin_tol=1e-12, charge_mode=1)
    assert ref["status"] == 0
    grid = api.Grid.for_problem(prob)
    grid.set_charge_mode(api.PF_CHARGES_DECOMPOSED)
    prec = api.PF_FP64 if precision == "fp64" else api.PF_MIXED
    out, rep = grid.nonlinear_solve(api.nl_opts(tol_outer=1e-11, tol=1e-12, precision=prec))
    assert rep["status"] == 0
    assert _rel(out["phi_V"], ref["phi_V"]) < (TOL_FP64 if precision == "fp64" else TOL_MIXED)
    ns = len(prob.species)
    C = out["C_M"].reshape(ns, g.n)
    for i in range(ns):
        assert _rel(C[i], ref["C_M"][i]) < TOL_CONC, i
    sol = prob.solvent == 1
    assert _rel(out["S"][sol], ref["S"][sol], floor=1.0) < TOL_CONC
    # back to spread charges: the plain solve of the oracle
    grid.set_charge_mode(api.PF_CHARGES_SPREAD)
    plain, _ = grid.nonlinear_solve(api.nl_opts(tol_outer=1e-11, tol=1e-12, precision=prec))
    grid.close()
    ref0 = orc.pf_solve_problem(prob, tol_outer=1e-11, lin_tol=1e-12, charge_mode=0)
    assert _rel(plain["phi_V"], ref0["phi_V"]) < (TOL_FP64 if precision == "fp64" else TOL_MIXED)


def test_decomposition_refuses_bad_inputs(api):
    # a charge on a node
    prob = _slab(1.0, charges=[[1.0, 2.0, 0.0, 1.0]])
    grid = api.Grid.for_problem(prob)
    with pytest.raises(api.PFError) as e:
        grid.set_charge_mode(api.PF_CHARGES_DECOMPOSED)
    assert e.value.status == 1
    # two membrane dielectrics
    p2 = _slab(1.0)
    eps = p2.eps.copy()
    eps[np.flatnonzero(p2.solvent == 0)[:5]] = 4.0
    p2 = W.PFProblem(p2.grid, eps, p2.solvent, p2.charges, p2.phi_lo_V, p2.phi_hi_V, p2.species, p2.eps_s, p2.lc_A,
                     p2.T_K, "two_eps")
    grid.set_problem(p2)
    with pytest.raises(api.PFError) as e:
        grid.set_charge_mode(api.PF_CHARGES_DECOMPOSED)
    assert e.value.status == 1
    # the decomposition's outputs need the mode
    with pytest.raises(api.PFError):
        grid.get_decomposition(np.zeros(p2.grid.n))
    grid.close()
