"""Starting vectors of the outer iteration's linear solves (the paper does not fix them), on the oracle alone.

The Table 4 loop is restated here from the oracle's own primitives (Eq. 1 at the nodes, the PF1 and PF2
operators, FP64 BiCGSTAB) and first pinned to `oracle.pf_solve` itself: with the oracle's starts (the previous
iterates) it takes the same outer and BiCGSTAB iterations and reaches the same potential.  With the last solution
extrapolated along its last change -- c from the outer updates' ratio, or from the vector's own last two changes --
it reaches the same fixed point in fewer BiCGSTAB iterations: the start changes the Krylov path only."""
import numpy as np
import pytest

from paper_1711_04060_gb300 import workloads as W


def _problem():
    return W.config2(n=17)


def _table4(orc, prob, start, tol_outer, lin_tol):
    """Table 4 with the PF1 / PF2 starts chosen by `start` ("previous", "ratio" or "own"); returns phi_hat, the
    outer iterations and the BiCGSTAB iterations (the first Poisson solve included)."""
    g = prob.grid
    nx, ny, nz, N = g.nx, g.ny, g.nz, g.n
    plane = nx * ny
    lam, Tv = orc.lam(prob.T_K), orc.thermal_voltage(prob.T_K)
    z = [s.z for s in prob.species]
    sp = orc.species_setup(z, [s.radius_A for s in prob.species], [s.bulk_M for s in prob.species])
    zz = np.array(z, float)
    sol = prob.solvent.astype(bool)
    st, ffix = orc.spread_charges(nx, ny, nz, g.h, g.origin, prob.charges, lam)
    assert st == 0

    def dirichlet(v):
        v[:plane] = prob.phi_lo_V / Tv
        v[N - plane:] = prob.phi_hi_V / Tv

    b = ffix.copy()
    dirichlet(b)
    r = orc.bicgstab(nx, ny, nz, orc.assemble_eps(nx, ny, nz, g.h, prob.eps), b, max_it=20000, tol=lin_tol)
    assert r["status"] == 0
    phi0, its = r["x"], r["iters"]
    A1 = orc.assemble_pf1(nx, ny, nz, g.h, prob.solvent, prob.eps_s, prob.lc_A)
    psi = np.zeros(N)
    hist = {"psi": [], "phi": []}
    deltas = []

    def start_of(key, fallback):
        h = hist[key]
        if start == "previous" or not h:
            return fallback.copy()
        if len(h) == 1:
            return h[-1].copy()
        d1 = h[-1] - h[-2]
        if start == "own" and len(h) >= 3:
            d0 = h[-2] - h[-3]
            den = float(d0 @ d0)
            c = min(max(float(d1 @ d0) / den, 0.0), 1.0) if den > 0 else 0.0
        else:
            c = deltas[-1] / deltas[-2] if len(deltas) >= 2 and deltas[-1] < deltas[-2] else 0.0
        return h[-1] + c * d1

    for outer in range(1, 1000):
        C = orc.fermi_nodes(sp, z, phi0)["C"]
        rho = (zz[:, None] * C).sum(0) * sol
        kap = lam * (zz[:, None] ** 2 * C).sum(0) * sol
        b1 = np.where(sol, -lam * rho, 0.0)
        b1[:plane] = 0.0
        b1[N - plane:] = 0.0
        r = orc.bicgstab(nx, ny, nz, A1, b1, x0=start_of("psi", psi), max_it=20000, tol=lin_tol)
        assert r["status"] == 0
        psi, its = r["x"], its + r["iters"]
        hist["psi"] = (hist["psi"] + [psi])[-3:]
        A2 = orc.assemble_eps(nx, ny, nz, g.h, prob.eps, kap)
        b2 = np.where(sol, -prob.eps_s * psi + kap * phi0, 0.0) + ffix
        dirichlet(b2)
        r = orc.bicgstab(nx, ny, nz, A2, b2, x0=start_of("phi", phi0), max_it=20000, tol=lin_tol)
        assert r["status"] == 0
        phi, its = r["x"], its + r["iters"]
        hist["phi"] = (hist["phi"] + [phi])[-3:]
        new = 0.3 * phi0 + 0.7 * phi
        delta = float(np.abs(new - phi0).max())
        phi0 = new
        deltas.append(delta)
        if delta <= tol_outer:
            return phi0, outer, its
    raise AssertionError("no convergence")


def test_restated_loop_is_the_oracles(orc):
    """With the oracle's starts the restatement takes the oracle's iterations and reaches its potential."""
    prob = _problem()
    ref = orc.pf_solve_problem(prob, tol_outer=1e-6, lin_tol=1e-9)
    assert ref["status"] == 0
    phi, outer, its = _table4(orc, prob, "previous", 1e-6, 1e-9)
    assert outer == ref["report"]["outer_iters"]
    assert its == ref["report"]["lin_iters_total"]
    np.testing.assert_allclose(phi, ref["phi_hat"], rtol=0, atol=1e-12 * np.abs(ref["phi_hat"]).max())


@pytest.mark.parametrize("start", ["ratio", "own"])
def test_extrapolated_starts_same_fixed_point_fewer_iterations(orc, start):
    prob = _problem()
    phi_p, outer_p, its_p = _table4(orc, prob, "previous", 1e-3, 1e-6)
    phi_e, outer_e, its_e = _table4(orc, prob, start, 1e-3, 1e-6)
    assert abs(outer_e - outer_p) <= 1
    assert its_e < its_p, (its_e, its_p)
    # the same fixed point: at a tight tolerance both starts give the oracle's potential
    ref = orc.pf_solve_problem(prob, tol_outer=1e-10, lin_tol=1e-12)
    phi_t, _, _ = _table4(orc, prob, start, 1e-10, 1e-12)
    scale = np.abs(ref["phi_hat"]).max()
    assert np.abs(phi_t - ref["phi_hat"]).max() < 1e-8 * scale
