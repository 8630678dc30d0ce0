"""Filter region (pf_set_filter, GPU) against the oracle's pfo_pf_solve_fixed: synthetic binding sites in the pore hold
their Eq. (19) potentials as Dirichlet values of the continuum model; a region held at the free solution's own
potential changes nothing elsewhere (l_c = 0); clearing restores the plain solve; batches refuse such a grid."""
import numpy as np
import pytest

from paper_1711_04060_gb300 import workloads as W

pytestmark = pytest.mark.gpu

TOL_FP64 = 1e-8
TOL_MIXED = 1e-6
TOL_CONC = 1e-6


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


def _channel(lc):
    sp = [W.Species(1, 0.95, 0.1), W.Species(-1, 1.81, 0.1), W.Species(0, 1.4, 55.5)]
    return W.channel_problem(17, box_half=8.0, slab_half=3.0, pores=((0.0, 0.0, 3.0),), n_charges=4, charge_seed=9,
                             phi_hi_V=0.05, species=sp, lc_A=lc)


def _ball(g, centre, radius):
    X, Y, Z = g.coords()
    return ((X - centre[0]) ** 2 + (Y - centre[1]) ** 2 + (Z - centre[2]) ** 2 <= radius ** 2).ravel()


def _sites(orc, prob):
    """Three sites in the pore (two occupied), their Eq. (19) potentials from the wall charges, mapped to the nodes
    of their spheres (at least the nearest node)."""
    g = prob.grid
    centres = np.array([[0.3, -0.2, -1.5], [-0.4, 0.3, 0.6], [0.2, 0.1, 2.4]])
    radii, q_ion, occ = [0.95, 0.99, 0.95], [1.0, 2.0, 1.0], [1, 0, 1]
    st, phib = orc.site_potentials(centres, radii, q_ion, occ, 80.0, prob.charges, 20.0, orc.lam())
    assert st == 0
    Tv = orc.thermal_voltage(prob.T_K)
    fixed = np.zeros(g.n, bool)
    val = np.zeros(g.n)
    for c, r, p in zip(centres, radii, phib):
        ball = _ball(g, c, max(r, 0.87 * g.h))
        fixed |= ball
        val[ball] = p * Tv
    assert fixed.sum() >= 3 and np.all(prob.solvent[fixed] == 1)
    return fixed.astype(np.uint8), val


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_filter_region_matches_oracle(api, orc, precision):
    prob = _channel(1.2)
    g = prob.grid
    fixed, val = _sites(orc, prob)
    ref = orc.pf_solve_problem(prob, tol_outer=1e-11, lin_tol=1e-12, fixed=fixed, fixed_phi_V=val)
    assert ref["status"] == 0
    grid = api.Grid.for_problem(prob)
    grid.set_filter(fixed, val)
    prec = api.PF_FP64 if precision == "fp64" else api.PF_MIXED
    out, rep = grid.nonlinear_solve(api.nl_opts(tol_outer=1e-11, tol=1e-12, precision=prec, max_outer=2000))
    grid.close()
    assert rep["status"] == 0
    assert _rel(out["phi_V"], ref["phi_V"], floor=0.0257) < (TOL_FP64 if precision == "fp64" else TOL_MIXED)
    f = fixed == 1
    np.testing.assert_allclose(out["phi_V"][f], val[f], rtol=1e-14)
    assert np.all(out["Psi"][f] == 0.0)
    ns = len(prob.species)
    C = out["C_M"].reshape(ns, g.n)
    for i in range(ns):
        assert np.all(C[i][f] == 0.0)
        assert _rel(C[i], ref["C_M"][i]) < TOL_CONC


def test_filter_region_holding_the_solution_changes_nothing(api):
    """l_c = 0: fixing pore nodes at the potential the free solve found there leaves the rest unchanged."""
    prob = _channel(0.0)
    g = prob.grid
    opts = api.nl_opts(tol_outer=1e-12, tol=1e-13)
    grid = api.Grid.for_problem(prob)
    free, _ = grid.nonlinear_solve(opts)
    fixed = (_ball(g, (0.0, 0.0, 0.5), 1.6) & (prob.solvent == 1)).astype(np.uint8)
    grid.set_filter(fixed, np.where(fixed == 1, free["phi_V"], 0.0))
    held, rep = grid.nonlinear_solve(opts)
    assert rep["status"] == 0
    assert _rel(held["phi_V"], free["phi_V"]) < 1e-9
    # clearing the region gives the plain solve back
    grid.set_filter(None)
    again, _ = grid.nonlinear_solve(opts)
    grid.close()
    assert _rel(again["phi_V"], free["phi_V"]) < 1e-11


def test_filter_region_cleared_by_new_coefficients_and_refused_in_batches(api, orc):
    prob = _channel(1.2)
    fixed, val = _sites(orc, prob)
    grid = api.Grid.for_problem(prob)
    grid.set_filter(fixed, val)
    batch = api.Batch([grid], tiles_per_block=2)
    with pytest.raises(RuntimeError):
        batch.nonlinear_solve(api.nl_opts(tol_outer=1e-6, tol=1e-9))
    batch.close()
    grid.set_problem(prob)  # pf_set_coeffs clears the region
    out, _ = grid.nonlinear_solve(api.nl_opts(tol_outer=1e-9, tol=1e-11))
    plain = api.Grid.for_problem(prob)
    ref, _ = plain.nonlinear_solve(api.nl_opts(tol_outer=1e-9, tol=1e-11))
    plain.close()
    grid.close()
    assert _rel(out["phi_V"], ref["phi_V"]) < 1e-13


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_site_model_on_the_device_matches_oracle(api, orc, precision):
    """pf_set_filter_sites: the site potentials of Eq. (19) and the site steric potential of Eq. (20) computed
    on the device against the oracle's pfo_site_potentials / pfo_site_steric, and the nonlinear solve with the
    region they define against the oracle's fixed-region solve."""
    prob = _channel(1.2)
    g = prob.grid
    centres = np.array([[0.3, -0.2, -1.5], [-0.4, 0.3, 0.6], [0.2, 0.1, 2.4]])
    radii, q_ion, occ, ion_r = [0.95, 0.99, 0.95], [1.0, 2.0, 1.0], [1, 0, 1], [0.95, 0.99, 0.95]
    st, phib = orc.site_potentials(centres, radii, q_ion, occ, 80.0, prob.charges, 20.0, orc.lam())
    assert st == 0
    Tv = orc.thermal_voltage(prob.T_K)
    grid = api.Grid.for_problem(prob)
    phi_sites, S = grid.set_filter_sites(centres, radii, q_ion, occ, ion_r, 80.0, 20.0, map_radius_A=0.87 * g.h,
                                         v_sites_A3=20.0)
    np.testing.assert_allclose(phi_sites, phib * Tv, rtol=1e-12)
    gB = orc.species_setup([1, -1, 0], [0.95, 1.81, 1.4], [0.1, 0.1, 55.5])["gammaB"]
    assert S == pytest.approx(orc.site_steric(ion_r, occ, 20.0, gB)[1], rel=1e-13)
    fixed, val = _sites(orc, prob)
    ref = orc.pf_solve_problem(prob, tol_outer=1e-11, lin_tol=1e-12, fixed=fixed, fixed_phi_V=val)
    assert ref["status"] == 0
    prec = api.PF_FP64 if precision == "fp64" else api.PF_MIXED
    out, rep = grid.nonlinear_solve(api.nl_opts(tol_outer=1e-11, tol=1e-12, precision=prec, max_outer=2000))
    assert rep["status"] == 0
    assert _rel(out["phi_V"], ref["phi_V"], floor=0.0257) < (TOL_FP64 if precision == "fp64" else TOL_MIXED)
    f = fixed == 1
    np.testing.assert_allclose(out["phi_V"][f], val[f], rtol=1e-12)
    assert np.all(out["Psi"][f] == 0.0)
    # a six-point position on another occupied site's centre, or ions that fill the site volume, are refused and
    # leave the region as it was
    with pytest.raises(api.PFError):
        grid.set_filter_sites([[0.0, 0.0, 0.0], [0.5, 0.0, 0.0]], [0.5, 0.5], [1.0, 1.0], [1, 1], [0.5, 0.5], 80.0,
                              20.0, v_sites_A3=20.0)
    with pytest.raises(api.PFError):
        grid.set_filter_sites(centres, radii, q_ion, [1, 1, 1], ion_r, 80.0, 20.0, v_sites_A3=5.0)
    again, _ = grid.nonlinear_solve(api.nl_opts(tol_outer=1e-11, tol=1e-12, precision=prec, max_outer=2000))
    grid.close()
    assert _rel(again["phi_V"], out["phi_V"], floor=0.0257) < (TOL_FP64 if precision == "fp64" else TOL_MIXED)
