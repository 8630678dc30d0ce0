"""Pins of the FP64 CPU oracle against what the paper and the mathematics fix.

Each test ties one oracle function to something other than itself: values printed in the
paper (Table 1), textbook values, closed-form solutions, invariants the paper states
(saturation, the bath state, the reduction to Poisson-Boltzmann), a dense LU solve.
"""
import json
import math
import os

import numpy as np
import pytest

from paper_1711_04060_gb300 import workloads as W

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def _gold(name):
    with open(os.path.join(GOLD, name)) as f:
        return json.load(f)


# ---------------------------------------------------------------- constants / units
def test_table1_constants(orc):
    t1 = _gold("table1_constants.json")
    kT_e = t1["k_B_J_per_K"] * t1["T_K"] / t1["e_C"]
    assert orc.thermal_voltage(t1["T_K"]) == pytest.approx(kT_e, rel=1e-14)
    # 50 mV in units of k_B T / e
    assert 0.05 / orc.thermal_voltage() == pytest.approx(1.94679, abs=2e-5)
    eps0_F_per_m = t1["eps0_F_per_cm"] * 100.0
    lam = t1["e_C"] ** 2 / (eps0_F_per_m * t1["k_B_J_per_K"] * t1["T_K"] * 1e-10)
    assert orc.lam(t1["T_K"]) == pytest.approx(lam, rel=1e-14)


def test_debye_length_textbook(orc):
    """lambda and the mol/L -> A^-3 conversion give the textbook Debye length."""
    tb = _gold("textbook_values.json")
    assert orc.molar_to_per_A3() == pytest.approx(tb["molar_per_A3"], rel=1e-15)
    c = 0.1 * orc.molar_to_per_A3()
    kappa2 = orc.lam() * (1 * 1 * c + 1 * 1 * c) / 78.5
    assert 1.0 / math.sqrt(kappa2) == pytest.approx(tb["debye_length_0p1M_A"], abs=tb["debye_length_tol_A"])


def test_species_setup_definitions(orc):
    tb = _gold("textbook_values.json")
    sp = orc.species_setup([1, -1, 0], [1.0, 2.0, 1.5], [0.1, 0.1, 55.5])
    assert sp["status"] == 0
    assert sp["v"][0] == pytest.approx(tb["sphere_volume_r1_A3"], rel=1e-14)
    assert sp["v"][1] == pytest.approx(8 * tb["sphere_volume_r1_A3"], rel=1e-14)
    # v0 is the mean volume, so the p_i average to one
    assert sp["p"].sum() == pytest.approx(3.0, rel=1e-14)
    # water at 55.5 M with radius 1.4 A fills about 38 % of space
    sp2 = orc.species_setup([1, -1, 0], [0.95, 1.81, 1.4], [0.1, 0.1, 55.5])
    vol_water = 55.5 * tb["molar_per_A3"] * 4.0 / 3.0 * math.pi * 1.4 ** 3
    assert 0.38 < vol_water < 0.39
    assert 0.6 < sp2["gammaB"] < 1.0 - vol_water
    # a charged bath is rejected
    assert orc.species_setup([1, -1, 0], [0.95, 1.81, 1.4], [0.2, 0.1, 55.5])["status"] != 0


# ---------------------------------------------------------------- Eq. (1) pointwise step
SPEC = ([1, -1, 0], [0.95, 1.81, 1.4], [0.1, 0.1, 55.5])
SPEC2 = ([1, 2, -1, 0], [0.95, 0.99, 1.81, 1.4], [0.1, 0.001, 0.102, 55.5])


@pytest.mark.parametrize("spec", [SPEC, SPEC2])
def test_fermi_bath_state(orc, spec):
    """phi = 0 gives Gamma = Gamma^B, S = 0 and the bulk concentrations (Section 2)."""
    sp = orc.species_setup(*spec)
    r = orc.fermi_point(sp, spec[0], 0.0)
    assert r["status"] == 0
    assert r["Gamma"] == pytest.approx(sp["gammaB"], rel=1e-15)
    assert abs(r["S"]) < 1e-15
    np.testing.assert_allclose(r["C"], sp["cB"], rtol=1e-14)
    assert abs(np.dot(spec[0], r["C"])) < 1e-18  # neutral bath


@pytest.mark.parametrize("phi", [-50.0, -3.0, 0.7, 10.0, 200.0])
def test_fermi_equal_radii_closed_form(orc, phi):
    """With equal radii every p_i = 1 and the void fraction has the closed form
    Gamma = 1 / (1 + sum_i v cB_i exp(-z_i phi) / Gamma^B)."""
    z = [1, -1, 2, 0]
    sp = orc.species_setup(z, [1.2] * 4, [0.3, 0.5, 0.1, 40.0])
    r = orc.fermi_point(sp, z, phi)
    assert r["status"] == 0
    v = sp["v"][0]
    # sum in log space to stay finite at large |phi|
    logs = [math.log(v * c) - zi * phi - math.log(sp["gammaB"]) for zi, c in zip(z, sp["cB"])]
    m = max(logs)
    if m > 0:
        g = math.exp(-m) / (math.exp(-m) + sum(math.exp(l - m) for l in logs))
    else:
        g = 1.0 / (1.0 + sum(math.exp(l) for l in logs))
    assert r["Gamma"] == pytest.approx(g, rel=1e-12)


@pytest.mark.parametrize("phi", [10.0, -10.0, 100.0, -100.0, 1e3, -1e3, 1e6, -1e6])
@pytest.mark.parametrize("spec", [SPEC, SPEC2])
def test_fermi_saturation(orc, phi, spec):
    """C_i < 1/v_i for any potential, even a huge one (Section 2), and Gamma = 1 - sum v_i C_i."""
    sp = orc.species_setup(*spec)
    r = orc.fermi_point(sp, spec[0], phi)
    assert r["status"] == 0
    # Gamma > 0 is carried by the finite steric potential S = ln(Gamma/Gamma^B); Gamma itself
    # underflows to 0 in FP64 once ln Gamma < -745 (phi = -1e3 puts it near -3.7e3)
    assert math.isfinite(r["S"]) and r["S"] < 0.0
    assert 0.0 <= r["Gamma"] < 1.0
    vc = sp["v"] * r["C"]
    # v_i C_i = 1 - Gamma - (others) < 1 exactly; at |phi| >> 1 the exponent of Eq. (1) is a
    # difference of two large numbers, so v_i C_i carries a rounding error of ~|phi| * 1e-16
    tol = 1e-13 * max(1.0, abs(phi))
    assert np.all(vc <= 1.0 + tol)
    assert r["Gamma"] + vc.sum() == pytest.approx(1.0, abs=tol)


def test_fermi_counterion_packing(orc):
    """Far from the bath the counter-ion fills nearly all space."""
    sp = orc.species_setup(*SPEC)
    r = orc.fermi_point(sp, SPEC[0], -1e3)  # strongly negative potential attracts Na+
    assert sp["v"][0] * r["C"][0] > 0.99
    r = orc.fermi_point(sp, SPEC[0], 1e3)
    assert sp["v"][1] * r["C"][1] > 0.99


def test_fermi_boltzmann_limit(orc):
    """Vanishing ion and water volumes turn Eq. (1) into Boltzmann distributions."""
    z = [1, -1, 0]
    sp = orc.species_setup(z, [1e-3, 1e-3, 1e-3], [0.1, 0.1, 55.5])
    for phi in (-4.0, -1.0, 0.5, 3.0):
        r = orc.fermi_point(sp, z, phi)
        np.testing.assert_allclose(r["C"], sp["cB"] * np.exp(-np.array(z) * phi), rtol=1e-7)


def test_fermi_monotone(orc):
    sp = orc.species_setup(*SPEC)
    prev = None
    for phi in np.linspace(-6, 6, 49):  # beyond this the counter-ion is packed to 1e-13
        r = orc.fermi_point(sp, SPEC[0], phi)
        if prev is not None:
            assert r["C"][0] < prev[0]  # cation decreases with potential
            assert r["C"][1] > prev[1]  # anion increases
        prev = r["C"]


# ---------------------------------------------------------------- operators (Eqs. 7, 12-18)
def test_interface_1d_exact(orc):
    """Two dielectrics (eps_m = 2 below, eps_s = 78.5 above an interface midway between two
    node planes), phi = 0 and 1 on the Dirichlet planes: the SMIB/harmonic-face scheme
    reproduces the exact piecewise-linear solution at every node."""
    nx, ny, nz, h = 3, 4, 21, 0.5
    k0 = 8  # interface between planes k0-1 and k0
    eps = np.empty((nz, ny, nx))
    eps[:k0] = 2.0
    eps[k0:] = 78.5
    A = orc.assemble_eps(nx, ny, nz, h, eps.ravel())
    b = np.zeros((nz, ny, nx))
    b[-1] = 1.0
    r = orc.bicgstab(nx, ny, nz, A, b.ravel(), tol=1e-15, max_it=500)
    assert r["status"] == 0
    # continuum: interface at z_i = (k0 - 0.5) h, slopes J/eps on each side, total drop 1
    zi = (k0 - 0.5) * h
    L = (nz - 1) * h
    J = 1.0 / (zi / 2.0 + (L - zi) / 78.5)
    zz = h * np.arange(nz)
    exact = np.where(zz < zi, J * zz / 2.0, J * zi / 2.0 + J * (zz - zi) / 78.5)
    got = r["x"].reshape(nz, ny, nx)
    np.testing.assert_allclose(got, np.broadcast_to(exact[:, None, None], got.shape), atol=1e-12)


def test_mirror_eigenfunction_3d(orc):
    """cos(pi a i/(nx-1)) cos(pi b j/(ny-1)) sin(pi c k/(nz-1)) is an exact eigenvector of the
    7-point operator with mirror sides and Dirichlet planes: A phi = eps (lx + ly + lz) phi."""
    nx, ny, nz, h, e = 5, 6, 7, 0.7, 3.5
    a, b, c = 1, 2, 3
    i = np.arange(nx)
    j = np.arange(ny)
    k = np.arange(nz)
    ph = (np.cos(np.pi * a * i / (nx - 1))[None, None, :] * np.cos(np.pi * b * j / (ny - 1))[None, :, None]
          * np.sin(np.pi * c * k / (nz - 1))[:, None, None])
    lam = sum((2 - 2 * np.cos(np.pi * m / (n - 1))) / h ** 2 for m, n in ((a, nx), (b, ny), (c, nz)))
    A = orc.assemble_eps(nx, ny, nz, h, np.full(nx * ny * nz, e))
    y = orc.dia_apply(nx, ny, nz, A, ph.ravel()).reshape(nz, ny, nx)
    np.testing.assert_allclose(y[1:-1], e * lam * ph[1:-1], atol=1e-11)
    np.testing.assert_allclose(y[[0, -1]], ph[[0, -1]], atol=1e-15)


def test_operator_row_sums_and_symmetry(orc):
    """-div(eps grad) annihilates constants away from the Dirichlet planes, and its rows are
    symmetric between interior nodes (the mirror sides make the full matrix nonsymmetric)."""
    p = W.linear_problem(n=7, seed=5, n_spheres=3)
    g = p.grid
    sig = np.linspace(0.1, 0.9, g.n)
    A = orc.assemble_eps(g.nx, g.ny, g.nz, g.h, p.eps, sig)
    ones = np.ones(g.n)
    y = orc.dia_apply(g.nx, g.ny, g.nz, A, ones).reshape(g.shape_zyx)
    np.testing.assert_allclose(y[2:-2], sig.reshape(g.shape_zyx)[2:-2], rtol=1e-12)
    M = orc.dense_from_dia(g.nx, g.ny, g.nz, A)
    idx = np.arange(g.n).reshape(g.shape_zyx)
    inner = idx[1:-1, 1:-1, 1:-1].ravel()
    sub = M[np.ix_(inner, inner)]
    np.testing.assert_allclose(sub, sub.T, rtol=1e-14, atol=0)
    # a side node couples twice as strongly to its inner neighbour as that node couples back
    c = idx[3, 3, 0]
    assert M[c, c + 1] == pytest.approx(2.0 * M[c + 1, c], rel=1e-14)
    assert not np.allclose(M, M.T)


def test_debye_huckel_slab(orc):
    """-phi'' + kD^2 phi = 0 between two Dirichlet planes: the discrete solution is
    A r^k + B r^-k with r + 1/r = 2 + kD^2 h^2 (linear PB / Debye-Hueckel)."""
    nx, ny, nz, h, e, kd = 2, 3, 41, 0.8, 78.5, 0.3
    A = orc.assemble_eps(nx, ny, nz, h, np.full(nx * ny * nz, e), np.full(nx * ny * nz, e * kd * kd))
    b = np.zeros((nz, ny, nx))
    b[0] = 1.0
    b[-1] = 0.25
    r = orc.bicgstab(nx, ny, nz, A, b.ravel(), tol=1e-15, max_it=2000)
    assert r["status"] == 0
    q = 2 + (kd * h) ** 2
    rr = (q - math.sqrt(q * q - 4)) / 2
    K = nz - 1
    # phi_k = Ac rr^k + Bc rr^(K-k):  phi_0 = 1, phi_K = 0.25
    M = np.array([[1.0, rr ** K], [rr ** K, 1.0]])
    Ac, Bc = np.linalg.solve(M, [1.0, 0.25])
    k = np.arange(nz)
    exact = Ac * rr ** k + Bc * rr ** (K - k)
    got = r["x"].reshape(nz, ny, nx)
    np.testing.assert_allclose(got, np.broadcast_to(exact[:, None, None], got.shape), atol=1e-12)


def test_pf1_structure(orc):
    """PF1 rows: eps_s (6 lc^2/h^2 + 1) on the diagonal, identity rows in the membrane and on
    the Dirichlet planes; with lc = 0 the system is diagonal and Jacobi-BiCGSTAB ends in one step."""
    p = W.channel_problem(9, box_half=4.0, slab_half=2.0, pores=((0.0, 0.0, 2.0),), n_charges=0)
    g = p.grid
    A = orc.assemble_pf1(g.nx, g.ny, g.nz, g.h, p.solvent, 78.5, 1.2)
    free = (p.solvent.reshape(g.shape_zyx).copy() == 1)
    free[0] = free[-1] = False
    free = free.ravel()
    np.testing.assert_allclose(A[0][free], 78.5 * (6 * 1.44 / g.h ** 2 + 1))
    assert np.all(A[0][~free] == 1.0) and np.all(A[1:, ~free] == 0.0)
    A0 = orc.assemble_pf1(g.nx, g.ny, g.nz, g.h, p.solvent, 78.5, 0.0)
    b = np.where(free, np.linspace(-1, 1, g.n), 0.0)
    r = orc.bicgstab(g.nx, g.ny, g.nz, A0, b, tol=1e-14)
    assert r["status"] == 0 and r["iters"] == 1
    np.testing.assert_allclose(r["x"][free], b[free] / 78.5, rtol=1e-15)


# ---------------------------------------------------------------- Table 3 solver vs dense LU
@pytest.mark.parametrize("seed", [0, 1, 2])
def test_bicgstab_matches_dense_lu(orc, seed):
    nx, ny, nz, h = 5, 4, 6, 0.9
    rng_eps = W.to_f32_exact(2.0 + 76.5 * W.uniform(W.substream(seed, 1), nx * ny * nz))
    sig = W.uniform(W.substream(seed, 2), nx * ny * nz, 0.0, 3.0)
    b = W.uniform(W.substream(seed, 3), nx * ny * nz, -1.0, 1.0)
    x0 = W.uniform(W.substream(seed, 4), nx * ny * nz, -0.5, 0.5)
    A = orc.assemble_eps(nx, ny, nz, h, rng_eps, sig)
    M = orc.dense_from_dia(nx, ny, nz, A)
    xe = np.linalg.solve(M, b)
    r = orc.bicgstab(nx, ny, nz, A, b, x0=x0, tol=1e-15, max_it=2000)
    assert r["status"] == 0
    np.testing.assert_allclose(r["x"], xe, rtol=0, atol=1e-11 * np.abs(xe).max())
    # the paper's absolute infinity-norm stop also converges to the same solution
    r2 = orc.bicgstab(nx, ny, nz, A, b, tol=1e-13, norm_mode=1, max_it=2000)
    assert r2["status"] == 0 and r2["res"] < 1e-13
    np.testing.assert_allclose(r2["x"], xe, atol=1e-10 * np.abs(xe).max())


def test_bicgstab_pf1_matches_dense_lu(orc):
    p = W.channel_problem(9, box_half=4.0, slab_half=2.0, pores=((0.5, 0.0, 2.0),), n_charges=0)
    g = p.grid
    A = orc.assemble_pf1(g.nx, g.ny, g.nz, g.h, p.solvent, 78.5, 1.2)
    b = np.where(p.solvent == 1, W.uniform(11, g.n, -1, 1), 0.0)
    xe = np.linalg.solve(orc.dense_from_dia(g.nx, g.ny, g.nz, A), b)
    r = orc.bicgstab(g.nx, g.ny, g.nz, A, b, tol=1e-15, max_it=2000)
    assert r["status"] == 0
    np.testing.assert_allclose(r["x"], xe, atol=1e-12 * np.abs(xe).max())


def _distinct_eigenvalues_of_preconditioned(orc, dims, A):
    M = orc.dense_from_dia(*dims, A)
    n = M.shape[0]
    free = np.array([not np.array_equal(M[c], np.eye(n)[c]) for c in range(n)])
    ev = np.sort(np.linalg.eigvals(M[np.ix_(free, free)] / np.diag(M)[free][:, None]).real)
    return 1 + int(np.sum(np.diff(ev) > 1e-8 * np.abs(ev).max()))


@pytest.mark.parametrize("dims", [(2, 2, 3), (3, 3, 5), (4, 3, 5)])
def test_krylov_methods_terminate_within_the_distinct_eigenvalue_count(orc, dims):
    """With m distinct eigenvalues of M^-1 A on the free rows (uniform eps and kappa), the Krylov space of r0 has
    dimension at most m, so conjugate gradients and BiCGSTAB (whose BiCG part spans the same space) end
    within m iterations: a property of the recurrences themselves (Table 3), which a wrong
    beta or omega loses."""
    nx, ny, nz = dims
    n = nx * ny * nz
    A = orc.assemble_eps(nx, ny, nz, 0.8, np.full(n, 5.0), np.full(n, 0.7))
    m = _distinct_eigenvalues_of_preconditioned(orc, dims, A)
    b = W.uniform(7, n, -1.0, 1.0)
    r = orc.bicgstab(nx, ny, nz, A, b, tol=1e-12, max_it=m)
    c = orc.pcg(nx, ny, nz, A, b, tol=1e-12, max_it=m)
    assert r["status"] == 0 and r["iters"] <= m
    assert c["status"] == 0 and c["iters"] <= m


def test_bicgstab_reports_noconv(orc):
    p = W.linear_problem(n=9, seed=3, n_spheres=4)
    g = p.grid
    A = orc.assemble_eps(g.nx, g.ny, g.nz, g.h, p.eps)
    r = orc.bicgstab(g.nx, g.ny, g.nz, A, p.b, tol=1e-14, max_it=3)
    assert r["status"] == 3 and r["iters"] == 3


# ---------------------------------------------------------------- charge spreading (Eq. 3)
def test_spread_charges_moments(orc):
    nx, ny, nz, h = 6, 5, 7, 0.8
    org = (-2.0, -1.5, -2.4)
    ch = np.array([[-1.1, 0.3, 0.77, 0.5], [1.0, -0.9, -1.3, -0.25], [0.4, 0.4, 2.4, 1.0]])
    st, f = orc.spread_charges(nx, ny, nz, h, org, ch, 7.0)
    assert st == 0
    g = W.Grid(nx, ny, nz, h, org)
    X, Y, Z = (a.ravel() for a in g.coords())
    scale = 7.0 / h ** 3
    assert f.sum() == pytest.approx(scale * ch[:, 3].sum(), rel=1e-14)
    for coord, col in ((X, 0), (Y, 1), (Z, 2)):
        assert (f * coord).sum() == pytest.approx(scale * (ch[:, 3] * ch[:, col]).sum(), rel=1e-13, abs=1e-10)
    # a charge exactly on a node lands on that node only (binary-exact grid spacing)
    hb, ob = 0.5, (-2.0, -1.5, -2.5)
    st, f1 = orc.spread_charges(nx, ny, nz, hb, ob, np.array([[ob[0] + 2 * hb, ob[1] + 3 * hb, ob[2] + hb, 1.0]]), 1.0)
    assert st == 0 and np.count_nonzero(f1) == 1
    assert f1[2 + nx * (3 + ny * 1)] == 1.0 / hb ** 3
    # and one on the last plane is kept inside the grid
    st, f2 = orc.spread_charges(nx, ny, nz, hb, ob, np.array([[ob[0] + (nx - 1) * hb, ob[1], ob[2], 1.0]]), 1.0)
    assert st == 0 and f2[nx - 1] == 1.0 / hb ** 3
    st, _ = orc.spread_charges(nx, ny, nz, h, org, np.array([[100.0, 0.0, 0.0, 1.0]]), 1.0)
    assert st != 0


# ---------------------------------------------------------------- Table 2 nonlinear loop
def _pb_newton(orc, prob, tiny):
    """Separately written nonlinear Poisson-Boltzmann solve (Newton with dense LU):
    -div(eps grad phi) = lambda [ s sum_i z_i cB_i exp(-z_i phi) ] + lambda rho_fix."""
    g = prob.grid
    lam = orc.lam(prob.T_K)
    z = np.array([s.z for s in prob.species], float)
    cB = np.array([s.bulk_M for s in prob.species]) * orc.molar_to_per_A3()
    s = prob.solvent.astype(float)
    _, ffix = orc.spread_charges(g.nx, g.ny, g.nz, g.h, g.origin, prob.charges, lam)
    Tv = orc.thermal_voltage(prob.T_K)
    phi = np.zeros(g.n).reshape(g.shape_zyx)
    phi[0] = prob.phi_lo_V / Tv
    phi[-1] = prob.phi_hi_V / Tv
    phi = phi.ravel()
    interior = np.ones(g.shape_zyx, bool)
    interior[0] = interior[-1] = False
    interior = interior.ravel()
    for _ in range(60):
        ez = np.exp(-np.outer(z, phi))
        rho = (z[:, None] * cB[:, None] * ez).sum(0)
        drho = (-(z * z)[:, None] * cB[:, None] * ez).sum(0)
        A = orc.assemble_eps(g.nx, g.ny, g.nz, g.h, prob.eps, -lam * s * drho)
        M = orc.dense_from_dia(g.nx, g.ny, g.nz, A)
        A0 = orc.assemble_eps(g.nx, g.ny, g.nz, g.h, prob.eps)
        F = orc.dia_apply(g.nx, g.ny, g.nz, A0, phi) - lam * s * rho - ffix
        F[~interior] = 0.0
        d = np.linalg.solve(M, -F)
        phi = phi + d
        if np.abs(d).max() < 1e-13:
            break
    return phi


def _small_channel(n=9, lc=1.2, tiny=False, charges=4, V=0.05, salt=0.1):
    radii = (1e-3, 1e-3, 1e-3) if tiny else (0.95, 1.81, 1.4)
    sp = [W.Species(1, radii[0], salt), W.Species(-1, radii[1], salt), W.Species(0, radii[2], 55.5)]
    return W.channel_problem(n, box_half=8.0, slab_half=3.0, pores=((0.0, 0.0, 3.0),), n_charges=charges,
                             charge_seed=9, phi_hi_V=V, species=sp, lc_A=lc)


def test_pf_reduces_to_pb(orc):
    """With lc = 0 and vanishing volumes the PF solution is the nonlinear PB solution."""
    prob = _small_channel(9, lc=0.0, tiny=True)
    out = orc.pf_solve_problem(prob, tol_outer=1e-12, lin_tol=1e-14)
    assert out["status"] == 0
    pb = _pb_newton(orc, prob, True)
    np.testing.assert_allclose(out["phi_hat"], pb, rtol=0, atol=1e-8 * np.abs(pb).max())


def test_gouy_chapman(orc):
    """1:1 salt next to a wall at potential phi0 (lc = 0, vanishing volumes): the discrete
    solution converges at second order to 4 artanh(tanh(phi0/4) exp(-kD z))."""
    errs = []
    phi0 = 2.0
    for nz in (101, 201):
        L = 100.0
        h = L / (nz - 1)
        g = W.Grid(2, 2, nz, h, (0.0, 0.0, 0.0))
        sp = [W.Species(1, 1e-3, 0.1), W.Species(-1, 1e-3, 0.1), W.Species(0, 1e-3, 55.5)]
        Tv = orc.thermal_voltage()
        z_ = [1, -1, 0]
        out = orc.pf_solve(2, 2, nz, h, g.origin, np.full(g.n, 78.5), np.ones(g.n, np.uint8), np.zeros((0, 4)),
                           phi0 * Tv, 0.0, z_, [s.radius_A for s in sp], [s.bulk_M for s in sp], 78.5, 0.0,
                           tol_outer=1e-12, lin_tol=1e-14)
        assert out["status"] == 0
        kd = math.sqrt(orc.lam() * 2 * 0.1 * orc.molar_to_per_A3() / 78.5)
        zz = h * np.arange(nz)
        exact = 4 * np.arctanh(np.tanh(phi0 / 4) * np.exp(-kd * zz))
        # far plane is held at 0 instead of the (tiny) exact value: compare away from it
        mask = zz < 40.0
        errs.append(np.abs(out["phi_hat"].reshape(nz, 2, 2)[:, 0, 0] - exact)[mask].max())
    assert errs[0] < 2e-3
    assert 3.0 < errs[0] / errs[1] < 5.0


@pytest.mark.parametrize("omega", [0.0, 0.5])
def test_fixed_point_independent_of_omega(orc, omega):
    prob = _small_channel(9)
    ref = orc.pf_solve_problem(prob, omega=0.3, tol_outer=1e-12, lin_tol=1e-14)
    out = orc.pf_solve_problem(prob, omega=omega, tol_outer=1e-12, lin_tol=1e-14)
    assert ref["status"] == 0 and out["status"] == 0
    np.testing.assert_allclose(out["phi_hat"], ref["phi_hat"], atol=1e-9 * np.abs(ref["phi_hat"]).max())


def test_fixed_point_independent_of_gamma_mode(orc):
    """Gamma as the root of its definition and the lagged reading of Eq. (11) (S from the previous iterate) reach
    the same fixed point: at convergence S = ln(Gamma(S)/Gamma^B) either way."""
    prob = _small_channel(9)
    ref = orc.pf_solve_problem(prob, tol_outer=1e-12, lin_tol=1e-14)
    lag = orc.pf_solve_problem(prob, tol_outer=1e-12, lin_tol=1e-14, gamma_mode=1)
    assert ref["status"] == 0 and lag["status"] == 0
    np.testing.assert_allclose(lag["phi_hat"], ref["phi_hat"], atol=1e-9 * np.abs(ref["phi_hat"]).max())
    for i in range(len(prob.species)):
        np.testing.assert_allclose(lag["C_M"][i], ref["C_M"][i], rtol=1e-8, atol=0)
    np.testing.assert_allclose(lag["S"], ref["S"], atol=1e-9)


def test_pf_fixed_point_satisfies_equations(orc):
    """At convergence the PF1/PF2 pair of Eqs. (12)-(13) holds with phi0 = phi, i.e.
    -div(eps grad phi) = -s eps_s Psi + lambda rho_fix and eps_s(lc^2 Lap - 1) Psi = lambda rho(phi)."""
    prob = _small_channel(9)
    g = prob.grid
    out = orc.pf_solve_problem(prob, tol_outer=1e-13, lin_tol=1e-14)
    assert out["status"] == 0
    lam = orc.lam()
    _, ffix = orc.spread_charges(g.nx, g.ny, g.nz, g.h, g.origin, prob.charges, lam)
    A = orc.assemble_eps(g.nx, g.ny, g.nz, g.h, prob.eps)
    phi = out["phi_hat"]
    s = prob.solvent.astype(float)
    res = orc.dia_apply(g.nx, g.ny, g.nz, A, phi) + s * prob.eps_s * out["Psi"] - ffix
    res = res.reshape(g.shape_zyx)[1:-1]
    scale = np.abs(ffix).max()
    assert np.abs(res).max() < 1e-8 * scale
    # PF1 with rho from the returned concentrations
    m = orc.molar_to_per_A3()
    rho = sum(sp.z * out["C_M"][i] * m for i, sp in enumerate(prob.species))
    A1 = orc.assemble_pf1(g.nx, g.ny, g.nz, g.h, prob.solvent, prob.eps_s, prob.lc_A)
    r1 = orc.dia_apply(g.nx, g.ny, g.nz, A1, out["Psi"]) + lam * rho * s
    free = (prob.solvent.reshape(g.shape_zyx).copy() == 1)
    free[0] = free[-1] = False
    assert np.abs(r1[free.ravel()]).max() < 1e-8 * np.abs(lam * rho).max()


def test_pf_zero_field_is_bath(orc):
    """No charges and no applied voltage: phi = 0 and the bath concentrations everywhere."""
    prob = _small_channel(9, charges=0, V=0.0)
    out = orc.pf_solve_problem(prob, tol_outer=1e-12, lin_tol=1e-12)
    assert out["status"] == 0
    assert np.abs(out["phi_hat"]).max() == 0.0
    sol = prob.solvent == 1
    for i, sp in enumerate(prob.species):
        np.testing.assert_allclose(out["C_M"][i][sol], sp.bulk_M, rtol=1e-14)
        assert np.all(out["C_M"][i][~sol] == 0.0)


def test_pf_antisymmetry(orc):
    """Reversing the applied voltage and every fixed charge, with cation and anion of equal
    size, reverses the potential and swaps the two ion profiles."""
    sp = [W.Species(1, 1.2, 0.1), W.Species(-1, 1.2, 0.1), W.Species(0, 1.4, 55.5)]
    a = W.channel_problem(9, box_half=8.0, slab_half=3.0, pores=((0.0, 0.0, 3.0),), n_charges=4, charge_seed=9,
                          phi_hi_V=0.05, phi_lo_V=-0.05, species=sp)
    b = W.channel_problem(9, box_half=8.0, slab_half=3.0, pores=((0.0, 0.0, 3.0),), n_charges=4, charge_seed=9,
                          phi_hi_V=-0.05, phi_lo_V=0.05, species=sp)
    b.charges[:, 3] *= -1
    oa = orc.pf_solve_problem(a, tol_outer=1e-12, lin_tol=1e-14)
    ob = orc.pf_solve_problem(b, tol_outer=1e-12, lin_tol=1e-14)
    np.testing.assert_allclose(ob["phi_hat"], -oa["phi_hat"], atol=1e-9 * np.abs(oa["phi_hat"]).max())
    np.testing.assert_allclose(ob["C_M"][0], oa["C_M"][1], rtol=1e-8, atol=1e-12)


def test_kappa_makes_pf2_a_newton_step(orc):
    """Without relaxation (omega = 0), with lc = 0 and vanishing volumes, the kappa term of Eq. (13) is the
    derivative of -lambda rho(phi), so each outer iteration is a Newton step of the PB equation: it converges
    quadratically (5 steps to 1e-12 here), where a wrong linearisation only converges linearly."""
    prob = _small_channel(9, lc=0.0, tiny=True)
    out = orc.pf_solve_problem(prob, omega=0.0, tol_outer=1e-12, lin_tol=1e-14)
    assert out["status"] == 0
    assert out["report"]["outer_iters"] <= 6


# ---------------------------------------------------------------- the correlation operator (lc > 0, Eqs. 2, 12-14)
def _linear_pf_slab_exact(K, h, lc, kd2, V, lam_t=0.0):
    """Exact discrete solution of the linearised PF pair on nodes k = 0..K of a slab, for a field
    phi = X(i) Y(j) f(k) whose transverse factor is an eigenvector of the 7-point Laplacian with
    eigenvalue -lam_t (lam_t = 0: uniform in x and y).  At the fixed point of Eqs. (11)-(13) with
    uniform eps = eps_s, no fixed charge and the Debye-Hueckel density lambda rho = -eps_s kd2 phi:
        PF2:  Psi = Lap_h phi,        PF1:  -lc^2 Lap_h Psi + Psi = kd2 phi,
    with phi = 0 / V and Psi = 0 (Eq. 14) on the planes k = 0 and k = K.  A mode f(k) = r^k has
    Lap_h = M = (r - 2 + 1/r)/h^2 - lam_t, so lc^2 M^2 - M + kd2 = 0 (the discrete form of
    Eq. 2's lc^2 phi'''' - phi'' + kd2 phi = 0): two values of M, two roots r, 1/r for each."""
    disc = np.sqrt(complex(1.0 - 4.0 * lc * lc * kd2))
    Ms = [(1.0 + disc) / (2.0 * lc * lc), (1.0 - disc) / (2.0 * lc * lc)]
    roots = []
    for M in Ms:
        q = 2.0 + (M + lam_t) * h * h
        r = (q - np.sqrt(q * q - 4.0)) / 2.0
        if abs(r) > 1.0:
            r = 1.0 / r
        roots.append(r)
    # f(k) = sum_m A_m r_m^k + B_m r_m^(K-k) (decaying from each plane); Psi-factor = sum_m M_m (...)
    rows, rhs = [], []
    for kk, fv in ((0, 0.0), (K, V)):
        rows.append([x for r in roots for x in (r ** kk, r ** (K - kk))])
        rhs.append(fv)
        rows.append([x for r, M in zip(roots, Ms) for x in (M * r ** kk, M * r ** (K - kk))])
        rhs.append(0.0)
    coef = np.linalg.solve(np.array(rows, complex), np.array(rhs, complex))
    k = np.arange(K + 1)
    f = sum(coef[2 * m] * roots[m] ** k + coef[2 * m + 1] * roots[m] ** (K - k) for m in range(2))
    psi = sum(Ms[m] * (coef[2 * m] * roots[m] ** k + coef[2 * m + 1] * roots[m] ** (K - k)) for m in range(2))
    assert np.abs(f.imag).max() < 1e-12 * abs(V) and np.abs(psi.imag).max() < 1e-12 * abs(V)
    return f.real, psi.real, [complex(M) for M in Ms]


_LC_SALT = 0.5   # mol/L 1:1 salt: 4 lc^2 kD^2 = 0.31 at lc = 1.2 A, so the two decay rates differ by 10x
_LC_V = 1e-5     # phi_hat on the upper plane: the sinh of Eq. (1) is linear to (1e-5)^2 / 6


def _lc_slab_solve(orc, nx, ny, nz, h, lc, fixed=None, fixed_phi_V=None):
    n = nx * ny * nz
    Tv = orc.thermal_voltage()
    out = orc.pf_solve(nx, ny, nz, h, (0.0, 0.0, 0.0), np.full(n, 78.5), np.ones(n, np.uint8), np.zeros((0, 4)),
                       0.0, _LC_V * Tv, [1, -1, 0], [1e-3, 1e-3, 1e-3], [_LC_SALT, _LC_SALT, 55.5], 78.5, lc,
                       tol_outer=1e-16, lin_tol=1e-14, max_outer=200, fixed=fixed, fixed_phi_V=fixed_phi_V)
    assert out["status"] == 0
    kd2 = orc.lam() * 2 * _LC_SALT * orc.molar_to_per_A3() / 78.5
    return out, kd2


@pytest.mark.parametrize("lc", [1.2, 2.0])
def test_linearised_pf_slab_closed_form(orc, lc):
    """Eq. (2) in the Debye-Hueckel limit on a slab with mirror sides: the nonlinear iteration's phi and Psi
    equal the exact discrete solution of the linearised PF pair built from the roots of its characteristic
    polynomial (two decay rates; lc = 2 A makes them complex).  This pins the off-diagonal couplings
    eps_s lc^2/h^2 of the PF1 rows (Eq. 12), the mirror doubling on their sides and Psi = 0 on the planes (Eq. 14)."""
    nx, ny, nz, h = 3, 2, 41, 0.5
    out, kd2 = _lc_slab_solve(orc, nx, ny, nz, h, lc)
    f, psi, Ms = _linear_pf_slab_exact(nz - 1, h, lc, kd2, _LC_V)
    got = out["phi_hat"].reshape(nz, ny, nx)
    gpsi = out["Psi"].reshape(nz, ny, nx)
    np.testing.assert_allclose(got, np.broadcast_to(f[:, None, None], got.shape), rtol=0, atol=2e-10 * _LC_V)
    np.testing.assert_allclose(gpsi, np.broadcast_to(psi[:, None, None], gpsi.shape), rtol=0,
                               atol=1e-9 * np.abs(psi).max())
    # the correlation term matters here: the Debye-Hueckel profile (lc = 0) is far from this one
    f0, _, _ = _linear_pf_slab_exact(nz - 1, h, 1e-6, kd2, _LC_V)
    assert np.abs(f - f0).max() > 1e-2 * _LC_V


def test_linearised_pf_transverse_mode(orc):
    """The same pair for phi = V cos(pi i/(nx-1)) cos(2 pi j/(ny-1)) held on the upper plane (fixed nodes): the
    solution keeps that transverse factor, an eigenvector of the mirrored x/y couplings with eigenvalue lam_t,
    and its z profile follows from lc^2 M^2 - M + kD^2 = 0 with M = (r - 2 + 1/r)/h^2 - lam_t.  Pins the x/y
    couplings of the PF1 rows and their mirror ghosts."""
    nx, ny, nz, h, lc = 5, 5, 33, 0.5, 1.2
    Tv = orc.thermal_voltage()
    i = np.arange(nx)
    j = np.arange(ny)
    X = np.cos(np.pi * i / (nx - 1))
    Y = np.cos(2 * np.pi * j / (ny - 1))
    lam_t = (2 - 2 * np.cos(np.pi / (nx - 1))) / h ** 2 + (2 - 2 * np.cos(2 * np.pi / (ny - 1))) / h ** 2
    fixed = np.zeros((nz, ny, nx), np.uint8)
    fixed[-1] = 1
    fval = np.zeros((nz, ny, nx))
    fval[-1] = _LC_V * Tv * Y[:, None] * X[None, :]
    out, kd2 = _lc_slab_solve(orc, nx, ny, nz, h, lc, fixed.ravel(), fval.ravel())
    f, psi, _ = _linear_pf_slab_exact(nz - 1, h, lc, kd2, _LC_V, lam_t)
    exact = f[:, None, None] * Y[None, :, None] * X[None, None, :]
    epsi = psi[:, None, None] * Y[None, :, None] * X[None, None, :]
    np.testing.assert_allclose(out["phi_hat"].reshape(nz, ny, nx), exact, rtol=0, atol=2e-10 * _LC_V)
    np.testing.assert_allclose(out["Psi"].reshape(nz, ny, nx), epsi, rtol=0, atol=1e-9 * np.abs(psi).max())


def test_linearised_pf_continuum_decay_rates(orc):
    """The discrete decay rates of the slab solution converge at second order to the continuum ones of
    lc^2 k^4 - k^2 + kD^2 = 0, k^2 = (1 +- sqrt(1 - 4 lc^2 kD^2)) / (2 lc^2) (Eq. 2 linearised)."""
    lc = 1.2
    kd2 = orc.lam() * 2 * _LC_SALT * orc.molar_to_per_A3() / 78.5
    cont = [math.sqrt((1 + s * math.sqrt(1 - 4 * lc * lc * kd2)) / (2 * lc * lc)) for s in (1, -1)]
    errs = []
    for h in (0.5, 0.25):
        _, _, Ms = _linear_pf_slab_exact(int(round(20 / h)), h, lc, kd2, _LC_V)
        disc = []
        for M in Ms:
            q = 2.0 + M.real * h * h
            r = (q - math.sqrt(q * q - 4.0)) / 2.0
            disc.append(-math.log(r) / h)
        errs.append(max(abs(a - b) / b for a, b in zip(disc, cont)))
    assert errs[0] < 2e-2
    assert 3.5 < errs[0] / errs[1] < 4.5


# ---------------------------------------------------------------- conjugate gradients for the symmetric systems
def _side_weights(nx, ny, nz):
    """1/2 for every x or y side a node lies on: the mirror ghost doubles a side row's inward coupling."""
    wx = np.where((np.arange(nx) == 0) | (np.arange(nx) == nx - 1), 0.5, 1.0)
    wy = np.where((np.arange(ny) == 0) | (np.arange(ny) == ny - 1), 0.5, 1.0)
    return np.broadcast_to(wy[:, None] * wx[None, :], (nz, ny, nx)).ravel()


def _free_rows(M):
    """Rows of a dense operator that are not identity rows (fixed nodes)."""
    eye = np.eye(M.shape[0])
    return np.array([not np.array_equal(M[c], eye[c]) for c in range(M.shape[0])])


def _eps_system(seed, nx=5, ny=4, nz=6, h=0.9):
    eps = W.to_f32_exact(2.0 + 76.5 * W.uniform(W.substream(seed, 1), nx * ny * nz))
    sig = W.uniform(W.substream(seed, 2), nx * ny * nz, 0.0, 3.0)
    b = W.uniform(W.substream(seed, 3), nx * ny * nz, -1.0, 1.0)
    x0 = W.uniform(W.substream(seed, 4), nx * ny * nz, -0.5, 0.5)
    return (nx, ny, nz), eps, sig, b, x0, h


def test_operators_symmetric_in_the_side_weighted_inner_product(orc):
    """Section 3 calls the Laplace and PF1 systems symmetric; with mirror sides and kept identity rows that holds
    for diag(w) A on the free rows, w = 1/2 per side direction (dense check on small grids, both operators)."""
    (nx, ny, nz), eps, sig, _, _, h = _eps_system(0)
    p = W.channel_problem(9, box_half=4.0, slab_half=2.0, pores=((0.5, 0.0, 2.0),), n_charges=0)
    g = p.grid
    for dims, A in (((nx, ny, nz), orc.assemble_eps(nx, ny, nz, h, eps, sig)),
                    ((g.nx, g.ny, g.nz), orc.assemble_pf1(g.nx, g.ny, g.nz, g.h, p.solvent, 78.5, 1.2))):
        M = orc.dense_from_dia(*dims, A)
        f = _free_rows(M)
        S = (_side_weights(*dims)[:, None] * M)[np.ix_(f, f)]
        np.testing.assert_allclose(S, S.T, rtol=0, atol=1e-14 * np.abs(S).max())
        assert np.all(np.linalg.eigvalsh(0.5 * (S + S.T)) > 0)  # positive definite on the free rows
        assert orc.weighted_asymmetry(*dims, A) < 1e-15
    # one coupling changed: the check sees it and conjugate gradients refuses the matrix
    A = orc.assemble_eps(nx, ny, nz, h, eps, sig).copy()
    A[1, nx + 1 + nx * ny * 2] *= 1.01
    assert orc.weighted_asymmetry(nx, ny, nz, A) > 1e-4
    assert orc.pcg(nx, ny, nz, A, b=np.ones(nx * ny * nz))["status"] == 1


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_pcg_matches_dense_lu(orc, seed):
    (nx, ny, nz), eps, sig, b, x0, h = _eps_system(seed)
    A = orc.assemble_eps(nx, ny, nz, h, eps, sig)
    xe = np.linalg.solve(orc.dense_from_dia(nx, ny, nz, A), b)
    r = orc.pcg(nx, ny, nz, A, b, x0=x0, tol=1e-15, max_it=2000)
    assert r["status"] == 0
    np.testing.assert_allclose(r["x"], xe, rtol=0, atol=1e-11 * np.abs(xe).max())
    r2 = orc.pcg(nx, ny, nz, A, b, tol=1e-13, norm_mode=1, max_it=2000)
    assert r2["status"] == 0 and r2["res"] < 1e-13
    np.testing.assert_allclose(r2["x"], xe, atol=1e-10 * np.abs(xe).max())


def test_pcg_pf1_matches_dense_lu_and_diagonal_case(orc):
    p = W.channel_problem(9, box_half=4.0, slab_half=2.0, pores=((0.5, 0.0, 2.0),), n_charges=0)
    g = p.grid
    A = orc.assemble_pf1(g.nx, g.ny, g.nz, g.h, p.solvent, 78.5, 1.2)
    b = np.where(p.solvent == 1, W.uniform(11, g.n, -1, 1), 0.0)
    xe = np.linalg.solve(orc.dense_from_dia(g.nx, g.ny, g.nz, A), b)
    r = orc.pcg(g.nx, g.ny, g.nz, A, b, tol=1e-15, max_it=2000)
    assert r["status"] == 0
    np.testing.assert_allclose(r["x"], xe, atol=1e-12 * np.abs(xe).max())
    # lc = 0: M^-1 A = I on the free rows, one step
    A0 = orc.assemble_pf1(g.nx, g.ny, g.nz, g.h, p.solvent, 78.5, 0.0)
    r0 = orc.pcg(g.nx, g.ny, g.nz, A0, b, tol=1e-14)
    assert r0["status"] == 0 and r0["iters"] == 1


def test_pcg_iterates_minimise_the_energy_norm(orc):
    """The k-th CG iterate is the minimiser of the W A-energy norm of the error over x0 plus the k-dimensional
    Krylov space of M^-1 A at M^-1 r0 (M = diag A); checked against a brute-force projection for k = 1..6."""
    (nx, ny, nz), eps, sig, b, x0, h = _eps_system(1)
    A = orc.assemble_eps(nx, ny, nz, h, eps, sig)
    M = orc.dense_from_dia(nx, ny, nz, A)
    w = _side_weights(nx, ny, nz)
    f = _free_rows(M)
    x0 = np.where(f, x0, b)  # the solver fixes the identity rows first
    xe = np.linalg.solve(M, b)
    WA = w[:, None] * M
    d = np.diag(M)
    r0 = b - M @ x0
    basis = []
    v = r0 / d
    prev = np.inf
    for k in range(1, 7):
        for q in basis:  # two Gram-Schmidt passes keep the Krylov basis orthonormal
            v = v - (q @ v) * q
        for q in basis:
            v = v - (q @ v) * q
        basis.append(v / np.linalg.norm(v))
        V = np.array(basis).T
        y = np.linalg.solve(V.T @ WA @ V, V.T @ (w * r0))
        x_best = x0 + V @ y
        got = orc.pcg(nx, ny, nz, A, b, x0=x0, tol=1e-30, max_it=k)
        assert got["status"] == 3 and got["iters"] == k
        np.testing.assert_allclose(got["x"], x_best, rtol=0, atol=1e-9 * np.abs(xe).max())
        e = got["x"] - xe
        energy = e @ WA @ e
        assert energy < prev
        prev = energy
        v = (M @ basis[-1]) / d


def test_pcg_reports_noconv_and_rejects_nonpositive_diagonal(orc):
    p = W.linear_problem(n=9, seed=3, n_spheres=4)
    g = p.grid
    A = orc.assemble_eps(g.nx, g.ny, g.nz, g.h, p.eps)
    r = orc.pcg(g.nx, g.ny, g.nz, A, p.b, tol=1e-14, max_it=3)
    assert r["status"] == 3 and r["iters"] == 3
    A2 = A.copy()
    A2[0, g.n // 2] = -1.0
    assert orc.pcg(g.nx, g.ny, g.nz, A2, p.b)["status"] == 1


@pytest.mark.parametrize("solver", [1, 2])
def test_pf_solve_with_cg_same_fixed_point(orc, solver):
    """Conjugate gradients for PF1 (and PF2) reaches the fixed point the BiCGSTAB path reaches."""
    prob = _small_channel(9)
    ref = orc.pf_solve_problem(prob, tol_outer=1e-12, lin_tol=1e-14)
    out = orc.pf_solve_problem(prob, tol_outer=1e-12, lin_tol=1e-14, solver=solver)
    assert ref["status"] == 0 and out["status"] == 0
    np.testing.assert_allclose(out["phi_hat"], ref["phi_hat"], rtol=0, atol=1e-10 * np.abs(ref["phi_hat"]).max())
    for i in range(len(prob.species)):
        np.testing.assert_allclose(out["C_M"][i], ref["C_M"][i], rtol=1e-9, atol=0)
    assert abs(out["report"]["outer_iters"] - ref["report"]["outer_iters"]) <= 1


# ---------------------------------------------------------------- a point charge in a dielectric slab (closed form)
# Box [-8, 8]^3 A with mirror sides and phi = 0 on the z planes, membrane |z| < 2.5 A (eps 2) in water (eps 80),
# one charge off the nodes.  The interface z = +-2.5 lies at face midpoints for h = 1 and h = 1/3.
SLAB = dict(L=8.0, Z=8.0, a=2.5, eps_m=2.0, eps_s=80.0)
SLAB_Q, SLAB_R0 = 1.0, (0.37, -0.21, 0.29)
SLAB_SOLVENT_PROBES = [(0, 0, 5), (2, -1, 4), (-3, 2, -5), (1, 1, -4)]
SLAB_MEMBRANE_PROBES = [(3, 2, 2), (-4, 0, -2), (0, 3, 1)]
_SLAB_REF = {}


def _slab_reference(lam):
    from tests.slab_reference import slab_potential
    if lam not in _SLAB_REF:
        _SLAB_REF[lam] = slab_potential(SLAB_SOLVENT_PROBES + SLAB_MEMBRANE_PROBES, SLAB_Q, SLAB_R0, SLAB["L"],
                                        SLAB["Z"], SLAB["a"], SLAB["eps_m"], SLAB["eps_s"], lam, 0.7)
    return _SLAB_REF[lam]


def _slab_grid(h):
    n = int(round(2 * SLAB["L"] / h)) + 1
    z = -SLAB["Z"] + h * np.arange(n)
    memb = np.broadcast_to((np.abs(z) < SLAB["a"])[:, None, None], (n, n, n)).ravel()
    eps = np.where(memb, SLAB["eps_m"], SLAB["eps_s"])
    return n, (~memb).astype(np.uint8), eps


def _at_probes(phi, n, h):
    L = SLAB["L"]
    out = []
    for (x, y, z) in SLAB_SOLVENT_PROBES + SLAB_MEMBRANE_PROBES:
        i, j, k = (int(round((c + L) / h)) for c in (x, y, z))
        out.append(phi[i + n * (j + n * k)])
    return np.array(out)


def _slab_solve(orc, h, decomposed):
    """phi at the probes: charges spread trilinearly (Eq. 3 on the grid), or the decomposition of Eqs. 5-10 with
    the interface right-hand side of Eq. 8 through the SMIB rows (17)-(18)."""
    n, sol, eps = _slab_grid(h)
    org = (-SLAB["L"], -SLAB["L"], -SLAB["Z"])
    ch = np.array([[*SLAB_R0, SLAB_Q]])
    A = orc.assemble_eps(n, n, n, h, eps)
    if decomposed:
        d = orc.decompose(n, n, n, h, org, sol, ch, SLAB["eps_m"], SLAB["eps_s"], orc.lam())
        assert d["status"] == 0
        b, G = d["bif"], d["G"]
    else:
        st, b = orc.spread_charges(n, n, n, h, org, ch, orc.lam())
        assert st == 0
        G = 0.0
    b = b.reshape(n, n, n).copy()
    b[0] = b[-1] = 0.0
    r = orc.bicgstab(n, n, n, A, b.ravel(), tol=1e-12, max_it=20000)
    assert r["status"] == 0
    return _at_probes(r["x"] + G, n, h)


def test_slab_reference_carries_the_point_charge(orc):
    """The series solution has the charge's singularity: phi(r0 + d e_z) - phi(r0 + 2d e_z) tends to
    lam q / (4 pi eps_m) (1/d - 1/(2d)), the free-space Coulomb difference, as d shrinks."""
    from tests.slab_reference import slab_potential
    lam = orc.lam()
    x0, y0, z0 = SLAB_R0
    devs = []
    for d in (0.4, 0.2):
        v = slab_potential([(x0, y0, z0 + d), (x0, y0, z0 + 2 * d)], SLAB_Q, SLAB_R0, SLAB["L"], SLAB["Z"],
                           SLAB["a"], SLAB["eps_m"], SLAB["eps_s"], lam, d)
        coulomb = lam * SLAB_Q / (4 * math.pi * SLAB["eps_m"]) * (1 / d - 1 / (2 * d))
        devs.append(abs((v[0] - v[1]) / coulomb - 1))
    assert devs[1] < 0.005 and devs[1] < devs[0] / 3


def test_slab_reference_satisfies_its_equations(orc):
    """Away from the charge: Laplace in each layer, eps dphi/dz continuous at the interface, zero normal
    derivative on a side, zero on a Dirichlet plane."""
    from tests.slab_reference import slab_potential
    lam, g = orc.lam(), SLAB
    f = lambda pts: slab_potential(pts, SLAB_Q, SLAB_R0, g["L"], g["Z"], g["a"], g["eps_m"], g["eps_s"], lam, 0.5)
    d = 0.02
    for c in ((1.0, 2.0, 4.5), (-2.0, 1.0, -1.5)):
        pts = [c] + [tuple(c[i] + s * d * (i == ax) for i in range(3)) for ax in range(3) for s in (1, -1)]
        v = f(pts)
        second = [(v[1 + 2 * ax] + v[2 + 2 * ax] - 2 * v[0]) / d ** 2 for ax in range(3)]
        assert abs(sum(second)) < 1e-3 * sum(abs(s) for s in second)
    za = g["a"]
    v = f([(1.0, 2.0, za - 2 * d), (1.0, 2.0, za - d), (1.0, 2.0, za + d), (1.0, 2.0, za + 2 * d),
           (g["L"], 1.0, 4.0), (g["L"] - d, 1.0, 4.0), (0.5, 0.5, g["Z"])])
    flux_in = g["eps_m"] * ((v[1] - v[0]) / d)  # one-sided differences: first order is enough here
    flux_out = g["eps_s"] * ((v[3] - v[2]) / d)
    assert abs(flux_in - flux_out) < 0.02 * abs(flux_in)
    assert abs(v[4] - v[5]) < 1e-3 * abs(v[4])       # dphi/dx = 0 at x = L
    assert abs(v[6]) < 1e-10


def test_spread_charge_converges_to_the_slab_solution(orc):
    """The 3D operator with trilinear charge spreading converges to the closed form at second order in the
    solvent (h = 1 -> 1/3), the assembly, the spreading and the Dirichlet/mirror treatment together."""
    ref = _slab_reference(orc.lam())
    ns = len(SLAB_SOLVENT_PROBES)
    e1 = np.abs(_slab_solve(orc, 1.0, False) - ref) / np.abs(ref)
    e3 = np.abs(_slab_solve(orc, 1.0 / 3.0, False) - ref) / np.abs(ref)
    assert e3[:ns].max() < 2.5e-3
    assert e1[:ns].mean() > 5 * e3[:ns].mean()


def test_decomposition_converges_to_the_slab_solution(orc):
    """The potential decomposition (Eqs. 5-10) with the interface right-hand side (Eqs. 8, 16-18) converges to the
    closed form at second order, and near the charge it is far more accurate than spreading the charge onto
    the grid, which is what the decomposition is for."""
    ref = _slab_reference(orc.lam())
    ns = len(SLAB_SOLVENT_PROBES)
    e1 = np.abs(_slab_solve(orc, 1.0, True) - ref) / np.abs(ref)
    e3 = np.abs(_slab_solve(orc, 1.0 / 3.0, True) - ref) / np.abs(ref)
    assert e3.max() < 2.5e-3
    assert e1.mean() > 5 * e3.mean()
    direct = np.abs(_slab_solve(orc, 1.0 / 3.0, False) - ref) / np.abs(ref)
    # the two membrane probes nearest the charge
    assert np.all(e3[ns + 1:] < direct[ns + 1:] / 10)


def test_decomposition_rejects_bad_input(orc):
    n, sol, _ = _slab_grid(1.0)
    org = (-8.0, -8.0, -8.0)
    for ch in ([[0.0, 0.0, 0.0, 1.0]],          # on a node
               [[0.3, 0.2, 9.5, 1.0]]):         # outside the box
        assert orc.decompose(n, n, n, 1.0, org, sol, np.array(ch), 2.0, 80.0, orc.lam())["status"] == 1
    s = sol.reshape(n, n, n).copy()
    s[3:6, 4, 0] = 0                           # membrane on a side whose mirror partner is solvent
    assert orc.decompose(n, n, n, 1.0, org, s.ravel(), np.array([[0.3, 0.2, 0.1, 1.0]]), 2.0, 80.0,
                         orc.lam())["status"] == 1


# ---------------------------------------------------------------- the decomposition inside the nonlinear iteration
_DEC_CHARGES = np.array([[0.37, -0.21, 0.29, 1.0], [-2.13, 1.41, -1.07, -0.5]])
_DEC_PROBES = [(0, 0, 5), (2, -1, 4), (-3, 2, -5), (1, 1, -4), (4, -4, 3)]


def _slab_channel(h):
    """The slab of the closed-form pins (membrane |z| < 2.5 A, eps 2) in 0.1 M NaCl at 50 mV."""
    n = int(round(16.0 / h)) + 1
    g = W.Grid(n, n, n, h, (-8.0, -8.0, -8.0))
    memb = np.abs(g.coords()[2]) < 2.5
    return g, (~memb).astype(np.uint8).ravel(), np.where(memb, 2.0, 78.5).ravel()


def _pf_slab(orc, h, mode, charges=_DEC_CHARGES, **kw):
    g, sol, eps = _slab_channel(h)
    out = orc.pf_solve(g.nx, g.ny, g.nz, g.h, g.origin, eps, sol, charges, 0.0, 0.05, [1, -1, 0],
                       [0.95, 1.81, 1.4], [0.1, 0.1, 55.5], 78.5, 1.2, charge_mode=mode, **kw)
    assert out["status"] == 0
    return g, sol, eps, out


def test_pf_decomposition_without_charges_is_the_plain_solve(orc):
    _, _, _, a = _pf_slab(orc, 1.0, 0, charges=np.zeros((0, 4)), tol_outer=1e-10, lin_tol=1e-12)
    _, _, _, b = _pf_slab(orc, 1.0, 1, charges=np.zeros((0, 4)), tol_outer=1e-10, lin_tol=1e-12)
    np.testing.assert_array_equal(a["phi_hat"], b["phi_hat"])


def test_pf_decomposition_fixed_point_satisfies_equations(orc):
    """With the decomposition, phi~ = phi - G solves PF2 of Eq. (13) with the jump terms of Eq. (8) as its only
    fixed-charge source: -div(eps grad phi~) = -s eps_s Psi + b_IF."""
    g, sol, eps, out = _pf_slab(orc, 1.0, 1, tol_outer=1e-13, lin_tol=1e-14)
    d = orc.decompose(g.nx, g.ny, g.nz, g.h, g.origin, sol, _DEC_CHARGES, 2.0, 78.5, orc.lam())
    phit = out["phi_hat"] - d["G"]
    A = orc.assemble_eps(g.nx, g.ny, g.nz, g.h, eps)
    res = orc.dia_apply(g.nx, g.ny, g.nz, A, phit) + sol * 78.5 * out["Psi"] - d["bif"]
    res = res.reshape(g.shape_zyx)[1:-1]
    assert np.abs(res).max() < 1e-8 * np.abs(d["bif"]).max()
    # in the solvent the returned potential is phi~ itself
    assert np.all(d["G"][sol == 1] == 0.0)


def test_pf_decomposition_agrees_with_spread_charges_as_h_shrinks(orc):
    """The two treatments of the fixed charges discretise the same PF problem: their potentials in the solvent
    approach each other under refinement (h = 1 -> 1/3)."""
    diffs = []
    for h in (1.0, 1.0 / 3.0):
        vals = []
        for mode in (0, 1):
            g, _, _, out = _pf_slab(orc, h, mode, tol_outer=1e-9, lin_tol=1e-11)
            ph = out["phi_hat"]
            vals.append(np.array([ph[int(round((x + 8) / h)) + g.nx * (int(round((y + 8) / h)) +
                                                                      g.ny * int(round((z + 8) / h)))]
                                  for x, y, z in _DEC_PROBES]))
        diffs.append(np.abs(vals[0] - vals[1]))
    assert diffs[1].max() < 2e-3
    assert diffs[0].mean() > 5 * diffs[1].mean()


# ---------------------------------------------------------------- filter-region site model (Eqs. 19-20) and coupling
def test_site_potential_of_a_charge_at_the_centre(orc):
    """All six surface points are a_b from the centre: phi_b = lam q / (4 pi eps_p a_b), plus the site's own ion
    q_b / (eps_b a_b) when occupied."""
    lam = orc.lam()
    c = np.array([[0.3, -0.2, 0.7]])
    st, phi = orc.site_potentials(c, [0.95], [1.0], [0], 10.0, [[0.3, -0.2, 0.7, -0.5]], 4.0, lam)
    assert st == 0
    assert phi[0] == pytest.approx(lam * -0.5 / (4 * math.pi * 4.0 * 0.95), rel=1e-14)
    st, phi = orc.site_potentials(c, [0.99], [2.0], [1], 10.0, [[0.3, -0.2, 0.7, -0.5]], 4.0, lam)
    assert phi[0] == pytest.approx(lam / (4 * math.pi) * (-0.5 / (4.0 * 0.99) + 2.0 / (10.0 * 0.99)), rel=1e-14)


def test_site_potential_of_another_occupied_site(orc):
    """An ion at distance D along x from site b: the six distances are D - a, D + a and four times sqrt(D^2 + a^2)."""
    lam, a, D = orc.lam(), 0.95, 3.1
    centers = np.array([[0.0, 0.0, 0.0], [D, 0.0, 0.0]])
    st, phi = orc.site_potentials(centers, [a, 0.99], [1.0, 2.0], [0, 1], 8.0, np.zeros((0, 4)), 4.0, lam)
    assert st == 0
    mean = (1 / (D - a) + 1 / (D + a) + 4 / math.sqrt(D * D + a * a)) / 6
    assert phi[0] == pytest.approx(lam / (4 * math.pi) * 2.0 / 8.0 * mean, rel=1e-14)
    # site 1 sees the empty site 0 not at all, and its own ion
    assert phi[1] == pytest.approx(lam / (4 * math.pi) * 2.0 / (8.0 * 0.99), rel=1e-14)


def test_site_potential_six_point_mean_of_a_far_charge(orc):
    """The six-point mean of 1/|c - A_k| is exact for the harmonic terms up to degree 3, so for a far charge it
    matches the sphere mean 1/d with an error falling as (a/d)^4 / d."""
    lam, a = orc.lam(), 0.95
    u = np.array([0.48, -0.6, 0.64])
    u /= np.linalg.norm(u)
    errs = []
    for d in (4.0, 8.0):
        ch = np.array([[*(d * u), 1.0]])
        st, phi = orc.site_potentials(np.zeros((1, 3)), [a], [1.0], [0], 8.0, ch, 4.0, lam)
        errs.append(abs(phi[0] * 4 * math.pi * 4.0 / lam - 1 / d))
    assert errs[0] < (a / 4.0) ** 4 / 4.0
    assert 20 < errs[0] / errs[1] < 45


def test_site_steric(orc):
    gB = 0.61412
    st, S = orc.site_steric([0.95, 0.99], [0, 0], 20.0, gB)
    assert st == 0 and S == pytest.approx(-math.log(gB), rel=1e-15)
    st, S = orc.site_steric([0.95, 0.99], [1, 0], 20.0, gB)
    assert S == pytest.approx(math.log((1 - 4 * math.pi * 0.95 ** 3 / 3 / 20.0) / gB), rel=1e-14)
    assert orc.site_steric([0.95, 0.99], [1, 1], 4.0, gB)[0] == 1  # the ions fill the site volume


def _filter_channel(lc):
    return _small_channel(17, lc=lc)


def _pore_ball(g, centre, radius):
    X, Y, Z = g.coords()
    return ((X - centre[0]) ** 2 + (Y - centre[1]) ** 2 + (Z - centre[2]) ** 2 <= radius ** 2).ravel()


def test_filter_region_holding_the_solution_changes_nothing(orc):
    """With lc = 0 each node's Psi depends only on its own density, so fixing a pore region at the potential the
    unconstrained solve found there leaves the fixed point everywhere else unchanged."""
    prob = _filter_channel(0.0)
    g = prob.grid
    free = orc.pf_solve_problem(prob, tol_outer=1e-12, lin_tol=1e-13)
    assert free["status"] == 0
    fixed = _pore_ball(g, (0.0, 0.0, 0.5), 1.6) & (prob.solvent == 1)
    assert 5 < fixed.sum() < 40
    out = orc.pf_solve_problem(prob, tol_outer=1e-12, lin_tol=1e-13, fixed=fixed.astype(np.uint8),
                               fixed_phi_V=np.where(fixed, free["phi_V"], 0.0))
    assert out["status"] == 0
    np.testing.assert_allclose(out["phi_V"], free["phi_V"], rtol=0, atol=1e-9 * np.abs(free["phi_V"]).max())
    assert np.all(out["C_M"][:, fixed] == 0.0)


def test_filter_region_with_site_potentials(orc):
    """Synthetic binding sites in the pore: Eq. (19) gives each site's potential from the wall charges and the
    occupied sites; the nodes in each site's sphere hold it as a Dirichlet value of the continuum model, and PF2
    holds at every other node."""
    prob = _filter_channel(1.2)
    g = prob.grid
    lam, Tv = orc.lam(), orc.thermal_voltage(prob.T_K)
    centres = np.array([[0.3, -0.2, -1.5], [-0.4, 0.3, 0.6], [0.2, 0.1, 2.4]])
    radii, q_ion, occ = [0.95, 0.99, 0.95], [1.0, 2.0, 1.0], [1, 0, 1]
    st, phib = orc.site_potentials(centres, radii, q_ion, occ, 20.0, prob.charges, 4.0, lam)
    assert st == 0
    fixed = np.zeros(g.n, bool)
    fval = np.zeros(g.n)
    for c, r, p in zip(centres, radii, phib):
        ball = _pore_ball(g, c, max(r, 0.87 * g.h))
        fixed |= ball
        fval[ball] = p * Tv
    assert fixed.sum() >= 3 and np.all(prob.solvent[fixed] == 1)
    out = orc.pf_solve_problem(prob, tol_outer=1e-12, lin_tol=1e-14, fixed=fixed.astype(np.uint8), fixed_phi_V=fval)
    assert out["status"] == 0
    np.testing.assert_allclose(out["phi_V"][fixed], fval[fixed], rtol=4e-16)  # volts -> k_BT/e -> volts
    _, ffix = orc.spread_charges(g.nx, g.ny, g.nz, g.h, g.origin, prob.charges, lam)
    A = orc.assemble_eps(g.nx, g.ny, g.nz, g.h, prob.eps)
    s = prob.solvent.astype(float)
    res = orc.dia_apply(g.nx, g.ny, g.nz, A, out["phi_hat"]) + s * prob.eps_s * out["Psi"] - ffix
    interior = np.zeros(g.shape_zyx, bool)
    interior[1:-1] = True
    check = interior.ravel() & ~fixed
    assert np.abs(res[check]).max() < 1e-8 * np.abs(ffix).max()
    assert np.all(out["Psi"][fixed] == 0.0) and np.all(out["C_M"][:, fixed] == 0.0)
