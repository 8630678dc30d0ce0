"""The oracle's pins catch plausible mistakes: each test compiles a copy of the oracle with one mistake planted
(on the CPU, in a temporary directory; the oracle source is untouched) and checks that at least one pin of
tests/test_oracle_pins.py fails against it."""
import os
import subprocess

import pytest

import oracle
from tests import test_oracle_pins as P

SRC = os.path.join(os.path.dirname(oracle.__file__), "pf_oracle.c")

# (name, exact text in pf_oracle.c, planted replacement)
MUTATIONS = [
    ("arithmetic-mean faces instead of the SMIB/harmonic ones (Eqs. 15-18)",
     "return 2.0 * a * b / (a + b);", "return 0.5 * (a + b);"),
    ("p_i dropped from the steric exponent of Eq. (1)",
     "double term = exp(la[i] + p[i] * u);", "double term = exp(la[i] + u);"),
    ("kappa = lambda sum z_i C_i (z_i^2 lost, Eq. 13)",
     "kap[c] += lam * z[i] * z[i] * Ci[i];", "kap[c] += lam * z[i] * Ci[i];"),
    ("east and west neighbours transposed in the operator product",
     "if (i < nx - 1) s += A[1 * N + c] * x[c + 1];\n        if (i > 0) s += A[2 * N + c] * x[c - 1];",
     "if (i < nx - 1) s += A[1 * N + c] * x[c - 1 + 2 * (i == 0)];\n"
     "        if (i > 0) s += A[2 * N + c] * x[c + 1 - 2 * (i == nx - 1)];"),
    ("sign of the -eps_s Psi term of the PF2 right-hand side (Eq. 13)",
     "(-eps_s * psi[c] + kap[c] * phi0[c])", "(eps_s * psi[c] + kap[c] * phi0[c])"),
    ("conjugate gradients with the unweighted inner product (mirror sides not symmetrised)",
     "s += side_weight(nx, ny, c) * a[c] * b[c];", "s += a[c] * b[c];"),
    ("conjugate gradients with the preconditioner left out of the search direction",
     "p[c] = z[c] + beta * p[c];", "p[c] = r[c] + beta * p[c];"),
    ("phi^L = +phi* on the interface (Eq. 10 as printed, phi discontinuous)",
     "val[sgn] = -p;", "val[sgn] = p;"),
    ("jump of Eq. 8 with the opposite sign (the sign printed in Eq. 16)",
     "const double J = eps_m * (dstar + dL);", "const double J = -eps_m * (dstar + dL);"),
    ("phi^L left out of the interface jump (Eq. 16 without it)",
     "const double J = eps_m * (dstar + dL);", "const double J = eps_m * dstar;"),
    ("BiCGSTAB beta without the alpha/omega factor (Table 3)",
     "const double beta = (rho / rho_prev) * (alpha / omega);", "const double beta = rho / rho_prev;"),
    ("BiCGSTAB omega from s.s instead of t.t (Table 3)",
     "omega = dot(N, t, s) / tt;", "omega = dot(N, t, s) / dot(N, s, s);"),
    ("phi^L boundary at the solvent node instead of the face midpoint",
     "hs[sgn] = 0.5 * h;", "hs[sgn] = h;"),
    ("first-order one-sided derivative of phi^L in the jump",
     "(8.0 * f0 - 9.0 * f1 + phiL[cm2]) / (3.0 * h)", "(f0 - f1) / (0.5 * h)"),
    ("zero normal derivative of G on the sides not imposed",
     "b[c] += -2.0 * nout * gr[a] / h;", "(void)nout;"),
    ("c0 and d0 of Eqs. 17-18 swapped",
     "bif[cm] += -eps_m * J / ((eps_m + eps_s) * h);", "bif[cm] += -eps_s * J / ((eps_m + eps_s) * h);"),
    ("site points only on the positive half-axes (Eq. 19 not symmetric)",
     "A[k / 2] += (k % 2 ? -1.0 : 1.0) * radius[b];", "A[k / 2] += radius[b];"),
    ("the site's own ion left out of Eq. 19",
     "const double own = occupied[b] ? q_ion[b] / (eps_b * radius[b]) : 0.0;", "const double own = 0.0;"),
    ("Psi left free on the filter region (Eq. 14 not applied there)",
     "fix_rows(N, fixed, A); /* Psi = 0", "/* Psi = 0"),
    ("PF1 couplings eps_s lc / h^2 instead of eps_s lc^2 / h^2 (Eq. 12)",
     "const double w = eps_s * lc * lc / (h * h);", "const double w = eps_s * lc / (h * h);"),
    ("PF1 mirror doubling dropped on the x sides (Eq. 4 for Psi)",
     "if (i < nx - 1) A[1 * N + c] -= w; else A[2 * N + c] -= w;\n        if (i > 0) A[2 * N + c] -= w; "
     "else A[1 * N + c] -= w;",
     "if (i < nx - 1) A[1 * N + c] -= w;\n        if (i > 0) A[2 * N + c] -= w;"),
    ("PF1 z couplings halved (a stray factor 1/2 on both off-diagonals)",
     "A[6 * N + c] -= w;\n        A[5 * N + c] -= w;\n        A[c] = 6.0 * w + eps_s;",
     "A[6 * N + c] -= 0.5 * w;\n        A[5 * N + c] -= 0.5 * w;\n        A[c] = 6.0 * w + eps_s;"),
]

# the pins, fastest first, with the arguments of one parametrisation each
PINS = [
    (P.test_fermi_bath_state, {"spec": P.SPEC2}),
    (P.test_fermi_equal_radii_closed_form, {"phi": 0.7}),
    (P.test_fermi_boltzmann_limit, {}),
    (P.test_interface_1d_exact, {}),
    (P.test_mirror_eigenfunction_3d, {}),
    (P.test_operator_row_sums_and_symmetry, {}),
    (P.test_debye_huckel_slab, {}),
    (P.test_bicgstab_matches_dense_lu, {"seed": 0}),
    (P.test_krylov_methods_terminate_within_the_distinct_eigenvalue_count, {"dims": (3, 3, 5)}),
    (P.test_pf_fixed_point_satisfies_equations, {}),
    (P.test_linearised_pf_slab_closed_form, {"lc": 1.2}),
    (P.test_linearised_pf_transverse_mode, {}),
    (P.test_kappa_makes_pf2_a_newton_step, {}),
    (P.test_pf_reduces_to_pb, {}),
    (P.test_pcg_iterates_minimise_the_energy_norm, {}),
    (P.test_decomposition_converges_to_the_slab_solution, {}),
    (P.test_site_potential_of_a_charge_at_the_centre, {}),
    (P.test_site_potential_six_point_mean_of_a_far_charge, {}),
    (P.test_filter_region_with_site_potentials, {}),
]


def _build_mutant(tmp_path, old, new):
    src = open(SRC).read()
    assert src.count(old) == 1, old
    path = tmp_path / "pf_oracle.c"
    path.write_text(src.replace(old, new))
    for h in ("pf_oracle.h",):
        (tmp_path / h).write_text(open(os.path.join(os.path.dirname(SRC), h)).read())
    so = tmp_path / "liboracle_mutant.so"
    subprocess.check_call(["gcc", "-O2", "-std=c11", "-D_DEFAULT_SOURCE", "-ffp-contract=off", "-fno-fast-math",
                           "-shared", "-fPIC", "-o", str(so), str(path), "-lm"])
    return oracle.load(str(so))


def test_pins_pass_on_the_oracle():
    for pin, kw in PINS:
        pin(oracle, **kw)


@pytest.mark.parametrize("name,old,new", MUTATIONS, ids=[m[0][:40] for m in MUTATIONS])
def test_planted_mistake_fails_a_pin(tmp_path, name, old, new):
    mutant = _build_mutant(tmp_path, old, new)
    failed = []
    with oracle.using(mutant):
        for pin, kw in PINS:
            try:
                pin(oracle, **kw)
            except AssertionError:
                failed.append(pin.__name__)
                break
    assert failed, f"no pin catches: {name}"
