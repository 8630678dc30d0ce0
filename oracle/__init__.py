"""Python access to the FP64 CPU oracle in pf_oracle.c.

TEST INFRASTRUCTURE ONLY.  Only the tests, the package smoke check and the CPU-baseline
leg of the benchmark may import this module.  It imports nothing from the CUDA library or
its package; callers pass plain arrays.
"""
from __future__ import annotations

import contextlib
import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "pf_oracle.c")
_SO = os.path.join(_HERE, "_build", "liboracle.so")
_lib = None

_D = ctypes.c_double
_I = ctypes.c_int
_PD = ctypes.POINTER(ctypes.c_double)
_PU8 = ctypes.POINTER(ctypes.c_uint8)
_PI = ctypes.POINTER(ctypes.c_int)


class NlOpts(ctypes.Structure):
    _fields_ = [("omega", _D), ("tol_outer", _D), ("lin_tol", _D), ("lin_norm", _I),
                ("max_outer", _I), ("max_lin", _I), ("solver", _I), ("charge_mode", _I), ("gamma_mode", _I)]


class NlReport(ctypes.Structure):
    _fields_ = [("status", _I), ("outer_iters", _I), ("lin_iters_total", _I),
                ("lin_iters_first", _I), ("delta", _D)]


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (plain IEEE arithmetic: no fast-math, no FMA contraction)."""
    os.makedirs(os.path.dirname(_SO), exist_ok=True)
    if force or not os.path.exists(_SO) or os.path.getmtime(_SO) < max(
            os.path.getmtime(_SRC), os.path.getmtime(os.path.join(_HERE, "pf_oracle.h"))):
        tmp = _SO + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-D_DEFAULT_SOURCE", "-ffp-contract=off",
                               "-fno-fast-math", "-shared", "-fPIC", "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _SO)
    return _SO


_SO_OMP = os.path.join(_HERE, "_build", "liboracle_omp.so")


def build_all_cores(force: bool = False) -> str:
    """The benchmark's all-cores timing copy: the same source compiled with -fopenmp, which turns on its
    OpenMP pragmas (operator product, inner products, vector updates, the pointwise node loop).  Its
    reductions run in another order, so it is never the checker: tests use build()."""
    os.makedirs(os.path.dirname(_SO_OMP), exist_ok=True)
    if force or not os.path.exists(_SO_OMP) or os.path.getmtime(_SO_OMP) < max(
            os.path.getmtime(_SRC), os.path.getmtime(os.path.join(_HERE, "pf_oracle.h"))):
        tmp = _SO_OMP + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-D_DEFAULT_SOURCE", "-ffp-contract=off",
                               "-fno-fast-math", "-fopenmp", "-shared", "-fPIC", "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _SO_OMP)
    return _SO_OMP


def lib():
    global _lib
    if _lib is None:
        _lib = load(build())
    return _lib


def load(path):
    """The oracle library at `path` with its ctypes signatures (the tests also load mutated copies)."""
    L = ctypes.CDLL(path)
    L.pfo_thermal_voltage.restype = _D
    L.pfo_thermal_voltage.argtypes = [_D]
    L.pfo_lambda.restype = _D
    L.pfo_lambda.argtypes = [_D]
    L.pfo_molar_to_per_A3.restype = _D
    L.pfo_molar_to_per_A3.argtypes = []
    L.pfo_species_setup.argtypes = [_I, _PD, _PD, _PD, _PD, _PD, _PD, _PD]
    L.pfo_fermi_point.argtypes = [_I, _PD, _PD, _PD, _PD, _D, _D, _PD, _PD, _PD, _PI]
    L.pfo_fermi_nodes.argtypes = [_I, _PD, _PD, _PD, _PD, _D, ctypes.c_long, _PD, _PD, _PD, _PD]
    L.pfo_assemble_eps.argtypes = [_I, _I, _I, _D, _PD, _PD, _PD]
    L.pfo_assemble_pf1.argtypes = [_I, _I, _I, _D, _PU8, _D, _D, _PD]
    L.pfo_dia_apply.argtypes = [_I, _I, _I, _PD, _PD, _PD]
    L.pfo_dia_apply.restype = None
    L.pfo_bicgstab.argtypes = [_I, _I, _I, _PD, _PD, _PD, _I, _D, _I, _PI, _PD]
    L.pfo_pcg.argtypes = [_I, _I, _I, _PD, _PD, _PD, _I, _D, _I, _PI, _PD]
    L.pfo_weighted_asymmetry.restype = _D
    L.pfo_weighted_asymmetry.argtypes = [_I, _I, _I, _PD]
    L.pfo_decompose.argtypes = [_I, _I, _I, _D, _PD, _PU8, _I, _PD, _D, _D, _D, _PD, _PD, _PI]
    L.pfo_spread_charges.argtypes = [_I, _I, _I, _D, _PD, _I, _PD, _D, _PD]
    L.pfo_pf_solve.argtypes = [_I, _I, _I, _D, _PD, _PD, _PU8, _I, _PD, _D, _D, _I, _PD, _PD, _PD,
                               _D, _D, _D, ctypes.POINTER(NlOpts), _PD, _PD, _PD, _PD, _PD, _PD,
                               ctypes.POINTER(NlReport)]
    L.pfo_pf_solve_fixed.argtypes = [_I, _I, _I, _D, _PD, _PD, _PU8, _I, _PD, _D, _D, _I, _PD, _PD, _PD,
                                     _D, _D, _D, ctypes.POINTER(NlOpts), _PU8, _PD, _PD, _PD, _PD, _PD, _PD, _PD,
                                     ctypes.POINTER(NlReport)]
    L.pfo_site_potentials.argtypes = [_I, _PD, _PD, _PD, _PI, _D, _I, _PD, _D, _D, _PD]
    L.pfo_site_steric.argtypes = [_I, _PD, _PI, _D, _D, _PD]
    return L


@contextlib.contextmanager
def using(L):
    """Routes every oracle call inside the block to the library L."""
    global _lib
    saved = _lib
    _lib = L
    try:
        yield
    finally:
        _lib = saved


def _pd(a):
    return a.ctypes.data_as(_PD) if a is not None else None


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def thermal_voltage(T=298.15) -> float:
    return lib().pfo_thermal_voltage(T)


def lam(T=298.15) -> float:
    return lib().pfo_lambda(T)


def molar_to_per_A3() -> float:
    return lib().pfo_molar_to_per_A3()


def species_setup(z, radius, bulk):
    z, radius, bulk = _f64(z), _f64(radius), _f64(bulk)
    n = len(z)
    v, p, cB = np.zeros(n), np.zeros(n), np.zeros(n)
    g = ctypes.c_double(0.0)
    st = lib().pfo_species_setup(n, _pd(z), _pd(radius), _pd(bulk), _pd(v), _pd(p), _pd(cB), ctypes.byref(g))
    return {"status": st, "v": v, "p": p, "cB": cB, "gammaB": g.value}


def fermi_point(sp: dict, z, phi_hat: float):
    """Eq. (1) at one node; sp is the result of species_setup."""
    z = _f64(z)
    n = len(z)
    C = np.zeros(n)
    S, G = ctypes.c_double(0.0), ctypes.c_double(0.0)
    it = ctypes.c_int(0)
    st = lib().pfo_fermi_point(n, _pd(z), _pd(sp["v"]), _pd(sp["p"]), _pd(sp["cB"]), sp["gammaB"],
                               float(phi_hat), _pd(C), ctypes.byref(S), ctypes.byref(G), ctypes.byref(it))
    return {"status": st, "C": C, "S": S.value, "Gamma": G.value, "iters": it.value}


def fermi_nodes(sp: dict, z, phi_hat):
    """Eq. (1) at every node of the array phi_hat: C (species-major, A^-3), S, Gamma and the status."""
    z = _f64(z)
    ph = _f64(phi_hat)
    n, ns = len(ph), len(z)
    C, S, G = np.zeros(ns * n), np.zeros(n), np.zeros(n)
    st = lib().pfo_fermi_nodes(ns, _pd(z), _pd(sp["v"]), _pd(sp["p"]), _pd(sp["cB"]), sp["gammaB"], n, _pd(ph),
                               _pd(C), _pd(S), _pd(G))
    return {"status": st, "C": C.reshape(ns, n), "S": S, "Gamma": G}


def assemble_eps(nx, ny, nz, h, eps, sigma=None):
    eps = _f64(eps)
    sig = _f64(sigma) if sigma is not None else None
    A = np.zeros(7 * nx * ny * nz)
    st = lib().pfo_assemble_eps(nx, ny, nz, h, _pd(eps), _pd(sig), _pd(A))
    assert st == 0, st
    return A.reshape(7, -1)


def assemble_pf1(nx, ny, nz, h, solvent, eps_s, lc):
    sol = np.ascontiguousarray(solvent, dtype=np.uint8)
    A = np.zeros(7 * nx * ny * nz)
    st = lib().pfo_assemble_pf1(nx, ny, nz, h, sol.ctypes.data_as(_PU8), eps_s, lc, _pd(A))
    assert st == 0, st
    return A.reshape(7, -1)


def dia_apply(nx, ny, nz, A, x):
    A = _f64(A).ravel()
    x = _f64(x)
    y = np.zeros_like(x)
    lib().pfo_dia_apply(nx, ny, nz, _pd(A), _pd(x), _pd(y))
    return y


def dense_from_dia(nx, ny, nz, A):
    """The N x N matrix of a 7-diagonal operator (tiny grids only)."""
    N = nx * ny * nz
    M = np.zeros((N, N))
    e = np.zeros(N)
    for j in range(N):
        e[:] = 0.0
        e[j] = 1.0
        M[:, j] = dia_apply(nx, ny, nz, A, e)
    return M


def bicgstab(nx, ny, nz, A, b, x0=None, max_it=1000, tol=1e-12, norm_mode=0):
    A = _f64(A).ravel()
    b = _f64(b)
    x = np.zeros_like(b) if x0 is None else _f64(x0).copy()
    it = ctypes.c_int(0)
    res = ctypes.c_double(0.0)
    st = lib().pfo_bicgstab(nx, ny, nz, _pd(A), _pd(b), _pd(x), max_it, tol, norm_mode, ctypes.byref(it),
                            ctypes.byref(res))
    return {"status": st, "x": x, "iters": it.value, "res": res.value}


def pcg(nx, ny, nz, A, b, x0=None, max_it=1000, tol=1e-12, norm_mode=0):
    """Jacobi-preconditioned conjugate gradients (pfo_pcg); same results dict as bicgstab."""
    A = _f64(A).ravel()
    b = _f64(b)
    x = np.zeros_like(b) if x0 is None else _f64(x0).copy()
    it = ctypes.c_int(0)
    res = ctypes.c_double(0.0)
    st = lib().pfo_pcg(nx, ny, nz, _pd(A), _pd(b), _pd(x), max_it, tol, norm_mode, ctypes.byref(it),
                       ctypes.byref(res))
    return {"status": st, "x": x, "iters": it.value, "res": res.value}


def weighted_asymmetry(nx, ny, nz, A):
    A = _f64(A).ravel()
    return lib().pfo_weighted_asymmetry(nx, ny, nz, _pd(A))


def spread_charges(nx, ny, nz, h, origin, charges, lam_value):
    ch = _f64(charges).ravel()
    org = _f64(origin)
    f = np.zeros(nx * ny * nz)
    st = lib().pfo_spread_charges(nx, ny, nz, h, _pd(org), len(ch) // 4, _pd(ch), lam_value, _pd(f))
    return st, f


def decompose(nx, ny, nz, h, origin, solvent, charges, eps_m, eps_s, lam_value):
    """G = phi* + phi^L at membrane nodes and the interface right-hand side (pfo_decompose)."""
    sol = np.ascontiguousarray(solvent, dtype=np.uint8)
    ch = _f64(charges).ravel()
    org = _f64(origin)
    N = nx * ny * nz
    G, bif = np.zeros(N), np.zeros(N)
    it = ctypes.c_int(0)
    st = lib().pfo_decompose(nx, ny, nz, h, _pd(org), sol.ctypes.data_as(_PU8), len(ch) // 4, _pd(ch), eps_m,
                             eps_s, lam_value, _pd(G), _pd(bif), ctypes.byref(it))
    return {"status": st, "G": G, "bif": bif, "iters": it.value}


def pf_solve(nx, ny, nz, h, origin, eps, solvent, charges, phi_lo_V, phi_hi_V, z, radius, bulk,
             eps_s, lc, T=298.15, omega=0.3, tol_outer=1e-10, lin_tol=1e-12, lin_norm=0, max_outer=500,
             max_lin=20000, solver=0, charge_mode=0, fixed=None, fixed_phi_V=None, gamma_mode=0):
    """Table 2 nonlinear PF solve; returns a dict of fields and the report."""
    N = nx * ny * nz
    ns = len(z)
    eps = _f64(eps)
    sol = np.ascontiguousarray(solvent, dtype=np.uint8)
    ch = _f64(charges).ravel()
    org = _f64(origin)
    z, radius, bulk = _f64(z), _f64(radius), _f64(bulk)
    out = {k: np.zeros(N) for k in ("phi_V", "S", "Gamma", "Psi", "phi_hat")}
    out["C_M"] = np.zeros(ns * N)
    opts = NlOpts(omega, tol_outer, lin_tol, lin_norm, max_outer, max_lin, solver, charge_mode, gamma_mode)
    rep = NlReport()
    outs = (_pd(out["phi_V"]), _pd(out["C_M"]), _pd(out["S"]), _pd(out["Gamma"]), _pd(out["Psi"]),
            _pd(out["phi_hat"]), ctypes.byref(rep))
    head = (nx, ny, nz, h, _pd(org), _pd(eps), sol.ctypes.data_as(_PU8), len(ch) // 4, _pd(ch), phi_lo_V, phi_hi_V,
            ns, _pd(z), _pd(radius), _pd(bulk), eps_s, lc, T, ctypes.byref(opts))
    if fixed is None:
        st = lib().pfo_pf_solve(*head, *outs)
    else:
        fx = np.ascontiguousarray(fixed, dtype=np.uint8)
        fv = _f64(fixed_phi_V)
        st = lib().pfo_pf_solve_fixed(*head, fx.ctypes.data_as(_PU8), _pd(fv), *outs)
    out["C_M"] = out["C_M"].reshape(ns, N)
    out["status"] = st
    out["report"] = {f: getattr(rep, f) for f, _ in NlReport._fields_}
    return out


def pf_solve_problem(prob, **kw):
    """pf_solve on any object with the fields of a channel problem (grid, eps, solvent, ...)."""
    g = prob.grid
    z = [s.z for s in prob.species]
    r = [s.radius_A for s in prob.species]
    c = [s.bulk_M for s in prob.species]
    return pf_solve(g.nx, g.ny, g.nz, g.h, g.origin, prob.eps, prob.solvent, prob.charges, prob.phi_lo_V,
                    prob.phi_hi_V, z, r, c, prob.eps_s, prob.lc_A, prob.T_K, **kw)


def site_potentials(centers, radii, q_ion, occupied, eps_b, charges, eps_p, lam_value):
    """Eq. (19) for every site; returns (status, phi_hat per site)."""
    c = _f64(centers).ravel()
    r, q = _f64(radii), _f64(q_ion)
    occ = np.ascontiguousarray(occupied, dtype=np.int32)
    ch = _f64(charges).ravel()
    out = np.zeros(len(r))
    st = lib().pfo_site_potentials(len(r), _pd(c), _pd(r), _pd(q), occ.ctypes.data_as(_PI), eps_b, len(ch) // 4,
                                   _pd(ch), eps_p, lam_value, _pd(out))
    return st, out


def site_steric(ion_radii, occupied, v_sites, gammaB):
    """Eq. (20); returns (status, S)."""
    r = _f64(ion_radii)
    occ = np.ascontiguousarray(occupied, dtype=np.int32)
    S = ctypes.c_double(0.0)
    st = lib().pfo_site_steric(len(r), _pd(r), occ.ctypes.data_as(_PI), v_sites, gammaB, ctypes.byref(S))
    return st, S.value
