"""Closed-form continuum reference for the pins of the 3D operator and of the potential decomposition.

A point charge q at r0 inside a dielectric slab: -div(eps grad phi) = lam q delta(r - r0) in the box
[-L, L]^2 x [-Z, Z], eps = eps_m for |z| < a and eps_s outside, zero normal derivative on the sides
x, y = +-L (the mirror sides of Eq. 4) and phi = 0 on the planes z = +-Z.  The cosine series in x and y
turns it into one 1D problem per mode k: -(eps Phi')' + eps k^2 Phi = s delta(z - z0), Phi(+-Z) = 0, with
Phi and eps Phi' continuous at z = +-a.  It is solved exactly by matching the homogeneous solutions u-
(zero at -Z) and u+ (zero at +Z) at z0.  Both are carried with their growth factors exp(k(z + Z)) and
exp(k(Z - z)) divided out, so no mode overflows.  The mode sum converges geometrically at points off
the plane of the charge.  Test infrastructure only.
"""
import numpy as np


def _propagate(k, z, Z, a, eps_m, eps_s, from_below):
    """Scaled (u, eps u') at z of the homogeneous solution with u = 0, u' = +1 at -Z (from_below) or
    u = 0, u' = -1 at +Z, for an array of k; the growth factor exp(k * distance travelled) is divided out."""
    bounds = [-Z, -a, a, Z]
    eps = [eps_s, eps_m, eps_s]
    u = np.zeros_like(k)
    f = np.full_like(k, eps[0] if from_below else -eps[2])
    zc, li = (-Z, 0) if from_below else (Z, 2)
    kk = np.where(k > 0, k, 1.0)
    while True:
        zend = min(bounds[li + 1], z) if from_below else max(bounds[li], z)
        d = abs(zend - zc)
        sgn = 1.0 if from_below else -1.0
        du = f / eps[li]
        E = np.exp(-2.0 * k * d)
        ch = 0.5 * (1.0 + E)                          # cosh(kd) exp(-kd)
        shk = np.where(k > 0, 0.5 * (1.0 - E) / kk, d)  # sinh(kd) exp(-kd) / k  (d at k = 0)
        ksh = k * k * shk                                  # k sinh(kd) exp(-kd)
        u, du = u * ch + sgn * du * shk, sgn * u * ksh + du * ch
        f = du * eps[li]
        if (from_below and zend >= z) or (not from_below and zend <= z):
            return u, f
        zc, li = zend, li + (1 if from_below else -1)


def slab_potential(points, q, r0, L, Z, a, eps_m, eps_s, lam, dz_min):
    """phi at the given points (each at least dz_min from the plane z = z0 of the charge)."""
    kmax = 36.0 / dz_min  # a term decays like exp(-k |z - z0|)
    M = int(kmax * 2 * L / np.pi) + 2
    km = np.arange(M) * np.pi / (2 * L)
    norm = np.where(np.arange(M) == 0, 2 * L, L)  # integral of cos^2 over [-L, L]
    mi, ni = np.meshgrid(np.arange(M), np.arange(M), indexing="ij")
    k = np.hypot(km[mi], km[ni])
    keep = k <= kmax
    mi, ni, k = mi[keep], ni[keep], k[keep]
    x0, y0, z0 = r0
    s = lam * q * np.cos(km[mi] * (x0 + L)) * np.cos(km[ni] * (y0 + L)) / (norm[mi] * norm[ni])
    um, fm = _propagate(k, z0, Z, a, eps_m, eps_s, True)    # scaled by exp(-k (z0 + Z))
    up, fp = _propagate(k, z0, Z, a, eps_m, eps_s, False)   # scaled by exp(-k (Z - z0))
    det = um * fp - up * fm                                   # scaled by exp(-2 k Z)
    out = np.zeros(len(points))
    for t, (x, y, z) in enumerate(points):
        if z <= z0:   # Phi = -s u+(z0) u-(z) / det
            u, _ = _propagate(k, z, Z, a, eps_m, eps_s, True)
            Phi = -s * up * u / det * np.exp(-k * (z0 - z))
        else:         # Phi = -s u-(z0) u+(z) / det
            u, _ = _propagate(k, z, Z, a, eps_m, eps_s, False)
            Phi = -s * um * u / det * np.exp(-k * (z - z0))
        out[t] = np.sum(Phi * np.cos(km[mi] * (x + L)) * np.cos(km[ni] * (y + L)))
    return out
