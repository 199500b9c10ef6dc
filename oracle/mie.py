"""Analytic scattering by a homogeneous dielectric cylinder (2D) and sphere (3D), scalar Mie series.

Not from the paper: a textbook closed form that pins the discretised model of
Sec. II (Green's function sign of Eq. 1, the k^2 delta^2 quadrature, the self
term).  A plane wave exp(j k x) hits a cylinder of radius a and contrast f
(interior wavenumber k1 = k sqrt(1 + f)); matching u and du/dr at r = a for
each angular order m gives the scattered field outside

    u_sc(r, phi) = sum_m j^m a_m H_m(k r) e^{j m phi},
    a_m = [k1 J_m'(k1 a) J_m(k a) - k J_m(k1 a) J_m'(k a)]
        / [k J_m(k1 a) H_m'(k a) - k1 J_m'(k1 a) H_m(k a)],

with H_m the Hankel function of the first kind (outgoing for e^{-j w t}).
"""
from __future__ import annotations

import numpy as np
from scipy import special


def mie_cylinder(points, radius, contrast, k, orders=None):
    """Scattered field at ``points`` [M, 2] outside a centred cylinder, incidence along +x."""
    pts = np.asarray(points, dtype=np.float64)
    r = np.hypot(pts[:, 0], pts[:, 1])
    phi = np.arctan2(pts[:, 1], pts[:, 0])
    k1 = k * np.sqrt(1.0 + contrast + 0j)
    ka, k1a = k * radius, k1 * radius
    if orders is None:
        orders = int(abs(k1a) + 4.0 * abs(k1a) ** (1.0 / 3.0) + 12)
    out = np.zeros(len(pts), dtype=np.complex128)
    for m in range(-orders, orders + 1):
        Jm_k1a = special.jv(m, k1a)
        dJm_k1a = special.jvp(m, k1a)
        num = k1 * dJm_k1a * special.jv(m, ka) - k * Jm_k1a * special.jvp(m, ka)
        den = k * Jm_k1a * special.h1vp(m, ka) - k1 * dJm_k1a * special.hankel1(m, ka)
        am = num / den
        out += (1j ** m) * am * special.hankel1(m, k * r) * np.exp(1j * m * phi)
    return out


def mie_sphere(points, radius, contrast, k, orders=None):
    """Scattered field at ``points`` [M, 3] outside a centred sphere, scalar wave
    exp(j k z) incident along +z:
        u_sc = sum_l (2l + 1) j^l a_l h_l(k r) P_l(cos theta),
        a_l = [k1 j_l'(k1 a) j_l(k a) - k j_l(k1 a) j_l'(k a)]
            / [k j_l(k1 a) h_l'(k a) - k1 j_l'(k1 a) h_l(k a)],
    with h_l = j_l + j y_l the outgoing spherical Hankel function."""
    pts = np.asarray(points, dtype=np.float64)
    r = np.linalg.norm(pts, axis=1)
    cth = pts[:, 2] / r
    k1 = k * np.sqrt(1.0 + contrast)
    ka, k1a = k * radius, k1 * radius
    if orders is None:
        orders = int(k1a + 4.0 * k1a ** (1.0 / 3.0) + 12)
    out = np.zeros(len(pts), dtype=np.complex128)
    for l in range(orders + 1):
        jl_k1a = special.spherical_jn(l, k1a)
        djl_k1a = special.spherical_jn(l, k1a, derivative=True)
        jl_ka = special.spherical_jn(l, ka)
        djl_ka = special.spherical_jn(l, ka, derivative=True)
        hl_ka = jl_ka + 1j * special.spherical_yn(l, ka)
        dhl_ka = djl_ka + 1j * special.spherical_yn(l, ka, derivative=True)
        al = (k1 * djl_k1a * jl_ka - k * jl_k1a * djl_ka) / (k * jl_k1a * dhl_ka - k1 * djl_k1a * hl_ka)
        hl_kr = special.spherical_jn(l, k * r) + 1j * special.spherical_yn(l, k * r)
        out += (2 * l + 1) * (1j ** l) * al * hl_kr * special.eval_legendre(l, cth)
    return out
