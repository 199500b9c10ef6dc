"""Discretised scalar Lippmann-Schwinger model (Sec. II) in FP64.

Grid (Appendix A, Sec. "Discretization", used here in 2D as well): pixel l of
an n-pixel axis sits at r_l = (l - n/2 - 0.5) * delta, l = 1..n; images are
row-major with x fastest, f[iy, ix].

Green's function (Eq. 1): the paper prints -(j/4) H0(k_b r) for d = 2 but
+e^{j k_b r}/(4 pi r) for d = 3.  Only +(j/4) H0 agrees with the 3D sign and
with u = u_in + k^2 int g f u for (lap + k_b^2) g = -delta; this oracle uses
+(j/4) H0^(1)(k_b r) (the Mie-series pin fixes the sign).

G (Eq. 3) and H (Eq. 2) are the midpoint-rule discretisations
k^2 delta^d g(|r_i - r_j|); the singular self term G_ii, on which the paper is
silent, integrates g over the disk (2D) or ball (3D) of the pixel's area or
volume.

Pinned by: dense brute-force G vs the FFT convolution, padding independence,
the adjoint identity, the Mie series (tests/test_oracle_model.py).
"""
from __future__ import annotations

import math

import numpy as np
from scipy import special


def wavenumbers(wavelength: float = 1.0, eps_b: float = 1.0):
    """k = 2 pi / lambda (vacuum) and k_b = k sqrt(eps_b) (Sec. II, after Eq. 1)."""
    k = 2.0 * math.pi / wavelength
    return k, k * math.sqrt(eps_b)


def axis_centres(n: int, delta: float) -> np.ndarray:
    """r_l = (l - n/2 - 0.5) delta for l = 1..n (Appendix A grid)."""
    return (np.arange(1, n + 1) - n / 2.0 - 0.5) * delta


def grid_points(n: int, delta: float, dim: int = 2) -> np.ndarray:
    """[N, dim] pixel centres, x fastest."""
    c = axis_centres(n, delta)
    if dim == 2:
        Y, X = np.meshgrid(c, c, indexing="ij")
        return np.stack([X.ravel(), Y.ravel()], axis=1)
    Z, Y, X = np.meshgrid(c, c, c, indexing="ij")
    return np.stack([X.ravel(), Y.ravel(), Z.ravel()], axis=1)


def green(r: np.ndarray, kb: float, dim: int = 2) -> np.ndarray:
    """Free-space Green's function g(r) of Eq. 1 (2D sign read as +j/4)."""
    r = np.asarray(r, dtype=np.float64)
    if dim == 2:
        return 0.25j * special.hankel1(0, kb * r)
    return np.exp(1j * kb * r) / (4.0 * math.pi * r)


def self_term(k: float, kb: float, delta: float, dim: int = 2) -> complex:
    """G_ii = k^2 * integral of g over the pixel's equal-area disk / equal-volume ball.

    2D: int_0^a H0(kb r) r dr = a H1(kb a)/kb + 2j/(pi kb^2), times (j/4) 2 pi.
    3D: int_0^a r e^{j kb r} dr = [(1 - j kb a) e^{j kb a} - 1] / kb^2.
    """
    if dim == 2:
        a = delta / math.sqrt(math.pi)
        return k * k * (1j * math.pi * a / (2.0 * kb) * special.hankel1(1, kb * a) - 1.0 / (kb * kb))
    a = delta * (3.0 / (4.0 * math.pi)) ** (1.0 / 3.0)
    return (k * k / (kb * kb)) * ((1.0 - 1j * kb * a) * np.exp(1j * kb * a) - 1.0)


def green_matrix(n: int, delta: float, k: float, kb: float, dim: int = 2) -> np.ndarray:
    """Dense G in C^{N x N} (Eq. 3): G_ij = k^2 delta^d g(|r_i - r_j|), G_ii = self term."""
    pts = grid_points(n, delta, dim)
    d = np.sqrt(((pts[:, None, :] - pts[None, :, :]) ** 2).sum(-1))
    N = pts.shape[0]
    G = np.empty((N, N), dtype=np.complex128)
    off = ~np.eye(N, dtype=bool)
    G[off] = k * k * delta ** dim * green(d[off], kb, dim)
    G[np.eye(N, dtype=bool)] = self_term(k, kb, delta, dim)
    return G


def circulant_column(n: int, P: int, delta: float, k: float, kb: float, dim: int = 2) -> np.ndarray:
    """First column of the P^d circulant embedding of the (block-)Toeplitz G.

    Index j of an axis holds the offset m = j for j < n, m = j - P for
    j > P - n, and 0 for the unused offsets in between (P >= 2n - 1).
    """
    assert P >= 2 * n - 1
    j = np.arange(P)
    m = np.where(j < n, j, j - P).astype(np.float64)
    used = (j < n) | (j > P - n)
    if dim == 2:
        MY, MX = np.meshgrid(m, m, indexing="ij")
        UY, UX = np.meshgrid(used, used, indexing="ij")
        r = delta * np.sqrt(MX ** 2 + MY ** 2)
        mask = UX & UY
    else:
        MZ, MY, MX = np.meshgrid(m, m, m, indexing="ij")
        UZ, UY, UX = np.meshgrid(used, used, used, indexing="ij")
        r = delta * np.sqrt(MX ** 2 + MY ** 2 + MZ ** 2)
        mask = UX & UY & UZ
    c = np.zeros(r.shape, dtype=np.complex128)
    nz = mask & (r > 0)
    c[nz] = k * k * delta ** dim * green(r[nz], kb, dim)
    c[(0,) * dim] = self_term(k, kb, delta, dim)
    return c


def green_spectrum(n: int, P: int, delta: float, k: float, kb: float, dim: int = 2) -> np.ndarray:
    """ghat = FFT_P(c): the spectrum that turns G into a pointwise product (Sec. III-A, FFT)."""
    return np.fft.fftn(circulant_column(n, P, delta, k, kb, dim))


def conv_G(x: np.ndarray, ghat: np.ndarray, n: int, adjoint: bool = False) -> np.ndarray:
    """G x (or G^H x) for x of shape [..., n, n(, n)]: pad, FFT, multiply, IFFT, crop.

    G^H = conj(G) because G is symmetric (g is even); its embedding spectrum
    is conj(ghat) since the circulant column is even.
    """
    dim = ghat.ndim
    P = ghat.shape[0]
    shp = x.shape[:-dim] + (P,) * dim
    pad = np.zeros(shp, dtype=np.complex128)
    sl = (Ellipsis,) + (slice(0, n),) * dim
    pad[sl] = x
    axes = tuple(range(-dim, 0))
    spec = np.conj(ghat) if adjoint else ghat
    out = np.fft.ifftn(spec * np.fft.fftn(pad, axes=axes), axes=axes)
    return out[sl]


def apply_A(f: np.ndarray, x: np.ndarray, ghat: np.ndarray) -> np.ndarray:
    """A x = x - G diag(f) x (Eq. 4)."""
    return x - conv_G(f * x, ghat, f.shape[0])


def apply_AH(f: np.ndarray, x: np.ndarray, ghat: np.ndarray) -> np.ndarray:
    """A^H x = x - diag(conj f) G^H x (adjoint of Eq. 4)."""
    return x - np.conj(f) * conv_G(x, ghat, f.shape[0], adjoint=True)


def sensing_matrix(rx: np.ndarray, n: int, delta: float, k: float, kb: float) -> np.ndarray:
    """H in C^{M x N} (Eq. 2): H_mn = k^2 delta^d g(|r_m - r_n|), receivers outside the grid."""
    dim = rx.shape[1]
    pts = grid_points(n, delta, dim)
    d = np.sqrt(((rx[:, None, :] - pts[None, :, :]) ** 2).sum(-1))
    return k * k * delta ** dim * green(d, kb, dim)


def plane_waves(angles: np.ndarray, n: int, delta: float, kb: float) -> np.ndarray:
    """[T, n, n] incident plane waves u_in,t(r) = exp(j kb (cos th_t x + sin th_t y))."""
    c = axis_centres(n, delta)
    Y, X = np.meshgrid(c, c, indexing="ij")
    th = np.asarray(angles)[:, None, None]
    return np.exp(1j * kb * (np.cos(th) * X[None] + np.sin(th) * Y[None]))


def plane_waves_3d(dirs: np.ndarray, n: int, delta: float, kb: float) -> np.ndarray:
    """[T, n, n, n] incident plane waves exp(j kb d_t . r) for unit directions d_t [T, 3]."""
    c = axis_centres(n, delta)
    Z, Y, X = np.meshgrid(c, c, c, indexing="ij")
    d = np.asarray(dirs, dtype=np.float64)
    ph = d[:, 0, None, None, None] * X[None] + d[:, 1, None, None, None] * Y[None] + d[:, 2, None, None, None] * Z[None]
    return np.exp(1j * kb * ph)


def point_sources(src: np.ndarray, n: int, delta: float, kb: float) -> np.ndarray:
    """[T, n, n(, n)] incident fields of point (3D) or line (2D) sources at src [T, d]:
    u_in,t(r) = g(|r - r_t|), Eq. 1's Green's function without the k^2 delta^d
    quadrature weight (the field radiated by a unit source)."""
    src = np.asarray(src, dtype=np.float64)
    dim = src.shape[1]
    pts = grid_points(n, delta, dim)
    d = np.sqrt(((src[:, None, :] - pts[None, :, :]) ** 2).sum(-1))
    return green(d, kb, dim).reshape((len(src),) + (n,) * dim)


class Problem:
    """Tables of one geometry: ghat (padded spectrum), H, incident fields.

    2D: ``angles`` are plane-wave angles; 3D (dim = 3): ``angles`` are unit
    propagation directions [T, 3] and receivers are [M, 3].  With
    tx_kind = "point", ``angles`` are source positions [T, d] instead."""

    def __init__(self, n: int, delta: float, angles, rx, wavelength: float = 1.0,
                 eps_b: float = 1.0, P: int | None = None, u_in=None, dim: int = 2, tx_kind: str = "plane"):
        self.n, self.delta, self.dim = n, delta, dim
        self.k, self.kb = wavenumbers(wavelength, eps_b)
        self.P = P if P is not None else 2 * n
        self.ghat = green_spectrum(n, self.P, delta, self.k, self.kb, dim)
        self.rx = np.asarray(rx, dtype=np.float64)
        self.H = sensing_matrix(self.rx, n, delta, self.k, self.kb)
        if u_in is None and tx_kind == "point":
            u_in = point_sources(np.asarray(angles), n, delta, self.kb)
        if u_in is None:
            if dim == 2:
                u_in = plane_waves(np.asarray(angles), n, delta, self.kb)
            else:
                u_in = plane_waves_3d(np.asarray(angles), n, delta, self.kb)
        self.u_in = np.asarray(u_in, dtype=np.complex128)
        self.T = self.u_in.shape[0]

    def A(self, f, x):
        return apply_A(f, x, self.ghat)

    def AH(self, f, x):
        return apply_AH(f, x, self.ghat)

    def sense(self, f, u):
        """Z = H diag(u) f for every transmitter: [T, M] (Eq. 5)."""
        return (f * u).reshape(u.shape[0], -1) @ self.H.T
