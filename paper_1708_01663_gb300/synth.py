"""Seeded synthetic inputs for the CISOR hot path.

This module is the only code shared between the FP64 oracle (``oracle/``) and
the CUDA path.  It draws random numbers and rasterises phantoms; it holds none
of the reconstruction method's arithmetic: no Green's function, no operator,
no solver, no forward model.  Everything here is an *input*: the permittivity
contrast image f, transmitter directions, receiver positions and unit complex
Gaussian noise draws that the caller scales.

Random numbers come from SplitMix64 (Steele, Lea and Flood, "Fast splittable
pseudorandom number generators", OOPSLA 2014): state advances by the golden
gamma 0x9E3779B97F4A7C15 and each output is the state passed through the
published 30/27/31 xor-shift-multiply finaliser.  Uniform doubles take the top
53 bits; normals come from the Box-Muller transform.  The generator is plain
integer arithmetic, so every machine produces the same inputs for a seed.

Lengths are in units of the vacuum wavelength (lambda = 1).  Images are stored
row-major with the x index fastest: ``f[iy, ix]`` (2D), ``f[iz, iy, ix]`` (3D).
"""
from __future__ import annotations

import math

import numpy as np

_GAMMA = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)


def splitmix64(seed: int, start: int, count: int) -> np.ndarray:
    """Outputs ``start .. start+count-1`` of the SplitMix64 stream for ``seed``."""
    with np.errstate(over="ignore"):
        idx = np.arange(start + 1, start + count + 1, dtype=np.uint64)
        z = np.uint64(seed & 0xFFFFFFFFFFFFFFFF) + idx * _GAMMA
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
        z = z ^ (z >> np.uint64(31))
    return z


class Rng:
    """Sequential reader of one SplitMix64 stream."""

    def __init__(self, seed: int):
        self.seed = int(seed)
        self.pos = 0

    def bits(self, count: int) -> np.ndarray:
        z = splitmix64(self.seed, self.pos, count)
        self.pos += count
        return z

    def uniform(self, lo: float = 0.0, hi: float = 1.0, count: int = 1) -> np.ndarray:
        u = (self.bits(count) >> np.uint64(11)).astype(np.float64) * (1.0 / 9007199254740992.0)
        return lo + (hi - lo) * u

    def normal(self, count: int) -> np.ndarray:
        m = (count + 1) // 2
        u1 = self.uniform(count=m)
        u2 = self.uniform(count=m)
        rad = np.sqrt(-2.0 * np.log1p(-u1))
        z = np.concatenate([rad * np.cos(2.0 * np.pi * u2), rad * np.sin(2.0 * np.pi * u2)])
        return z[:count]


def _centres(n: int) -> np.ndarray:
    """Pixel centres of an n-pixel axis, as fractions of the side, in (-0.5, 0.5)."""
    return (np.arange(n) + 0.5) / n - 0.5


def ellipse_phantom(n: int, count: int, contrast: tuple[float, float], seed: int,
                    imag: float = 0.0) -> np.ndarray:
    """n x n complex contrast image made of ``count`` seeded random ellipses.

    Centres are uniform in the inner 70% of the image, semi-axes uniform in
    [0.05, 0.25] x side, rotation uniform in [0, pi), real contrast uniform in
    ``contrast``; pixels whose centre lies inside take the value
    ``c + 1j*imag`` and later ellipses overwrite earlier ones.
    """
    rng = Rng(seed)
    c = _centres(n)
    X, Y = np.meshgrid(c, c, indexing="xy")
    f = np.zeros((n, n), dtype=np.complex128)
    for _ in range(count):
        cx, cy = rng.uniform(-0.35, 0.35, 2)
        a, b = rng.uniform(0.05, 0.25, 2)
        th = rng.uniform(0.0, math.pi, 1)[0]
        val = rng.uniform(contrast[0], contrast[1], 1)[0]
        dx, dy = X - cx, Y - cy
        xr = dx * math.cos(th) + dy * math.sin(th)
        yr = -dx * math.sin(th) + dy * math.cos(th)
        inside = (xr / a) ** 2 + (yr / b) ** 2 <= 1.0
        f[inside] = val + 1j * imag
    return f


def sphere_phantom(n: int, count: int, contrast: tuple[float, float], seed: int,
                   imag: float = 0.0) -> np.ndarray:
    """n^3 complex contrast volume of ``count`` seeded random spheres.

    Centres uniform in the inner 70% of the cube, radii uniform in
    [0.05, 0.2] x side, contrast uniform in ``contrast``.
    """
    rng = Rng(seed)
    c = _centres(n)
    Z, Y, X = np.meshgrid(c, c, c, indexing="ij")
    f = np.zeros((n, n, n), dtype=np.complex128)
    for _ in range(count):
        cx, cy, cz = rng.uniform(-0.35, 0.35, 3)
        rad = rng.uniform(0.05, 0.2, 1)[0]
        val = rng.uniform(contrast[0], contrast[1], 1)[0]
        inside = (X - cx) ** 2 + (Y - cy) ** 2 + (Z - cz) ** 2 <= rad * rad
        f[inside] = val + 1j * imag
    return f


def disk_phantom(n: int, delta: float, radius: float, contrast: complex) -> np.ndarray:
    """Centred homogeneous disk of the given physical radius (pixels whose centre is inside)."""
    x = (np.arange(n) - n / 2 + 0.5) * delta
    X, Y = np.meshgrid(x, x, indexing="xy")
    f = np.zeros((n, n), dtype=np.complex128)
    f[X * X + Y * Y <= radius * radius] = contrast
    return f


def plane_wave_angles(T: int) -> np.ndarray:
    """Propagation angles 2*pi*t/T of T plane waves in the x-y plane."""
    return 2.0 * np.pi * np.arange(T) / T


def circle_receivers(M: int, radius: float) -> np.ndarray:
    """[M, 2] receiver positions uniformly spaced on a circle."""
    phi = 2.0 * np.pi * np.arange(M) / M
    return np.stack([radius * np.cos(phi), radius * np.sin(phi)], axis=1)


def hemisphere_directions(rings=(11.25, 33.75, 56.25, 78.75), per_ring=12) -> np.ndarray:
    """[rings x per_ring, 3] unit propagation directions towards +z: polar angles
    ``rings`` (degrees from +z), azimuths spaced 360/per_ring, odd rings offset by
    half a step."""
    out = []
    for i, th in enumerate(np.radians(rings)):
        off = (np.pi / per_ring) if i % 2 else 0.0
        ph = off + 2.0 * np.pi * np.arange(per_ring) / per_ring
        out.append(np.stack([np.sin(th) * np.cos(ph), np.sin(th) * np.sin(ph), np.full(per_ring, np.cos(th))], 1))
    return np.concatenate(out)


def planar_receivers(side: int, pitch: float, z: float) -> np.ndarray:
    """[side^2, 3] receivers on a centred square grid in the plane z = const."""
    c = (np.arange(side) - (side - 1) / 2.0) * pitch
    Y, X = np.meshgrid(c, c, indexing="ij")
    return np.stack([X.ravel(), Y.ravel(), np.full(side * side, z)], axis=1)


def polarised_hemisphere(n_polar: int = 9, n_azimuth: int = 9) -> np.ndarray:
    """[n_polar x n_azimuth, 6] unit propagation directions over the upper
    hemisphere (polar angles (i + 0.5) 90 / n_polar degrees from +z, azimuths
    360 j / n_azimuth) with the polar unit vector theta^ as polarisation
    (orthogonal to the direction)."""
    out = []
    for i in range(n_polar):
        th = np.radians((i + 0.5) * 90.0 / n_polar)
        for j in range(n_azimuth):
            ph = 2.0 * np.pi * j / n_azimuth
            d = [np.sin(th) * np.cos(ph), np.sin(th) * np.sin(ph), np.cos(th)]
            p = [np.cos(th) * np.cos(ph), np.cos(th) * np.sin(ph), -np.sin(th)]
            out.append(d + p)
    return np.array(out)


def circle_sources(T: int, radius: float, offset: float = 0.0) -> np.ndarray:
    """[T, 2] source positions uniformly spaced on a circle, starting at angle ``offset``."""
    phi = offset + 2.0 * np.pi * np.arange(T) / T
    return np.stack([radius * np.cos(phi), radius * np.sin(phi)], axis=1)


def angular_mask(src: np.ndarray, rx: np.ndarray, min_deg: float) -> np.ndarray:
    """[T, M] 0/1 mask: receiver m is active for source t when their directions
    from the origin differ by more than ``min_deg`` degrees."""
    a = np.arctan2(src[:, 1], src[:, 0])[:, None]
    b = np.arctan2(rx[:, 1], rx[:, 0])[None, :]
    d = np.abs((b - a + np.pi) % (2.0 * np.pi) - np.pi)
    return (d > np.radians(min_deg)).astype(np.uint8)


def complex_noise(seed: int, shape) -> np.ndarray:
    """Unit-variance circular complex Gaussian draws (a + ib)/sqrt(2)."""
    cnt = int(np.prod(shape))
    rng = Rng(seed)
    z = rng.normal(2 * cnt)
    return ((z[:cnt] + 1j * z[cnt:]) / math.sqrt(2.0)).reshape(shape)


def random_field(seed: int, shape) -> np.ndarray:
    """Complex vector with i.i.d. standard normal real and imaginary parts."""
    cnt = int(np.prod(shape))
    z = Rng(seed).normal(2 * cnt)
    return (z[:cnt] + 1j * z[cnt:]).reshape(shape)


# Workloads.  Lengths in wavelengths.  Seeds are 1708 + workload index.
CONFIGS = {
    # 2D plain CISOR: 64x64 at lambda/8 (FFT padded to 128x128), 3 ellipses with
    # real contrast in [0, 0.2], 8 plane waves, 32 receivers on r = 6 lambda,
    # 40 dB SNR, 20 outer iterations, TV weight 1e-3.
    "c1": dict(dim=2, n=64, delta=1.0 / 8, T=8, M=32, rx_radius=6.0, shapes=3,
               contrast=(0.0, 0.2), imag=0.0, snr_db=40.0, outer=20, tau=1e-3,
               tv_iters=20, alpha=0.96, seed=1709),
    # 2D high contrast: 256x256 at lambda/8 (512x512 padded), 64 transmitters,
    # 256 receivers on r = 24 lambda, 10 ellipses with contrast up to 1.0 plus
    # 0.05i absorption inside the ellipses, 100 outer iterations, tol 1e-4.
    "c2": dict(dim=2, n=256, delta=1.0 / 8, T=64, M=256, rx_radius=24.0, shapes=10,
               contrast=(0.0, 1.0), imag=0.05, snr_db=40.0, outer=100, tau=1e-3,
               tv_iters=20, alpha=0.96, seed=1710),
    # 3D scalar: 64^3 voxels at lambda/6 (FFT 128^3), 5 spheres with contrast
    # in [0, 0.3], 48 plane waves over the upper hemisphere (4 polar rings x 12
    # azimuths), 32 x 32 receivers at lambda/2 pitch in the plane z = 8 lambda.
    "c3": dict(dim=3, n=64, delta=1.0 / 6, T=48, M=1024, rx_plane=8.0, shapes=5,
               contrast=(0.0, 0.3), imag=0.0, snr_db=40.0, outer=50, tau=1e-3,
               tv_iters=20, alpha=0.96, seed=1711),
    # 2D Fresnel-style: the sizes of the 2D experimental set-up of Sec. IV at
    # 3 GHz (lambda = 100 mm): a 150 mm domain on 128 x 128 pixels (delta =
    # 1.5 lambda / 128), 8 line sources on a circle of 7.2 lambda, 360
    # receivers on a circle of 7.6 lambda, each source recording the receivers
    # more than 60 degrees away from it (240 of 360); 3 seeded ellipses with
    # real contrast up to 1.0 stand in for the measured objects.
    "c6": dict(dim=2, n=128, delta=1.5 / 128, T=8, M=360, rx_radius=7.6, tx_radius=7.2, tx_kind="point",
               rx_min_deg=60.0, shapes=3, contrast=(0.0, 1.0), imag=0.0, snr_db=40.0, outer=100, tau=1e-3,
               tv_iters=20, alpha=0.96, seed=1714),
    # 3D vectorial (appendix): the sizes of the 3D experimental set-up of Sec.
    # IV at 4 GHz (lambda = 75 mm): a 150 mm cube on 32^3 voxels (delta =
    # lambda / 16), 81 polarised plane waves over the upper hemisphere (9
    # polar x 9 azimuth, theta-polarised), 36 receivers on a circle of 20
    # lambda in the azimuth plane measuring E_z, each transmitter recording the
    # receivers more than 50 degrees from its azimuth; 2 seeded spheres with
    # contrast up to 1.5 stand in for the measured objects.
    "c7": dict(dim=3, vectorial=True, n=32, delta=1.0 / 16, T=81, M=36, rx_radius=20.0, rx_min_deg=50.0,
               shapes=2, contrast=(0.5, 1.5), imag=0.0, snr_db=40.0, outer=50, tau=1e-3, tv_iters=20,
               alpha=0.96, seed=1715),
}


def make_inputs(name: str, T: int | None = None):
    """Phantom, transmitters (2D: angles; 3D: unit directions [T, 3]) and receivers of a named workload."""
    cfg = dict(CONFIGS[name])
    if T is not None:
        cfg["T"] = T
    if cfg.get("vectorial"):
        f = sphere_phantom(cfg["n"], cfg["shapes"], cfg["contrast"], cfg["seed"], cfg["imag"])
        tx = polarised_hemisphere()[: cfg["T"]]
        rx3 = circle_receivers(cfg["M"], cfg["rx_radius"])
        rx = np.concatenate([rx3, np.zeros((cfg["M"], 1))], axis=1)
        cfg["rx_mask"] = angular_mask(tx[:, :2], rx3, cfg["rx_min_deg"])
        return cfg, f, tx, rx
    if cfg["dim"] == 3:
        f = sphere_phantom(cfg["n"], cfg["shapes"], cfg["contrast"], cfg["seed"], cfg["imag"])
        tx = hemisphere_directions()[: cfg["T"]]
        rx = planar_receivers(32, 0.5, cfg["rx_plane"])
        return cfg, f, tx, rx
    if cfg.get("tx_kind") == "point":
        f = ellipse_phantom(cfg["n"], cfg["shapes"], cfg["contrast"], cfg["seed"], cfg["imag"])
        src = circle_sources(CONFIGS[name]["T"], cfg["tx_radius"])[: cfg["T"]]
        rx = circle_receivers(cfg["M"], cfg["rx_radius"])
        cfg["rx_mask"] = angular_mask(src, rx, cfg["rx_min_deg"])
        return cfg, f, src, rx
    f = ellipse_phantom(cfg["n"], cfg["shapes"], cfg["contrast"], cfg["seed"], cfg["imag"])
    angles = plane_wave_angles(CONFIGS[name]["T"])[: cfg["T"]]
    rx = circle_receivers(cfg["M"], cfg["rx_radius"])
    return cfg, f, angles, rx
