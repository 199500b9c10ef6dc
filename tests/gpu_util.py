"""Shared set-up of the GPU parity tests: a context, the oracle problem and seeded inputs."""
import numpy as np

from oracle import model
from paper_1708_01663_gb300 import build, cisor, synth


def c64(a):
    return np.ascontiguousarray(a, dtype=np.complex64)


def rel(a, b):
    return float(np.linalg.norm(np.asarray(a) - np.asarray(b)) / np.linalg.norm(np.asarray(b)))


def make(n, T, M, rx_radius, delta=1.0 / 8, pad=0, complex_f=False):
    build.build()
    angles = synth.plane_wave_angles(T)
    rx = synth.circle_receivers(M, rx_radius)
    ctx = cisor.Cisor(n, delta, angles, rx, complex_f=complex_f, pad=pad)
    prob = model.Problem(n, delta, angles, rx, P=ctx.P)
    return ctx, prob
