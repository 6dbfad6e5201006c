"""Seeded synthetic inputs shared by the tests, the benchmark and the oracle checks.

This module only draws random numbers and lays out the workloads (sizes, sources,
wavenumber fields, request streams); it holds none of the solver's arithmetic.  The
paper's benchmarks are analytic (Sec. 5): a unit point source in a constant-k square
(Benchmark 1) and smooth wavenumber fields (Benchmark 3); the larger workloads below
keep those shapes and add seeded random sources and a seeded 3D bump field.

Arrays use the natural layout: shape ``(n,)*dim``, x fastest (C order).
"""
from __future__ import annotations

from dataclasses import dataclass
from typing import List, Optional

import numpy as np

THETA_GAMMA = 0.5   # ECS layer angle (rad) of every workload
ECS_FRAC = 0.125    # layer width: last 1/8 of the domain on each side


def rng(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(seed))


def point_source(dim: int, n: int) -> np.ndarray:
    """Unit point source at the centre node (1-based index (n+1)/2 per axis)."""
    b = np.zeros((n,) * dim, dtype=np.complex128)
    c = (n + 1) // 2 - 1
    b[(c,) * dim] = 1.0
    return b


def random_source(dim: int, n: int, seed: int) -> np.ndarray:
    """I.i.d. complex normal source with E|b_p|^2 = 1 (real and imaginary parts
    N(0, 1/2)) at every unknown, layers included."""
    g = rng(seed)
    re = g.standard_normal((n,) * dim)
    im = g.standard_normal((n,) * dim)
    return ((re + 1j * im) * np.sqrt(0.5)).astype(np.complex128)


def bump_field(n: int, seed: int, k0: float = 80.0, amp: float = 0.3, nbumps: int = 8,
               sigma: float = 0.1) -> np.ndarray:
    """phi = k(x)^2 with k(x) = k0 (1 + amp g(x)), g a clipped sum of Gaussian bumps.

    Centres ~ U[0,1]^3, amplitudes ~ U[-1,1], g = sum a exp(-|x-c|^2 / (2 sigma^2))
    clipped to [-1, 1]; evaluated at the real node coordinates x_i = i/(n+1),
    i = 1..n.  Returned as float32 (the library takes an FP32 phi field).
    """
    g = rng(seed)
    centres = g.uniform(0.0, 1.0, size=(nbumps, 3))
    amps = g.uniform(-1.0, 1.0, size=nbumps)
    x = np.arange(1, n + 1) / (n + 1)
    field = np.zeros((n, n, n), dtype=np.float64)
    for c, a in zip(centres, amps):
        gz = np.exp(-((x - c[2]) ** 2) / (2 * sigma ** 2))
        gy = np.exp(-((x - c[1]) ** 2) / (2 * sigma ** 2))
        gx = np.exp(-((x - c[0]) ** 2) / (2 * sigma ** 2))
        field += a * gz[:, None, None] * gy[None, :, None] * gx[None, None, :]
    gfield = np.clip(field, -1.0, 1.0)
    k = k0 * (1.0 + amp * gfield)
    return (k * k).astype(np.float32)


@dataclass
class Workload:
    """One solve: grid, wavenumber, source, CSG angle and tolerances."""
    dim: int
    n: int
    theta_beta: float
    k: Optional[float] = None           # constant wavenumber (phi = k^2)
    phi: Optional[np.ndarray] = None    # float32 field, shape (n,)*dim
    b: Optional[np.ndarray] = None      # complex128 source, shape (n,)*dim
    tol: float = 1e-6
    restart: int = 0                    # 0 = no restart
    precision: str = "c64"              # preconditioner precision
    theta_gamma: float = THETA_GAMMA
    ecs_frac: float = ECS_FRAC
    ecs_sides: str = "both"             # "high": layers at the far end of each axis only


def small_2d(seed: int = 1000) -> Workload:
    """2D, 127^2 interior, k = 20, point source, theta_beta = 0.4, complex128
    throughout, tolerance 1e-8 (the latency-bound small case)."""
    return Workload(dim=2, n=127, theta_beta=0.4, k=20.0, b=point_source(2, 127), tol=1e-8,
                    precision="c128")


def large_2d(theta_beta: float = 0.3, seed: int = 1001) -> Workload:
    """2D, 1023^2 interior, k = 160 (kh ~ 0.16), unit-variance complex normal source,
    complex64 preconditioner, FP64 outer solve to 1e-6."""
    return Workload(dim=2, n=1023, theta_beta=theta_beta, k=160.0, b=random_source(2, 1023, seed),
                    tol=1e-6, precision="c64")


LARGE_2D_BETAS = (0.1, 0.2, 0.3, 0.5)


def cube_3d(n: int = 255, seed: int = 1002) -> Workload:
    """3D unit cube, n^3 interior, phi = (80 (1 + 0.3 g))^2 with 8 seeded bumps,
    point source at the centre, theta_beta = 0.4, restart 40, tolerance 1e-6."""
    return Workload(dim=3, n=n, theta_beta=0.4, phi=bump_field(n, seed), b=point_source(3, n),
                    tol=1e-6, restart=40, precision="c64")


GAUSS_DOMAIN = 50.0                       # physical box (0, 50)^2 of the Gaussian model
GAUSS_THETA_BETA = float(np.radians(10.3132))  # CSG angle of every Sec. 5 benchmark
GAUSS_THETA_GAMMA = float(np.pi / 6)      # ECS angle of Sec. 4 and 5


def gaussian_model(nint: int, k: float, nu: float) -> Workload:
    """Benchmark 3 of Sec. 5 (the Gaussian model) on the unit box.

    The physical problem lives on (0, 50)^2 with phi = nu (e^{-x^2} + e^{-y^2}) + k^2
    and the source chi = 1 / (e^{x^2} + e^{y^2}), homogeneous Dirichlet on the south and
    west edges (x = 0, y = 0) and ECS layers beyond the north and east edges.  Readings
    (the paper leaves them open): ``nint`` intervals across (0, 50) per axis (the
    table's "interior grid"), followed by a layer of nint/4 intervals (the layer width
    of Sec. 4.4), theta_beta = 10.3132 degrees, theta_gamma = pi/6, relative residual
    1e-7.  So a grid of n = 1.25 nint - 1 unknowns per axis covers a box of length
    Lam = 50 (n + 1) / nint, the last fifth of it the layer.

    Mapped to the unit box (x = Lam xi) the operator -Delta_x - phi becomes
    (-Delta_xi - Lam^2 phi) / Lam^2; the returned problem is Lam^2 times the physical one
    (phi and b both scaled by Lam^2), which has the same solution, the same relative
    residuals and the same preconditioned iterations.  phi is float32 (the library's
    field precision); b is complex128 and vanishes to rounding inside the layer.  The
    preconditioner precision is the library's automatic choice (complex128 on the 64^2
    column's 79^2 grid, complex64 on the larger ones).
    """
    if nint % 4:
        raise ValueError("nint must be a multiple of 4 (the layer has nint/4 intervals)")
    n = nint + nint // 4 - 1
    lam = GAUSS_DOMAIN * (n + 1) / nint
    x = np.arange(1, n + 1) * (lam / (n + 1))
    ex = np.exp(-x * x)
    phi = lam * lam * (nu * (ex[None, :] + ex[:, None]) + k * k)
    # 1 / (e^{x^2} + e^{y^2}) without overflow: divide through by the larger exponential
    sx, sy = (x * x)[None, :], (x * x)[:, None]
    m = np.maximum(sx, sy)
    chi = np.exp(-m) / (np.exp(sx - m) + np.exp(sy - m))
    return Workload(dim=2, n=n, theta_beta=GAUSS_THETA_BETA, phi=phi.astype(np.float32),
                    b=(lam * lam * chi).astype(np.complex128), tol=1e-7, restart=0, precision="auto",
                    theta_gamma=GAUSS_THETA_GAMMA, ecs_frac=(nint // 4) / (n + 1), ecs_sides="high")


GAUSS_COLUMNS = ((0.5, 64), (1.5, 128), (2.5, 256), (3.5, 512), (4.5, 512))  # (k, nint) of Tables 4-5


def batch_2d(count: int = 64, seed: int = 1003, sizes=(255, 511, 1023), theta_beta: float = 0.3
             ) -> List[Workload]:
    """Independent 2D problems: n ~ U(sizes), kh ~ U[0.1, 0.3] so k = kh (n+1),
    theta_beta = 0.3, random sources, restart 40, tolerance 1e-6."""
    g = rng(seed)
    out = []
    for i in range(count):
        n = int(g.choice(sizes))
        kh = float(g.uniform(0.1, 0.3))
        out.append(Workload(dim=2, n=n, theta_beta=theta_beta, k=kh * (n + 1),
                            b=random_source(2, n, seed * 1000 + i), tol=1e-6, restart=40))
    return out


@dataclass
class Request:
    arrival: float      # seconds since stream start
    work: Workload


def request_stream(count: int = 2000, rate: float = 200.0, seed: int = 1004,
                   shapes=((2, 127), (2, 511), (2, 1023), (3, 127), (3, 255))) -> List[Request]:
    """Poisson arrivals (mean ``rate`` per second), shapes uniform over ``shapes``,
    kh ~ U[0.1, 0.3], random sources drawn lazily per request (seeded by index),
    theta_beta = 0.3, restart 40, tolerance 1e-6."""
    g = rng(seed)
    t = np.cumsum(g.exponential(1.0 / rate, size=count))
    out = []
    for i in range(count):
        dim, n = shapes[int(g.integers(len(shapes)))]
        kh = float(g.uniform(0.1, 0.3))
        out.append(Request(arrival=float(t[i]),
                           work=Workload(dim=dim, n=n, theta_beta=0.3, k=kh * (n + 1), b=None,
                                         tol=1e-6, restart=40)))
    return out


def request_source(req_index: int, dim: int, n: int, seed: int = 1004) -> np.ndarray:
    return random_source(dim, n, seed * 100000 + req_index)
