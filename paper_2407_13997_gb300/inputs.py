"""Seeded synthetic workloads (shared by the tests, the bench and smoke).

This module holds no arithmetic of the method: it only names the problem
parameters and draws the random amplitudes of the divergence-free Fourier
forcing, which both the CUDA path and the oracle then evaluate themselves.

Fourier forcing: stream-function modes psi_j = sin(mx_j pi x) sin(my_j pi y),
f = sum_j amp_j (d_y psi_j, -d_x psi_j), using the 8 lowest mode pairs ordered
by (mx^2 + my^2, mx), amp_j = z_j / (mx_j^2 + my_j^2) with z_j ~ N(0, 1) from
numpy.random.default_rng(seed) (amplitudes decaying as |k|^-2).
"""
from dataclasses import dataclass, field

import numpy as np

KIND_TAYLOR_GREEN = 0
KIND_POLY = 1
KIND_FOURIER = 2
KIND_LID = 3
KIND_HEAT = 4          # heat equation, u(0) = sin(pi x) + cos(2 pi y)
KIND_HEAT_EIGEN = 5    # heat equation, u(0) = cos(pi x)
KIND_NAMES = {KIND_TAYLOR_GREEN: "taylor_green", KIND_POLY: "poly", KIND_FOURIER: "fourier", KIND_LID: "lid"}

FOURIER_MODES = ((1, 1), (1, 2), (2, 1), (2, 2), (1, 3), (3, 1), (2, 3), (3, 2))


def fourier_forcing(seed, n_modes=8):
    """(mx, my, amp) arrays of the seeded divergence-free Fourier forcing."""
    rng = np.random.default_rng(seed)
    z = rng.standard_normal(n_modes)
    mx = np.array([m for m, _ in FOURIER_MODES[:n_modes]], dtype=np.int32)
    my = np.array([n for _, n in FOURIER_MODES[:n_modes]], dtype=np.int32)
    amp = z / (mx.astype(np.float64) ** 2 + my.astype(np.float64) ** 2)
    return mx, my, amp


@dataclass
class Workload:
    """One space-time solve: mesh n_fine -> n_coarse, Q_{k+1}^2/Q_k, DG(q), N slabs."""

    name: str
    n_fine: int
    n_coarse: int
    k: int
    q: int
    N: int
    T: float
    nu: float
    conv: float
    kind: int
    steady: bool = False
    mx: np.ndarray = field(default_factory=lambda: np.zeros(0, dtype=np.int32))
    my: np.ndarray = field(default_factory=lambda: np.zeros(0, dtype=np.int32))
    amp: np.ndarray = field(default_factory=lambda: np.zeros(0))
    t0: float = 0.0  # time at the start of slab 0

    def ndofs(self, n=None):
        n = self.n_fine if n is None else n
        if self.kind in (KIND_HEAT, KIND_HEAT_EIGEN):  # one scalar Q_k field
            return self.N * (self.q + 1) * (n * self.k + 1) ** 2
        nv = n * (self.k + 1) + 1
        np_ = n * self.k + 1
        return self.N * (self.q + 1) * (2 * nv * nv + np_ * np_)


def taylor_green_8x8():
    """Plain FP64 parity workload: 8x8 Q2/Q1, DG(0), 8 slabs on [0, 1], nu = 1e-2,
    decaying Taylor-Green data, coarsened to 2x2."""
    return Workload("tg_q2q1_dg0_n8_N8", 8, 2, 1, 0, 8, 1.0, 1e-2, 1.0, KIND_TAYLOR_GREEN)


def chorin(n=16, k=1, q=0, N=10, R=10.0):
    """The Chorin (Taylor-Green) test problem of Sec. 4 in its Reynolds-number form:
    nu = 1, convection R, t in [0, 0.1], exact velocity data on the whole boundary,
    n x n mesh coarsened to 2 x 2, N slabs."""
    return Workload(f"chorin_R{R:g}_q{k + 1}q{k}_dg{q}_n{n}_N{N}", n, 2, k, q, N, 0.1, 1.0, R, KIND_TAYLOR_GREEN)


def lid_cavity(n=16, k=1, q=0, N=20, R=10.0, T=0.02):
    """The lid-driven cavity of Sec. 4 in Reynolds-number form (nu = 1, convection
    R), started from rest, t in [0, T], n x n mesh coarsened to 2 x 2, N slabs."""
    return Workload(f"lid_R{R:g}_q{k + 1}q{k}_dg{q}_n{n}_N{N}", n, 2, k, q, N, T, 1.0, R, KIND_LID)


def heat(n=16, k=1, q=0, N=20, nu=1.0, T=0.02, eigen=False, n_coarse=None):
    """The heat equation of Sec. 5: u_t - nu lap u = 0, natural boundary conditions,
    u(0) = sin(pi x) + cos(2 pi y) (eigen: cos(pi x)), t in [0, T], Q_k x DG(q) (k = 1..3,
    q = 0..3), N slabs, n x n mesh coarsened to 2 x 2 (1 x 1 for k = q = 3, whose 2 x 2
    coarse block is too large for the GPU's direct solve)."""
    if n_coarse is None:
        n_coarse = 1 if (k == 3 and q == 3) else 2
    return Workload(f"heat_q{k}_dg{q}_n{n}_N{N}", n, n_coarse, k, q, N, T, nu, 0.0,
                    KIND_HEAT_EIGEN if eigen else KIND_HEAT)


def fourier_64x64_q3q2_dg1(seed=0):
    """64x64 Q3/Q2, DG(1), 64 slabs on [0, 1], nu = 1e-3, seeded Fourier forcing,
    no-slip walls, u(0) = 0, coarsened to 2x2 (11,665,792 space-time DoFs)."""
    mx, my, amp = fourier_forcing(seed)
    return Workload("fourier_q3q2_dg1_n64_N64", 64, 2, 2, 1, 64, 1.0, 1e-3, 1.0,
                    KIND_FOURIER, False, mx, my, amp)


def fourier_128x128_q2q1_dg0(seed=0):
    """128x128 Q2/Q1, DG(0), 128 slabs, nu = 1e-3, seeded Fourier forcing."""
    mx, my, amp = fourier_forcing(seed)
    return Workload("fourier_q2q1_dg0_n128_N128", 128, 2, 1, 0, 128, 1.0, 1e-3, 1.0,
                    KIND_FOURIER, False, mx, my, amp)


def fourier_small(n=8, k=1, q=0, N=4, nu=1e-2, seed=0, T=1.0, n_coarse=2):
    mx, my, amp = fourier_forcing(seed)
    return Workload(f"fourier_k{k}_q{q}_n{n}_N{N}", n, n_coarse, k, q, N, T, nu, 1.0,
                    KIND_FOURIER, False, mx, my, amp)


def poly_small(n=4, k=1, q=1, N=3, nu=0.1, steady=False, n_coarse=2):
    return Workload(f"poly_k{k}_q{q}_n{n}_N{N}", n, n_coarse, k, q, N, 1.0, nu, 1.0,
                    KIND_POLY, steady)


def seeded_vector(seed, size, scale=1.0):
    """A reproducible N(0, scale^2) test vector."""
    return scale * np.random.default_rng(seed).standard_normal(size)


def forcing_shaped_iterate(w, scale=1.0):
    """A synthetic linearisation point with the structure of a forced flow: the
    divergence-free field sum_j amp_j curl(psi_j) of the workload's Fourier modes
    at the velocity nodes, normalised to max |u| = scale, zero on the walls and at
    every temporal DoF, zero pressure (canonical layout)."""
    nv = w.n_fine * (w.k + 1) + 1
    np_ = w.n_fine * w.k + 1
    x = np.linspace(0.0, 1.0, nv)
    X, Y = np.meshgrid(x, x, indexing="xy")
    ux = np.zeros_like(X)
    uy = np.zeros_like(X)
    for m, n, a in zip(w.mx, w.my, w.amp):
        ux += a * n * np.pi * np.sin(m * np.pi * X) * np.cos(n * np.pi * Y)
        uy -= a * m * np.pi * np.cos(m * np.pi * X) * np.sin(n * np.pi * Y)
    wall = np.zeros_like(X, dtype=bool)
    wall[0, :] = wall[-1, :] = wall[:, 0] = wall[:, -1] = True
    ux[wall] = 0.0
    uy[wall] = 0.0
    mag = max(np.abs(ux).max(), np.abs(uy).max(), 1e-300)
    blk = np.concatenate([ux.ravel(), uy.ravel(), np.zeros(np_ * np_)]) * (scale / mag)
    return np.tile(blk, w.N * (w.q + 1))


def batching_workloads(count=256, seed=1):
    """Independent Q2/Q1 DG(0) solves with uneven sizes: n uniform in {8, 16, 24, 32, 48}
    (24 and 48 coarsen to 3x3), N uniform in {8, 16, 32, 64}, nu log-uniform in
    [1e-3, 1e-1], each with its own Fourier forcing seed (1000 * seed + i)."""
    rng = np.random.default_rng(seed)
    ns = rng.choice([8, 16, 24, 32, 48], size=count)
    Ns = rng.choice([8, 16, 32, 64], size=count)
    nus = 10.0 ** rng.uniform(-3.0, -1.0, size=count)
    out = []
    for i in range(count):
        n = int(ns[i])
        mx, my, amp = fourier_forcing(1000 * seed + i)
        out.append(Workload(f"batch{seed}_{i}_n{n}_N{int(Ns[i])}", n, 3 if n % 3 == 0 else 2, 1, 0, int(Ns[i]),
                            1.0, float(nus[i]), 1.0, KIND_FOURIER, False, mx, my, amp))
    return out


def serving_workloads(count=32, seed=2, ns=(16, 32, 64), slabs=(16, 32, 64)):
    """Space-time solve requests of the serving stream: Q2/Q1 DG(0) or Q3/Q2 DG(1)
    with equal probability, n uniform in `ns`, N uniform in `slabs`, nu log-uniform
    in [1e-3, 1e-1], Fourier forcing seeded 5000 * seed + i, coarsened to 2x2."""
    rng = np.random.default_rng(seed)
    kinds = rng.integers(0, 2, size=count)
    ns_ = rng.choice(list(ns), size=count)
    Ns = rng.choice(list(slabs), size=count)
    nus = 10.0 ** rng.uniform(-3.0, -1.0, size=count)
    out = []
    for i in range(count):
        k, q = (1, 0) if kinds[i] == 0 else (2, 1)
        n, N = int(ns_[i]), int(Ns[i])
        mx, my, amp = fourier_forcing(5000 * seed + i)
        out.append(Workload(f"serve{seed}_{i}_q{k + 1}q{k}_dg{q}_n{n}_N{N}", n, 2, k, q, N, 1.0, float(nus[i]), 1.0,
                            KIND_FOURIER, False, mx, my, amp))
    return out


def poisson_arrivals(count, rate, seed=2):
    """Arrival times (s) of a Poisson stream of `rate` requests per second."""
    rng = np.random.default_rng(seed)
    return np.cumsum(rng.exponential(1.0 / rate, size=count))
