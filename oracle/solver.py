"""Newton-FGMRES-waveform-relaxation-multigrid (oracle; test infrastructure only).

* Hierarchy (Sec. 3): spatial meshes n_fine, n_fine/2, ..., n_coarse with the
  same time mesh on every level (semi-coarsening).  Coarse operators are
  rediscretised about the injected iterate.
* V(2,2) cycle (Algorithm Vcycle): pre-relax, residual, restrict with zero
  coarse guess, ..., direct coarse solve, interpolate-and-add, post-relax.
* Relaxation: 2 steps of Chebyshev iteration preconditioned by the waveform
  Vanka+star smoother, on [0.25 lam, 1.05 lam] where lam is the largest real
  part of the Ritz values from 10 Arnoldi steps on M^{-1} J (Sec. 3, Chebyshev
  weights).  The Chebyshev recurrence is Saad's preconditioned Chebyshev
  iteration (Iterative Methods for Sparse Linear Systems, Alg. 12.1).
  The Arnoldi start vector is uniform(-1, 1) on the free DoFs drawn from the
  counter-based splitmix64 generator (seed = level index), value i =
  mix(seed + (i+1) * 0x9E3779B97F4A7C15).
* Coarse solve: J is block lower bidiagonal in slabs, so the direct solve is a
  forward substitution over slabs with a dense LU of every diagonal slab block
  on the free DoFs; the pressure DoF at vertex (0, 0) of every temporal DoF is
  pinned (row and column replaced by the identity, right-hand side 0) and the
  result is made mean-free.
* FGMRES (Sec. 3): restart 30, modified Gram-Schmidt, Givens rotations, zero
  initial guess, right preconditioner = one V-cycle whose output is made
  pressure-mean-free, stop when the residual norm <= tol.
* Inexact Newton (Sec. 5, Chorin experiments): stop when ||F_k|| <= rtol ||F_0||
  (rtol 1e-8), full steps; forcing terms by Eisenstat-Walker choice 2 with
  gamma 0.9, alpha 2, eta_0 0.5, eta_max 0.9, the gamma eta_{k-1}^alpha > 0.1
  safeguard and the oversolving floor eta_k >= 0.5 rtol ||F_0|| / ||F_k||
  (Kelley, Iterative Methods for Linear and Nonlinear Equations, Sec. 6.3);
  or a fixed eta.

Parity unpinned by the paper (fixed by convention only): the EW constants, the
Arnoldi start vector and the FGMRES restart length.
"""
import dataclasses

import numpy as np
import scipy.linalg as sla

from .fem import Discretisation
from .patches import PatchSmoother
from .transfer import injection, prolongation

_GOLDEN = np.uint64(0x9E3779B97F4A7C15)


def splitmix64_raw(seed, count):
    """Outputs 1..count of splitmix64 started from state ``seed``:
    value i = mix(seed + i * 0x9E3779B97F4A7C15) (Steele, Lea & Flood, 2014)."""
    with np.errstate(over="ignore"):
        i = np.arange(1, count + 1, dtype=np.uint64)
        z = np.uint64(seed) + i * _GOLDEN
        z = (z ^ (z >> np.uint64(30))) * np.uint64(0xBF58476D1CE4E5B9)
        z = (z ^ (z >> np.uint64(27))) * np.uint64(0x94D049BB133111EB)
        return z ^ (z >> np.uint64(31))


def splitmix64_uniform(seed, count):
    """uniform(-1, 1) values from the top 53 bits of the splitmix64 stream."""
    z = splitmix64_raw(seed, count)
    u = (z >> np.uint64(11)).astype(np.float64) * (1.0 / 9007199254740992.0)
    return 2.0 * u - 1.0


class Options:
    def __init__(self, cheb_steps=2, cheb_lo=0.25, cheb_hi=1.05, eig_steps=10,
                 newton_rtol=1e-8, newton_maxit=20, ew=True, eta_fixed=1e-4,
                 restart=30, gmres_maxit=200, newton_divtol=1e6, newton_stall=3):
        self.cheb_steps, self.cheb_lo, self.cheb_hi = cheb_steps, cheb_lo, cheb_hi
        self.eig_steps = eig_steps
        self.newton_rtol, self.newton_maxit = newton_rtol, newton_maxit
        self.ew, self.eta_fixed = ew, eta_fixed
        self.restart, self.gmres_maxit = restart, gmres_maxit
        # give up on divergence (||F|| > divtol ||F_0||) or after `stall` consecutive
        # Newton steps whose FGMRES used all its iterations (0 switches either off)
        self.newton_divtol, self.newton_stall = newton_divtol, newton_stall


class CoarseSolver:
    """Exact solve with the coarsest level's block lower bidiagonal J."""

    def __init__(self, disc, J):
        self.disc, self.J = disc, J
        free = ~disc.spatial_dirichlet()
        self.sfree = np.nonzero(free)[0]
        pin = disc.pres_index(0, 0)
        self.idx, self.lu, self.sub, self.pins = [], [], [], []
        for n in range(disc.N):
            ix = np.concatenate([disc.block(n, a) + self.sfree for a in range(disc.nt)])
            A = J[ix][:, ix].toarray()
            pins = [int(np.nonzero(ix == disc.block(n, a) + pin)[0][0]) for a in range(disc.nt)]
            for p in pins:
                A[p, :] = 0.0
                A[:, p] = 0.0
                A[p, p] = 1.0
            self.idx.append(ix)
            self.pins.append(pins)
            self.lu.append(sla.lu_factor(A, check_finite=False))
            self.sub.append(J[ix][:, self.idx[n - 1]].toarray() if n > 0 else None)

    def solve(self, b):
        out = np.zeros_like(b)
        prev = None
        for n in range(self.disc.N):
            rhs = b[self.idx[n]].copy()
            if n > 0:
                rhs -= self.sub[n] @ prev
            for p in self.pins[n]:
                rhs[p] = 0.0
            prev = sla.lu_solve(self.lu[n], rhs, check_finite=False)
            out[self.idx[n]] = prev
        return self.disc.project_pressure(out)


def chebyshev(Jop, Mop, b, x0, lam, opts):
    """``opts.cheb_steps`` steps of preconditioned Chebyshev iteration on
    [cheb_lo lam, cheb_hi lam] (Saad Alg. 12.1); x0 = None means a zero guess."""
    a, bb = opts.cheb_lo * lam, opts.cheb_hi * lam
    theta, delta = 0.5 * (bb + a), 0.5 * (bb - a)
    sigma = theta / delta
    if x0 is None:
        x = np.zeros_like(b)
        r = b.copy()
    else:
        x = x0.copy()
        r = b - Jop(x)
    rho = 1.0 / sigma
    d = Mop(r) / theta
    for step in range(opts.cheb_steps):
        x = x + d
        if step == opts.cheb_steps - 1:
            break
        r = b - Jop(x)
        z = Mop(r)
        rho_new = 1.0 / (2.0 * sigma - rho)
        d = rho_new * rho * d + (2.0 * rho_new / delta) * z
        rho = rho_new
    return x


def arnoldi_ritz_max(Aop, v0, steps):
    """Largest real part of the Ritz values of ``steps`` Arnoldi steps (MGS) on Aop from v0."""
    V = [v0 / np.linalg.norm(v0)]
    H = np.zeros((steps + 1, steps))
    m = steps
    for j in range(steps):
        w = Aop(V[j])
        for i in range(j + 1):
            H[i, j] = np.dot(w, V[i])
            w = w - H[i, j] * V[i]
        H[j + 1, j] = np.linalg.norm(w)
        if H[j + 1, j] <= 1e-14 * abs(H[j, j]) + 1e-300:
            m = j + 1
            break
        V.append(w / H[j + 1, j])
    return float(np.max(np.real(np.linalg.eigvals(H[:m, :m]))))


class Level:
    def __init__(self, disc):
        self.disc = disc
        self.free = ~disc.dirichlet_mask()
        self.J = None
        self.smoother = None
        self.lam = None


class Hierarchy:
    """Levels n_coarse, 2 n_coarse, ..., n_fine (index 0 = coarsest)."""

    def __init__(self, n_fine, n_coarse, k, q, N, problem, opts=None):
        self.opts = opts or Options()
        ns = []
        n = n_fine
        while n >= n_coarse:
            ns.append(n)
            n //= 2
        ns = ns[::-1]
        assert ns[0] == n_coarse
        self.levels = [Level(Discretisation(n, k, q, N, problem)) for n in ns]
        self.P = [None] + [prolongation(self.levels[l].disc, self.levels[l - 1].disc)
                           for l in range(1, len(ns))]
        self.coarse = None

    @property
    def fine(self):
        return self.levels[-1].disc

    def linearise(self, W):
        """J(W) on every level (rediscretised about the injected iterate), the
        patch factorisations, the Chebyshev eigen-estimates and the coarse LU."""
        Ws = [None] * len(self.levels)
        Ws[-1] = W
        for l in range(len(self.levels) - 1, 0, -1):
            Ws[l - 1] = injection(self.levels[l].disc, self.levels[l - 1].disc, Ws[l])
        for l, lev in enumerate(self.levels):
            lev.J = lev.disc.jacobian(Ws[l])
            if l == 0:
                self.coarse = CoarseSolver(lev.disc, lev.J)
                continue
            lev.smoother = PatchSmoother(lev.disc, lev.J)
            v0 = splitmix64_uniform(l, lev.disc.ndofs) * lev.free
            J, M = lev.J, lev.smoother
            lev.lam = arnoldi_ritz_max(lambda v: M.apply(J @ v), v0, self.opts.eig_steps)

    def vcycle(self, b):
        """One V(2,2) cycle (Algorithm Vcycle) for J_fine x = b from a zero guess."""
        L = len(self.levels) - 1
        bs = [None] * (L + 1)
        xs = [None] * (L + 1)
        bs[L] = b
        for l in range(L, 0, -1):
            lev = self.levels[l]
            Jop = lambda v, J=lev.J: J @ v
            xs[l] = chebyshev(Jop, lev.smoother.apply, bs[l], None, lev.lam, self.opts)
            r = bs[l] - lev.J @ xs[l]
            bs[l - 1] = self.P[l].T @ r
        xs[0] = self.coarse.solve(bs[0])
        for l in range(1, L + 1):
            lev = self.levels[l]
            Jop = lambda v, J=lev.J: J @ v
            x = xs[l] + self.P[l] @ xs[l - 1]
            xs[l] = chebyshev(Jop, lev.smoother.apply, bs[l], x, lev.lam, self.opts)
        return xs[L]

    def precondition(self, v):
        return self.fine.project_pressure(self.vcycle(v))


def fgmres(Jop, Mop, b, tol, restart=30, maxit=200):
    """Right-preconditioned flexible GMRES(restart), MGS, Givens; zero initial guess.
    Returns (x, iterations)."""
    x = np.zeros_like(b)
    r = b.copy()
    beta = np.linalg.norm(r)
    its = 0
    while beta > tol and its < maxit:
        V = [r / beta]
        Z = []
        H = np.zeros((restart + 1, restart))
        cs, sn = np.zeros(restart), np.zeros(restart)
        g = np.zeros(restart + 1)
        g[0] = beta
        j_end = 0
        for j in range(restart):
            Z.append(Mop(V[j]))
            w = Jop(Z[j])
            for i in range(j + 1):
                H[i, j] = np.dot(w, V[i])
                w = w - H[i, j] * V[i]
            H[j + 1, j] = np.linalg.norm(w)
            V.append(w / H[j + 1, j] if H[j + 1, j] != 0.0 else w)
            for i in range(j):
                t = cs[i] * H[i, j] + sn[i] * H[i + 1, j]
                H[i + 1, j] = -sn[i] * H[i, j] + cs[i] * H[i + 1, j]
                H[i, j] = t
            den = np.hypot(H[j, j], H[j + 1, j])
            cs[j], sn[j] = H[j, j] / den, H[j + 1, j] / den
            H[j, j] = den
            H[j + 1, j] = 0.0
            g[j + 1] = -sn[j] * g[j]
            g[j] = cs[j] * g[j]
            its += 1
            j_end = j + 1
            if abs(g[j + 1]) <= tol or its >= maxit:
                break
        y = sla.solve_triangular(H[:j_end, :j_end], g[:j_end])
        for i in range(j_end):
            x = x + y[i] * Z[i]
        r = b - Jop(x)
        beta = np.linalg.norm(r)
    return x, its


def newton_solve(hier, U0=None, stats=None):
    """Inexact Newton with FGMRES + V-cycle inner solves; returns the iterate."""
    opts = hier.opts
    disc = hier.fine
    U = disc.initial_guess() if U0 is None else U0.copy()
    F = disc.residual(U)
    f0 = fnorm = np.linalg.norm(F)
    eta = 0.5 if opts.ew else opts.eta_fixed
    hist = {"residuals": [fnorm], "gmres": [], "eta": []}
    stalls = 0
    for _ in range(opts.newton_maxit):
        if fnorm <= opts.newton_rtol * f0:
            break
        if (opts.newton_divtol > 0 and fnorm > opts.newton_divtol * f0) or \
                (opts.newton_stall > 0 and stalls >= opts.newton_stall):
            break
        hier.linearise(U)
        J = hier.levels[-1].J
        delta, its = fgmres(lambda v: J @ v, hier.precondition, -F, eta * fnorm,
                            opts.restart, opts.gmres_maxit)
        stalls = stalls + 1 if its >= opts.gmres_maxit else 0
        U = U + delta
        F = disc.residual(U)
        fnew = np.linalg.norm(F)
        hist["gmres"].append(its)
        hist["eta"].append(eta)
        hist["residuals"].append(fnew)
        if opts.ew:
            gamma, alpha = 0.9, 2.0
            eta_new = gamma * (fnew / fnorm) ** alpha
            safe = gamma * eta ** alpha
            if safe > 0.1:
                eta_new = max(eta_new, safe)
            eta = min(0.9, max(eta_new, 0.5 * opts.newton_rtol * f0 / fnew))
        fnorm = fnew
    if stats is not None:
        stats.update(hist)
    return U


def timestepping_solve(n_fine, n_coarse, k, q, N, problem, opts=None, stats=None):
    """The timestepping comparator (Sec. 5): the N slabs of ``problem`` solved one
    after another, each as the one-slab space-time problem on
    [t0 + n dt, t0 + (n + 1) dt] whose slab-0 jump takes the previous step's end
    state (the last temporal DoF of its slab), with the same Newton-FGMRES-V-cycle
    solver coupling across one time element only.  Because the space-time system
    is block lower bidiagonal in slabs, its solution is the all-at-once one.
    Returns the N-slab global vector; stats (if given) gets per-step histories."""
    dt = problem.T / N
    prev = None
    out = []
    steps = []
    for n in range(N):
        pb = dataclasses.replace(problem, t0=problem.t0 + n * dt, T=dt)
        hier = Hierarchy(n_fine, n_coarse, k, q, 1, pb, opts)
        if prev is not None:
            hier.fine.initial_state = prev
        st = {}
        U = newton_solve(hier, stats=st)
        steps.append(st)
        out.append(U)
        d = hier.fine
        prev = U[d.block(0, d.nt - 1):d.block(0, d.nt - 1) + d.S].copy()
    if stats is not None:
        stats["steps"] = steps
    return np.concatenate(out)
