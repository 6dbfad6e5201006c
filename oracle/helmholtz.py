"""FP64 oracle for the CSG-preconditioned Helmholtz solve (test infrastructure only).

Notation follows the paper: H u = -(Laplacian + phi) u = chi (Eq. helm, Sec. 1), with
phi = k^2.  Grids are the unit interval per axis with N interior nodes, real spacing
h = 1/(N+1); u = 0 on the outer edge of the absorbing layers (and on the near edge of
the interior where the layers sit at the far end only, Benchmark 3 of Sec. 5).  Arrays are
``(N,)*d`` complex128 with the x axis last (C order), i.e. flat index
``(iz*N + iy)*N + ix``.
"""
from __future__ import annotations

from dataclasses import dataclass, field
from typing import Callable, List, Optional

import numpy as np


# ----------------------------------------------------------------------------------
# Grid (Sec. 2, Eq. csggrid; Remark 2.2 for layers on both sides)
# ----------------------------------------------------------------------------------

def complex_map(x: float, ecs_frac: float, theta_gamma: float, theta_beta: float,
                ecs_sides: str = "both") -> complex:
    """Complex coordinate z(x) = integral_0^x s(t) dt of the stretched grid.

    Sec. 2, Eq. csggrid: interior spacing h_beta = h e^{i theta_beta}, ECS layer
    spacing h_gamma = h e^{i theta_gamma}.  Remark 2.2: the layer is applied on both
    sides with the same angle.  Reading: s(t) = e^{i theta_gamma} for t < w or
    t > 1 - w (w = ``ecs_frac``), e^{i theta_beta} otherwise.  The printed interior
    grid ends at j h_beta and restarts the layer at 1 (garbled); only spacings enter
    the scheme, so the continuous map is used.

    ``ecs_sides = "high"`` puts the layer at the far end only (Benchmark 3 of Sec. 5:
    homogeneous Dirichlet on the south and west edges, ECS layers on the north and
    east edges): s(t) = e^{i theta_gamma} for t > 1 - w, e^{i theta_beta} otherwise,
    which is Eq. csggrid as printed (n interior intervals followed by m layer ones).
    """
    w = ecs_frac
    eg = np.exp(1j * theta_gamma)
    eb = np.exp(1j * theta_beta)
    if ecs_sides == "high":
        if x <= 1.0 - w:
            return x * eb
        return (1.0 - w) * eb + (x - (1.0 - w)) * eg
    if ecs_sides != "both":
        raise ValueError("ecs_sides is 'both' or 'high'")
    if x <= w:
        return x * eg
    if x <= 1.0 - w:
        return w * eg + (x - w) * eb
    return w * eg + (1.0 - 2.0 * w) * eb + (x - (1.0 - w)) * eg


def spacings(n: int, ecs_frac: float, theta_gamma: float, theta_beta: float,
             ecs_sides: str = "both") -> np.ndarray:
    """Complex spacings h_i = z(x_{i+1}) - z(x_i), i = 0..n, for nodes x_i = i/(n+1).

    The exact integral of the map handles an interval that straddles the
    layer/interior turning point (this happens on coarse levels).  Sec. 2.
    """
    h = 1.0 / (n + 1)
    z = np.array([complex_map(i * h, ecs_frac, theta_gamma, theta_beta, ecs_sides) for i in range(n + 2)])
    return np.diff(z)


def coefficients_1d(sp: np.ndarray):
    """Three-point non-uniform second difference (Shortley-Weller), Sec. 2.

    With h_l = h_{i-1}, h_r = h_i at interior node i,
        (L u)_i = -2/(h_l + h_r) * [ (u_{i+1} - u_i)/h_r - (u_i - u_{i-1})/h_l ],
    i.e. L ~ -d^2/dz^2.  Returned as (a, dg, c) with
        (L u)_i = a_i u_{i-1} + dg_i u_i + c_i u_{i+1}.
    """
    hl = sp[:-1]
    hr = sp[1:]
    s = hl + hr
    a = -2.0 / (s * hl)
    c = -2.0 / (s * hr)
    dg = 2.0 / (hl * hr)
    return a, dg, c


def apply_operator(u: np.ndarray, coef, phi) -> np.ndarray:
    """(M u)_p = sum over axes of (L_axis u)_p - phi_p u_p.

    Sec. 2, Eq. csg_dis and Lemma 2.1: the d-D operator is the Kronecker sum of the
    1D operators.  Reading of the garbled sign: the paper prints L + k^2 I but its
    own triangle vertex t0 = -k^2 and the proof of Lemma 2.1 use L - k^2 I with
    L ~ -Laplacian, consistent with Eq. helm; this oracle uses L - phi.
    ``phi`` is a scalar or an array shaped like ``u``.
    """
    a, dg, c = coef
    d = u.ndim
    n = u.shape[0]
    up = np.pad(u, 1)
    inner = tuple([slice(1, -1)] * d)
    out = -np.asarray(phi) * u
    for ax in range(d):
        shape = [1] * d
        shape[ax] = n
        lo = list(inner)
        lo[ax] = slice(0, -2)
        hi = list(inner)
        hi[ax] = slice(2, None)
        out = out + a.reshape(shape) * up[tuple(lo)] + dg.reshape(shape) * u + c.reshape(shape) * up[tuple(hi)]
    return out


# ----------------------------------------------------------------------------------
# Multigrid hierarchy (Sec. 3.1, Prop. 3.1: rediscretisation on 2h, 4h, ...)
# ----------------------------------------------------------------------------------

def level_sizes(n: int, coarsest: int = 3) -> List[int]:
    """Interior sizes per level: N_{l+1} = (N_l + 1)/2 - 1 while N_l > ``coarsest``
    and N_l + 1 is even.  Vertex-centred coarsening: coarse node I sits on fine node
    2I (1-based).  Reading: the paper's levels have spacing h, 2h, 4h (Prop. 3.1's
    "l h" is read as 2^l h, as its Fig. 3 uses h, 2h, 4h)."""
    sizes = [n]
    while sizes[-1] > coarsest and (sizes[-1] + 1) % 2 == 0:
        sizes.append((sizes[-1] + 1) // 2 - 1)
    return sizes


def _inject(field: np.ndarray) -> np.ndarray:
    """Sample a nodal field at the coarse nodes (fine 1-based index 2I = 0-based 2I+1)."""
    sl = tuple([slice(1, None, 2)] * field.ndim)
    return field[sl]


@dataclass
class Level:
    n: int
    dim: int
    coef: tuple                 # CSG operator M (theta_beta) coefficients
    phi: object                 # scalar or (n,)*dim array
    coef_h: Optional[tuple] = None   # ECS operator H (theta_beta = 0), finest level only
    lu: Optional[np.ndarray] = None  # dense coarsest matrix (coarsest level only)
    shift: complex = 1.0        # M uses shift * phi: 1 for CSG, 1 + i eps for the CSL variant

    def apply(self, u):
        return apply_operator(u, self.coef, self.shift * np.asarray(self.phi))

    def apply_h(self, u):
        return apply_operator(u, self.coef_h, self.phi)


def build_hierarchy(dim: int, n: int, theta_beta: float, theta_gamma: float = 0.5,
                    ecs_frac: float = 0.125, k: Optional[float] = None,
                    phi: Optional[np.ndarray] = None, coarsest: int = 3,
                    csl_eps: float = 0.0, ecs_sides: str = "both") -> List[Level]:
    """Rediscretised hierarchy of M^CSG (Sec. 3.1, Prop. 3.1).

    Each level uses the same complex map with doubled real spacing; phi is sampled
    at the level's nodes (constant k: phi = k^2 everywhere; a field given on the
    fine nodes is sampled at the coincident coarse nodes).  The finest level also
    carries H (theta_beta = 0, Sec. 2 after Eq. csg_dis).

    ``csl_eps`` > 0 gives the complex shifted Laplacian variant of the preconditioner
    (Sec. 1 and Sec. 2: the shift (1 + eps i) k^2 of Erlangga, Oosterlee and Vuik):
    M = L - (1 + i eps) phi on every level; with theta_beta = 0 this is M^CSL on the
    real interior grid (the ECS layers stay), with theta_beta > 0 both devices
    combine.  H is never shifted.

    ``ecs_sides = "high"``: layers at the far end of every axis only, homogeneous
    Dirichlet at the near end (Benchmark 3 of Sec. 5), see ``complex_map``.
    """
    if (k is None) == (phi is None):
        raise ValueError("give exactly one of k (constant) or phi (field)")
    levels = []
    cur_phi = float(k) ** 2 if k is not None else np.asarray(phi, dtype=np.float64)
    for li, nl in enumerate(level_sizes(n, coarsest)):
        if li > 0 and not np.isscalar(cur_phi):
            cur_phi = _inject(cur_phi)
        sp = spacings(nl, ecs_frac, theta_gamma, theta_beta, ecs_sides)
        lev = Level(n=nl, dim=dim, coef=coefficients_1d(sp), phi=cur_phi, shift=complex(1.0, csl_eps))
        if li == 0:
            lev.coef_h = coefficients_1d(spacings(nl, ecs_frac, theta_gamma, 0.0, ecs_sides))
        levels.append(lev)
    levels[-1].lu = dense_matrix(levels[-1])
    return levels


def dense_matrix(level: Level, which: str = "M") -> np.ndarray:
    """Dense matrix of a level's operator, column by column on unit vectors."""
    m = level.n ** level.dim
    shape = (level.n,) * level.dim
    op = level.apply if which == "M" else level.apply_h
    A = np.zeros((m, m), dtype=np.complex128)
    for j in range(m):
        e = np.zeros(m, dtype=np.complex128)
        e[j] = 1.0
        A[:, j] = op(e.reshape(shape)).ravel()
    return A


def coarse_solve(level: Level, b: np.ndarray) -> np.ndarray:
    """Coarsest-grid direct solve (3^d unknowns): LAPACK LU with partial pivoting.
    The paper leaves the coarsest treatment unstated; a direct solve is the reading."""
    return np.linalg.solve(level.lu, b.ravel()).reshape(b.shape)


# ----------------------------------------------------------------------------------
# Transfers.  The paper does not state them; reading: index-based full weighting
# (1/4, 1/2, 1/4)^{(x)d} and its scaled transpose, bi-/trilinear prolongation.
# ----------------------------------------------------------------------------------

def restrict_fw(r: np.ndarray) -> np.ndarray:
    """b_c[I] = sum over the 3^d fine nodes 2I-1, 2I, 2I+1 (1-based, per axis) with
    tensor weights (1/4, 1/2, 1/4); fine boundary values are zero."""
    out = np.asarray(r, dtype=np.complex128)
    for ax in range(r.ndim):
        f = np.moveaxis(out, ax, 0)
        n_c = (f.shape[0] + 1) // 2 - 1
        fp = np.concatenate([np.zeros_like(f[:1]), f, np.zeros_like(f[:1])])  # 1-based
        idx = 2 * np.arange(1, n_c + 1)
        red = 0.25 * fp[idx - 1] + 0.5 * fp[idx] + 0.25 * fp[idx + 1]
        out = np.moveaxis(red, 0, ax)
    return out


def prolong(e: np.ndarray, n_fine: int) -> np.ndarray:
    """Bi-/trilinear interpolation, vertex-centred: fine 2I <- e[I], fine 2I+1 <-
    (e[I] + e[I+1]) / 2 per axis (1-based), with e = 0 on the coarse boundary.
    Equals 2^d R^T for the full-weighting R above."""
    out = np.asarray(e, dtype=np.complex128)
    for ax in range(e.ndim):
        c = np.moveaxis(out, ax, 0)
        n_c = c.shape[0]
        cp = np.concatenate([np.zeros_like(c[:1]), c, np.zeros_like(c[:1])])  # 1-based
        f = np.zeros((n_fine,) + c.shape[1:], dtype=np.complex128)
        f[1::2] = cp[1:n_c + 1]                       # 1-based even fine index 2I
        f[0::2] = 0.5 * (cp[0:n_c + 1] + cp[1:n_c + 2])  # 1-based odd fine index 2I+1
        out = np.moveaxis(f, 0, ax)
    return out


# ----------------------------------------------------------------------------------
# GMRES(s) smoother (Sec. 3.1: one smoothing step = a GMRES solve on the error
# equation stopped after s iterations, s matrix-vector products)
# ----------------------------------------------------------------------------------

BREAKDOWN = 1e-14


def gmres_sweep(apply: Callable, b: np.ndarray, x: np.ndarray, s: int) -> np.ndarray:
    """One GMRES(s) step on A x = b from the current x (Sec. 3.1; Sec. 4 intro: the
    residual after s iterations is min over p in P_s, p(0) = 1, of ||p(A) r0||).

    GMRES on the error equation A e = r0 from e = 0 equals GMRES on A x = b from x.
    Arnoldi with modified Gram-Schmidt; the (j+1) x j least-squares problem is solved
    with LAPACK.  Reading (unstated): if h_{j+1,j} <= 1e-14 * beta the Krylov space
    is invariant and the sweep stops there.
    """
    r0 = b - apply(x)
    beta = np.linalg.norm(r0)
    if beta == 0.0:
        return x.copy()
    V = [r0 / beta]
    Hm = np.zeros((s + 1, s), dtype=np.complex128)
    m = s
    for j in range(s):
        w = apply(V[j])
        for i in range(j + 1):
            Hm[i, j] = np.vdot(V[i], w)
            w = w - Hm[i, j] * V[i]
        Hm[j + 1, j] = np.linalg.norm(w)
        if abs(Hm[j + 1, j]) <= BREAKDOWN * beta:
            m = j + 1
            break
        V.append(w / Hm[j + 1, j])
    rhs = np.zeros(m + 1, dtype=np.complex128)
    rhs[0] = beta
    y = np.linalg.lstsq(Hm[: m + 1, :m], rhs, rcond=None)[0]
    out = x.copy()
    for j in range(m):
        out = out + y[j] * V[j]
    return out


# ----------------------------------------------------------------------------------
# V-cycle (Sec. 3.1; Sec. 3.2: V(nu1, nu2) with GMRES(s) on every level; Sec. 5: one
# cycle from a zero initial guess approximates (M^CSG)^{-1})
# ----------------------------------------------------------------------------------

def vcycle(levels: List[Level], b: np.ndarray, nu1: int = 1, nu2: int = 1, s: int = 3,
           level: int = 0) -> np.ndarray:
    """x ~ M_l^{-1} b by one V(nu1, nu2) cycle with GMRES(s) smoothing, zero start."""
    lev = levels[level]
    if level == len(levels) - 1:
        return coarse_solve(lev, b)
    x = np.zeros_like(b, dtype=np.complex128)
    for _ in range(nu1):
        x = gmres_sweep(lev.apply, b, x, s)
    r = b - lev.apply(x)
    bc = restrict_fw(r)
    ec = vcycle(levels, bc, nu1, nu2, s, level + 1)
    x = x + prolong(ec, lev.n)
    for _ in range(nu2):
        x = gmres_sweep(lev.apply, b, x, s)
    return x


# ----------------------------------------------------------------------------------
# Outer flexible GMRES (Sec. 5: FGMRES [Saad 1993] on H u = b, right-preconditioned
# by one V-cycle on M^CSG, stop at a relative residual tolerance)
# ----------------------------------------------------------------------------------

@dataclass
class SolveInfo:
    iters: int = 0
    restarts: int = 0
    rel_res_est: float = np.inf
    rel_res_true: float = np.inf
    history: List[float] = field(default_factory=list)
    converged: bool = False


def fgmres(apply_h: Callable, precond: Callable, b: np.ndarray, x0: Optional[np.ndarray] = None,
           tol: float = 1e-6, restart: int = 0, maxit: int = 1000):
    """Right-preconditioned flexible GMRES(m) with modified Gram-Schmidt.

    z_j = P(v_j) (one V-cycle), w = H z_j, x = x0 + Z y with y the least-squares
    minimiser of ||beta e1 - Hbar y||.  The estimate ||beta e1 - Hbar y|| / ||b|| is
    checked after every iteration; at a cycle's end the true residual ||b - H x|| is
    recomputed, and the method restarts from x if it is still above ``tol``.
    ``restart = 0`` means no restart (the paper's iteration counts, up to 285 in
    Table 5, suggest none).  The iteration count is the number of preconditioner
    applications.
    """
    x = np.zeros_like(b, dtype=np.complex128) if x0 is None else np.array(x0, dtype=np.complex128)
    bnorm = np.linalg.norm(b)
    info = SolveInfo()
    if bnorm == 0.0:
        info.rel_res_est = info.rel_res_true = 0.0
        info.converged = True
        return np.zeros_like(x), info
    m = restart if restart > 0 else maxit
    while True:
        r = b - apply_h(x)
        beta = np.linalg.norm(r)
        info.rel_res_true = beta / bnorm
        if info.rel_res_true <= tol:
            info.converged = True
            return x, info
        if info.iters >= maxit:
            return x, info
        V = [r / beta]
        Z = []
        Hm = np.zeros((m + 1, m), dtype=np.complex128)
        y = np.zeros(0, dtype=np.complex128)
        for j in range(m):
            z = precond(V[j])
            Z.append(z)
            info.iters += 1
            w = apply_h(z)
            for i in range(j + 1):
                Hm[i, j] = np.vdot(V[i], w)
                w = w - Hm[i, j] * V[i]
            Hm[j + 1, j] = np.linalg.norm(w)
            rhs = np.zeros(j + 2, dtype=np.complex128)
            rhs[0] = beta
            y = np.linalg.lstsq(Hm[: j + 2, : j + 1], rhs, rcond=None)[0]
            est = np.linalg.norm(rhs - Hm[: j + 2, : j + 1] @ y) / bnorm
            info.rel_res_est = est
            info.history.append(est)
            breakdown = abs(Hm[j + 1, j]) <= BREAKDOWN * beta
            if est <= tol or info.iters >= maxit or breakdown:
                break
            V.append(w / Hm[j + 1, j])
        for j in range(len(y)):
            x = x + y[j] * Z[j]
        info.restarts += 1
