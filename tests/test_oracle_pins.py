"""Pins for the FP64 oracle: each test checks it against something other than itself.

Independent routes used here: node coordinates by numerical quadrature of the
stretching function, a sparse matrix assembled from Lagrange second-derivative
weights of the complex nodes, closed-form Dirichlet eigenpairs (no stretching), the
uniform-rotation identity, exactness of the 3-point scheme on complex quadratics,
brute-force Krylov least squares, dense/sparse direct solves and a manufactured
solution.
"""
import warnings

import numpy as np
import pytest
import scipy.integrate
import scipy.sparse as sps
import scipy.sparse.linalg as spla

import oracle as O
from paper_1012_5379_gb300 import inputs as I

TG, WF = 0.5, 0.125


# ------------------------------------------------------------------ independent grid
def nodes_by_quadrature(n, ecs, tg, tb):
    """z(x_i) by adaptive quadrature of s(t) = e^{i theta(t)} (Sec. 2)."""
    def s_re(t):
        th = tg if (t < ecs or t > 1 - ecs) else tb
        return np.cos(th)

    def s_im(t):
        th = tg if (t < ecs or t > 1 - ecs) else tb
        return np.sin(th)

    warnings.simplefilter("ignore", scipy.integrate.IntegrationWarning)
    z = [0j]
    for i in range(1, n + 2):
        x0, x1 = (i - 1) / (n + 1), i / (n + 1)
        pts = [p for p in (ecs, 1 - ecs) if x0 < p < x1]
        re = scipy.integrate.quad(s_re, x0, x1, points=pts or None, epsabs=1e-15, epsrel=1e-14)[0]
        im = scipy.integrate.quad(s_im, x0, x1, points=pts or None, epsabs=1e-15, epsrel=1e-14)[0]
        z.append(z[-1] + re + 1j * im)
    return np.array(z)


def lagrange_1d(z):
    """-u'' of the quadratic interpolant through (z_{i-1}, z_i, z_{i+1}), as a sparse
    n x n matrix (Dirichlet ends): a different algebraic route to the scheme."""
    n = len(z) - 2
    rows, cols, vals = [], [], []
    for i in range(1, n + 1):
        zs = (z[i - 1], z[i], z[i + 1])
        for k, j in enumerate((i - 1, i, i + 1)):
            others = [zs[m] for m in range(3) if m != k]
            w = -2.0 / ((zs[k] - others[0]) * (zs[k] - others[1]))
            if 1 <= j <= n:
                rows.append(i - 1)
                cols.append(j - 1)
                vals.append(w)
    return sps.csr_matrix((vals, (rows, cols)), shape=(n, n), dtype=np.complex128)


def assemble(dim, n, tb, tg=TG, ecs=WF, phi=0.0):
    L1 = lagrange_1d(nodes_by_quadrature(n, ecs, tg, tb))
    eye = sps.identity(n, dtype=np.complex128, format="csr")
    A = sps.csr_matrix((n ** dim, n ** dim), dtype=np.complex128)
    for ax in range(dim):
        mats = [eye] * dim
        mats[ax] = L1
        K = mats[0]
        for m in mats[1:]:
            K = sps.kron(K, m, format="csr")
        A = A + K
    phi_vec = np.broadcast_to(np.asarray(phi, dtype=np.float64), (n,) * dim).ravel()
    return (A - sps.diags(phi_vec)).tocsr()


def crand(shape, seed):
    g = np.random.default_rng(seed)
    return g.standard_normal(shape) + 1j * g.standard_normal(shape)


# ------------------------------------------------------------------ grid / operator
@pytest.mark.parametrize("n,tb", [(3, 0.4), (7, 0.1), (15, 0.3), (31, 0.5), (47, 0.18)])
def test_spacings_match_quadrature(n, tb):
    ecs = 1 / 6 if n == 47 else WF
    z = nodes_by_quadrature(n, ecs, TG, tb)
    sp = O.spacings(n, ecs, TG, tb)
    assert np.max(np.abs(sp - np.diff(z))) < 1e-13


@pytest.mark.parametrize("dim,n", [(1, 15), (2, 7), (2, 15), (3, 7)])
@pytest.mark.parametrize("field", [False, True])
def test_operator_matches_lagrange_assembly(dim, n, field):
    tb = 0.3
    phi = (np.random.default_rng(5).uniform(50, 400, (n,) * dim)) if field else 123.0
    lev = O.build_hierarchy(dim, n, tb, TG, WF, k=None if field else np.sqrt(123.0),
                            phi=phi if field else None)[0]
    A = assemble(dim, n, tb, phi=phi)
    u = crand((n,) * dim, 7)
    ref = (A @ u.ravel()).reshape(u.shape)
    got = lev.apply(u)
    assert np.linalg.norm(got - ref) / np.linalg.norm(ref) < 1e-13
    # H = the same scheme with theta_beta = 0 (Sec. 2)
    Ah = assemble(dim, n, 0.0, phi=phi)
    refh = (Ah @ u.ravel()).reshape(u.shape)
    assert np.linalg.norm(lev.apply_h(u) - refh) / np.linalg.norm(refh) < 1e-13


@pytest.mark.parametrize("dim,n", [(2, 31), (3, 15)])
def test_closed_form_dirichlet_eigenpairs(dim, n):
    """No stretching: eigenvalues 4/h^2 sum sin^2(j pi h / 2) - k^2 with sine modes
    (the t1 = 4d/h^2 bound of Lemma 2.1 is the j -> n+1 limit)."""
    k = 9.0
    lev = O.build_hierarchy(dim, n, 0.0, theta_gamma=0.0, ecs_frac=WF, k=k)[0]
    h = 1.0 / (n + 1)
    x = np.arange(1, n + 1) * h
    for js in [(1,) * dim, (2, 5, 3)[:dim], (n,) * dim, (n // 2, 1, n)[:dim]]:
        mode = np.ones((n,) * dim)
        lam = -k * k
        for ax, j in enumerate(js):
            shape = [1] * dim
            shape[ax] = n
            mode = mode * np.sin(j * np.pi * x).reshape(shape)
            lam += 4.0 / h ** 2 * np.sin(j * np.pi * h / 2) ** 2
        got = lev.apply(mode.astype(np.complex128))
        assert np.linalg.norm(got - lam * mode) <= 1e-12 * abs(lam) * np.linalg.norm(mode) + 1e-9


@pytest.mark.parametrize("dim,n,eps", [(2, 31, 0.5), (3, 15, 0.25)])
def test_closed_form_csl_eigenpairs(dim, n, eps):
    """Complex shifted Laplacian variant without stretching: the sine modes stay
    eigenvectors and the shift moves every eigenvalue by -(1 + i eps) k^2 (Sec. 2:
    the CSL spectrum is the Laplacian's translated by the shift), while H is unshifted."""
    k = 9.0
    lev = O.build_hierarchy(dim, n, 0.0, theta_gamma=0.0, ecs_frac=WF, k=k, csl_eps=eps)[0]
    h = 1.0 / (n + 1)
    x = np.arange(1, n + 1) * h
    for js in [(1,) * dim, (2, 5, 3)[:dim], (n,) * dim]:
        mode = np.ones((n,) * dim)
        lap = 0.0
        for ax, j in enumerate(js):
            shape = [1] * dim
            shape[ax] = n
            mode = mode * np.sin(j * np.pi * x).reshape(shape)
            lap += 4.0 / h ** 2 * np.sin(j * np.pi * h / 2) ** 2
        lam = lap - (1 + 1j * eps) * k * k
        got = lev.apply(mode.astype(np.complex128))
        assert np.linalg.norm(got - lam * mode) <= 1e-12 * abs(lam) * np.linalg.norm(mode) + 1e-9
        got_h = lev.apply_h(mode.astype(np.complex128))
        assert np.linalg.norm(got_h - (lap - k * k) * mode) <= 1e-12 * abs(lap) * np.linalg.norm(mode) + 1e-9


def test_uniform_rotation_identity():
    """theta_beta = theta_gamma = theta: every spacing is h e^{i theta}, so the
    Laplacian part is e^{-2 i theta} times the real one (closed form)."""
    n, th, k = 15, 0.37, 11.0
    rot = O.build_hierarchy(2, n, th, theta_gamma=th, ecs_frac=WF, k=k)[0]
    real = O.build_hierarchy(2, n, 0.0, theta_gamma=0.0, ecs_frac=WF, k=k)[0]
    u = crand((n, n), 3)
    lhs = rot.apply(u) + k * k * u
    rhs = np.exp(-2j * th) * (real.apply(u) + k * k * u)
    assert np.linalg.norm(lhs - rhs) / np.linalg.norm(rhs) < 1e-13


def quad_manufactured(dim, n, tb, tg=TG, ecs=WF):
    """u*(z) = prod_a z_a (Z - z_a) at the nodes, and -Laplacian u* analytically."""
    z = nodes_by_quadrature(n, ecs, tg, tb)
    Z = z[-1]
    zi = z[1:-1]
    f = zi * (Z - zi)             # per-axis factor
    lap = -2.0 * np.ones(n)       # second derivative of z (Z - z)
    u = np.ones((n,) * dim, dtype=np.complex128)
    for ax in range(dim):
        shape = [1] * dim
        shape[ax] = n
        u = u * f.reshape(shape)
    mlap = np.zeros_like(u)
    for ax in range(dim):
        term = np.ones((n,) * dim, dtype=np.complex128)
        for bx in range(dim):
            shape = [1] * dim
            shape[bx] = n
            term = term * (lap if bx == ax else f).reshape(shape)
        mlap = mlap - term
    return u, mlap


@pytest.mark.parametrize("dim,n", [(1, 3), (1, 7), (2, 3), (2, 15), (3, 7)])
def test_exact_on_complex_quadratics(dim, n):
    """The 3-point scheme differentiates quadratics in z exactly, layers and
    straddling coarse intervals included (Sec. 2)."""
    tb = 0.25
    lev = O.build_hierarchy(dim, n, tb, TG, WF, k=0.0)[0]
    u, mlap = quad_manufactured(dim, n, tb)
    got = lev.apply(u)
    assert np.linalg.norm(got - mlap) / np.linalg.norm(mlap) < 1e-12


@pytest.mark.parametrize("dim,n,k", [(1, 31, 10.0), (2, 15, 8.0)])
def test_spectrum_in_lemma_triangle(dim, n, k):
    """Lemma 2.1: sigma(M) lies in the triangle t0 = -k^2, t1 = -k^2 + 4d/h_b^2,
    t2 = -k^2 + 4d/h_g^2 (soft gate, slack 1e-8 |t1|)."""
    tb, tg = 0.2, np.pi / 6
    lev = O.build_hierarchy(dim, n, tb, tg, WF, k=k)[0]
    A = O.helmholtz.dense_matrix(lev)
    ev = np.linalg.eigvals(A)
    h = 1.0 / (n + 1)
    t0 = -k * k
    t1 = -k * k + 4 * dim / (h * np.exp(1j * tb)) ** 2
    t2 = -k * k + 4 * dim / (h * np.exp(1j * tg)) ** 2
    T = np.array([[t0.real if isinstance(t0, complex) else t0, t1.real, t2.real],
                  [0.0, t1.imag, t2.imag], [1.0, 1.0, 1.0]])
    for lam in ev:
        bary = np.linalg.solve(T, np.array([lam.real, lam.imag, 1.0]))
        assert bary.min() > -1e-8, (lam, bary)


# ------------------------------------------------------------------ transfers
def dense_op(fun, n_in, dim):
    m = n_in ** dim
    cols = []
    for j in range(m):
        e = np.zeros(m, dtype=np.complex128)
        e[j] = 1
        cols.append(fun(e.reshape((n_in,) * dim)).ravel())
    return np.array(cols).T


@pytest.mark.parametrize("dim,n", [(1, 15), (2, 7), (3, 7), (2, 11)])
def test_prolongation_is_scaled_transpose(dim, n):
    nc = (n + 1) // 2 - 1
    R = dense_op(O.restrict_fw, n, dim)
    P = dense_op(lambda e: O.prolong(e, n), nc, dim)
    assert np.allclose(P, 2 ** dim * R.T, atol=1e-15)


def test_full_weighting_exact_on_linear_fields():
    n = 31
    x = np.arange(1, n + 1) / (n + 1)
    X, Y = np.meshgrid(x, x, indexing="ij")
    f = (2.0 + 3.0 * X - 1.5 * Y) * (1 + 0.5j)
    xc = np.arange(1, (n + 1) // 2) * 2 / (n + 1)
    Xc, Yc = np.meshgrid(xc, xc, indexing="ij")
    fc = (2.0 + 3.0 * Xc - 1.5 * Yc) * (1 + 0.5j)
    assert np.max(np.abs(O.restrict_fw(f) - fc)) < 1e-14


def test_prolongation_exact_on_linear_fields():
    n = 31
    nc = (n + 1) // 2 - 1
    xc = np.arange(1, nc + 1) * 2 / (n + 1)
    x = np.arange(1, n + 1) / (n + 1)
    # f = x y vanishes on the x = 0 and y = 0 edges; it is bilinear, so interpolation is
    # exact wherever both neighbours are interior coarse nodes or the zero edge
    Xc, Yc = np.meshgrid(xc, xc, indexing="ij")
    X, Y = np.meshgrid(x, x, indexing="ij")
    got = O.prolong((Xc * Yc).astype(np.complex128), n)
    assert np.max(np.abs(got[:-1, :-1] - (X * Y)[:-1, :-1])) < 1e-14


# ------------------------------------------------------------------ GMRES(s)
@pytest.mark.parametrize("s", [1, 2, 3])
def test_gmres_sweep_equals_bruteforce_krylov_lstsq(s):
    """GMRES(s) from x: x + K c with K = [r0, M r0, ..., M^{s-1} r0] and
    c = argmin ||r0 - M K c|| (Sec. 4 intro: min over p in P_s of ||p(A) r0||)."""
    n = 15
    lev = O.build_hierarchy(2, n, 0.3, TG, WF, k=12.0)[0]
    A = O.helmholtz.dense_matrix(lev)
    b = crand(n * n, 1)
    x = crand(n * n, 2) * 1e-3
    r0 = b - A @ x
    K = [r0]
    for _ in range(s - 1):
        K.append(A @ K[-1])
    K = np.array(K).T
    # scale columns for a well-posed brute-force solve
    sc = np.linalg.norm(K, axis=0)
    c = np.linalg.lstsq(A @ (K / sc), r0, rcond=None)[0]
    ref = x + (K / sc) @ c
    got = O.gmres_sweep(lev.apply, b.reshape(n, n), x.reshape(n, n), s).ravel()
    assert np.linalg.norm(got - ref) / np.linalg.norm(ref) < 1e-9


def test_gmres_residual_never_increases():
    n = 31
    lev = O.build_hierarchy(2, n, 0.3, TG, WF, k=25.0)[0]
    b = crand((n, n), 4)
    x = np.zeros_like(b)
    prev = np.linalg.norm(b)
    for s in (1, 2, 3, 4):
        xs = O.gmres_sweep(lev.apply, b, x, s)
        res = np.linalg.norm(b - lev.apply(xs))
        assert res <= prev * (1 + 1e-12)
        prev = res
    # repeated sweeps from zero keep the residual non-increasing as well
    prev = np.linalg.norm(b)
    for _ in range(4):
        x = O.gmres_sweep(lev.apply, b, x, 3)
        res = np.linalg.norm(b - lev.apply(x))
        assert res <= prev * (1 + 1e-12)
        prev = res


def test_gmres_breakdown_returns_exact_solution():
    """An eigenvector right-hand side makes the Krylov space invariant after one
    step: the sweep must return the exact solution (reading of breakdown)."""
    n, k = 15, 9.0
    lev = O.build_hierarchy(2, n, 0.0, theta_gamma=0.0, ecs_frac=WF, k=k)[0]
    h = 1 / (n + 1)
    x = np.arange(1, n + 1) * h
    mode = np.outer(np.sin(2 * np.pi * x), np.sin(3 * np.pi * x)).astype(np.complex128)
    lam = -k * k + 4 / h ** 2 * (np.sin(2 * np.pi * h / 2) ** 2 + np.sin(3 * np.pi * h / 2) ** 2)
    got = O.gmres_sweep(lev.apply, mode, np.zeros_like(mode), 3)
    assert np.linalg.norm(got - mode / lam) / np.linalg.norm(mode / lam) < 1e-12


@pytest.mark.parametrize("s", [1, 2, 3, 4])
def test_vcycle_is_exact_on_s_eigenvectors(s):
    """A source spanned by s eigenvectors of M (sine modes, no stretching) lies in an
    s-dimensional invariant Krylov space: the pre-smoothing GMRES(s) sweep solves it
    exactly, the residual it leaves is rounding, and the whole V(1,1) cycle returns
    M^{-1} b.  With s + 1 modes the sweep is no longer exact and neither is the cycle."""
    n, k = 31, 9.0
    levels = O.build_hierarchy(2, n, 0.0, theta_gamma=0.0, ecs_frac=WF, k=k)
    h = 1 / (n + 1)
    x = np.arange(1, n + 1) * h
    modes = [(1, 1), (2, 3), (5, 1), (4, 6), (7, 2)]

    def source(count):
        b = np.zeros((n, n), dtype=np.complex128)
        exact = np.zeros_like(b)
        for i, (jx, jy) in enumerate(modes[:count]):
            mode = np.outer(np.sin(jy * np.pi * x), np.sin(jx * np.pi * x))
            lam = -k * k + 4 / h ** 2 * (np.sin(jx * np.pi * h / 2) ** 2 + np.sin(jy * np.pi * h / 2) ** 2)
            coef = (1.0 + 0.5j) * (i + 1)
            b += coef * mode
            exact += coef * mode / lam
        return b, exact

    b, exact = source(s)
    got = O.vcycle(levels, b, 1, 1, s)
    assert np.linalg.norm(got - exact) <= 1e-10 * np.linalg.norm(exact)
    b, exact = source(s + 1)
    got = O.vcycle(levels, b, 1, 1, s)
    assert np.linalg.norm(got - exact) > 1e-6 * np.linalg.norm(exact)


def _dense_vcycle(Ms, Rs, Ps, b, nu1, nu2, s, level=0):
    """The V(nu1, nu2) cycle of Sec. 3.1 restated with dense matrices: every GMRES(s)
    step by brute force (x + K c, K the monomial Krylov basis of the residual, c by
    least squares), the coarsest level by a dense solve."""
    M = Ms[level]
    if level == len(Ms) - 1:
        return np.linalg.solve(M, b)

    def step(x):
        r0 = b - M @ x
        K = [r0]
        for _ in range(s - 1):
            K.append(M @ K[-1])
        K = np.array(K).T
        K = K / np.linalg.norm(K, axis=0)
        return x + K @ np.linalg.lstsq(M @ K, r0, rcond=None)[0]

    x = np.zeros_like(b)
    for _ in range(nu1):
        x = step(x)
    ec = _dense_vcycle(Ms, Rs, Ps, Rs[level] @ (b - M @ x), nu1, nu2, s, level + 1)
    x = x + Ps[level] @ ec
    for _ in range(nu2):
        x = step(x)
    return x


def _full_weighting_1d(n):
    """(nc x n) rows (1/4, 1/2, 1/4) centred on the fine node under each coarse node."""
    nc = (n + 1) // 2 - 1
    R = np.zeros((nc, n))
    for i in range(nc):
        R[i, 2 * i:2 * i + 3] = (0.25, 0.5, 0.25)
    return R


@pytest.mark.parametrize("dim,n,hetero,cyc", [(2, 15, False, (1, 1, 3)), (2, 15, True, (1, 1, 3)),
                                              (2, 15, False, (2, 1, 2)), (2, 15, True, (1, 0, 1)),
                                              (2, 31, True, (0, 2, 3)), (3, 7, True, (1, 1, 3))])
def test_vcycle_equals_dense_bruteforce_cycle(dim, n, hetero, cyc):
    """The whole cycle against a restatement that shares nothing with the oracle but the
    reading of the paper: each level's matrix assembled from quadrature nodes and Lagrange
    weights, transfers as Kronecker products of the 1D full weighting and its doubled
    transpose, phi sampled at the coincident coarse nodes, GMRES(s) by brute force.  A
    wrong correction sign, a restricted right-hand side instead of the residual, a
    post-sweep on the wrong system or a dropped level each fail it."""
    nu1, nu2, s = cyc
    tb, k = 0.3, 8.0
    phi = k * k * (1.0 + 0.3 * np.tanh(crand((n,) * dim, 9).real)) if hetero else k * k
    levels = (O.build_hierarchy(dim, n, tb, TG, WF, phi=phi) if hetero
              else O.build_hierarchy(dim, n, tb, TG, WF, k=k))
    Ms, Rs, Ps = [], [], []
    nl, ph = n, phi
    while True:
        Ms.append(assemble(dim, nl, tb, TG, WF, phi=ph).toarray())
        if nl <= 3:
            break
        R1 = _full_weighting_1d(nl)
        R = R1
        for _ in range(dim - 1):
            R = np.kron(R, R1)
        Rs.append(R)
        Ps.append(2 ** dim * R.T)
        if hetero:
            ph = ph[tuple([slice(1, None, 2)] * dim)]
        nl = (nl + 1) // 2 - 1
    assert [lev.n for lev in levels] == [round(M.shape[0] ** (1 / dim)) for M in Ms]
    b = crand((n,) * dim, 21)
    want = _dense_vcycle(Ms, Rs, Ps, b.ravel(), nu1, nu2, s)
    got = O.vcycle(levels, b, nu1, nu2, s).ravel()
    assert np.linalg.norm(got - want) <= 1e-9 * np.linalg.norm(want)


def test_zero_rhs_sweep_and_vcycle():
    levels = O.build_hierarchy(2, 15, 0.3, TG, WF, k=5.0)
    z = np.zeros((15, 15), dtype=np.complex128)
    assert not np.any(O.gmres_sweep(levels[0].apply, z, z, 3))
    assert not np.any(O.vcycle(levels, z))


# ------------------------------------------------------------------ coarse solve
@pytest.mark.parametrize("dim", [2, 3])
def test_coarse_solve_against_independent_matrix(dim):
    levels = O.build_hierarchy(dim, 7, 0.4, TG, WF, k=6.0)
    lev = levels[-1]
    assert lev.n == 3
    A = assemble(dim, 3, 0.4, phi=36.0).toarray()
    b = crand((3,) * dim, 9)
    x = O.coarse_solve(lev, b)
    assert np.linalg.norm(A @ x.ravel() - b.ravel()) / np.linalg.norm(b) < 1e-13


# ------------------------------------------------------------------ V-cycle
def test_vcycle_stationary_iteration_converges_to_direct_solve():
    """x <- x + V(b - M x) converges to M^{-1} b; the average V(1,1) rate at the
    paper's constant-k setup stays at or below 0.25 (Sec. 3.2, soft)."""
    n, k = 63, 20.0 * 1.5           # kh = 0.47 on the 1.5-long computational box
    tb, tg = 0.18, np.pi / 6
    levels = O.build_hierarchy(2, n, tb, tg, 1 / 6, k=k)
    A = assemble(2, n, tb, tg, 1 / 6, phi=k * k)
    b = I.point_source(2, n)
    xs = spla.spsolve(A.tocsc(), b.ravel()).reshape(n, n)
    x = np.zeros_like(b)
    res = [np.linalg.norm(b)]
    for _ in range(12):
        x = x + O.vcycle(levels, b - levels[0].apply(x))
        res.append(np.linalg.norm(b - levels[0].apply(x)))
    assert np.linalg.norm(x - xs) / np.linalg.norm(xs) < 1e-8
    avg_rate = (res[-1] / res[0]) ** (1 / (len(res) - 1))
    assert avg_rate <= 0.25


# ------------------------------------------------------------------ FGMRES
def test_fgmres_matches_sparse_direct_solve():
    n, k = 63, 30.0
    levels = O.build_hierarchy(2, n, 0.3, TG, WF, k=k)
    b = I.random_source(2, n, 11)
    x, info = O.fgmres(levels[0].apply_h, lambda v: O.vcycle(levels, v), b, tol=1e-11)
    assert info.converged
    H = assemble(2, n, 0.0, phi=k * k)
    xs = spla.spsolve(H.tocsc(), b.ravel()).reshape(n, n)
    assert np.linalg.norm(x - xs) / np.linalg.norm(xs) < 1e-8
    # the estimate tracks the true residual and the history never increases
    assert info.rel_res_true < 1e-10
    assert all(b2 <= a2 * (1 + 1e-12) for a2, b2 in zip(info.history, info.history[1:]))


@pytest.mark.parametrize("restart", [0, 3])
def test_fgmres_residual_history_equals_bruteforce_minimum(restart):
    """With a fixed linear preconditioner P (a dense solve with M) flexible GMRES is GMRES
    on H P (Sec. 5 uses FGMRES only because the GMRES-smoothed cycle is not linear): after
    j iterations of a cycle started at x_c its residual is the minimum of ||b - H (x_c + P y)||
    over y in the Krylov space K_j(H P, r_c).  Every estimate of the history is checked
    against that minimum, computed by least squares over an orthonormalised Krylov basis
    from a sparse matrix assembled without the oracle; restarted cycles start where the
    previous one stopped."""
    n, k, tb = 7, 6.0, 0.3
    levels = O.build_hierarchy(2, n, tb, TG, WF, k=k)
    H = assemble(2, n, 0.0, phi=k * k).toarray()
    M = assemble(2, n, tb, phi=k * k).toarray()
    HP = H @ np.linalg.inv(M)
    b = crand((n, n), 31)
    maxit = 9

    def precond(v):
        return np.linalg.solve(M, v.ravel()).reshape(v.shape)

    _, info = O.fgmres(levels[0].apply_h, precond, b, tol=1e-14, restart=restart, maxit=maxit)
    assert info.iters == maxit and len(info.history) == maxit
    bn = np.linalg.norm(b)
    r = b.ravel().copy()
    cyc = restart if restart > 0 else maxit
    want = []
    for j in range(1, maxit + 1):
        jj = (j - 1) % cyc + 1          # iterations into the current cycle
        K = [r]
        for _ in range(jj - 1):
            K.append(HP @ K[-1])
        Q = np.linalg.qr(np.array(K).T)[0]
        y = np.linalg.lstsq(HP @ Q, r, rcond=None)[0]
        res = r - HP @ (Q @ y)
        want.append(np.linalg.norm(res) / bn)
        if jj == cyc:
            r = res                     # the next cycle starts from this residual
    got = np.array(info.history)
    assert np.all(np.abs(got - np.array(want)) <= 1e-7 * np.array(want) + 1e-13), (got, want)


def test_fgmres_with_the_exact_inverse_stops_after_one_iteration():
    """With P = H^{-1} the preconditioned operator is the identity: the first Arnoldi
    step breaks down (w - h v = 0) and x = H^{-1} b after one iteration (reading of the
    breakdown rule, Sec. 5's FGMRES)."""
    n, k = 7, 6.0
    levels = O.build_hierarchy(2, n, 0.3, TG, WF, k=k)
    H = assemble(2, n, 0.0, phi=k * k).toarray()
    b = crand((n, n), 41)
    x, info = O.fgmres(levels[0].apply_h, lambda v: np.linalg.solve(H, v.ravel()).reshape(v.shape), b,
                       tol=1e-14, maxit=20)
    assert info.iters == 1
    xs = np.linalg.solve(H, b.ravel()).reshape(n, n)
    assert np.linalg.norm(x - xs) <= 1e-12 * np.linalg.norm(xs)


def test_fgmres_restarted_reaches_tolerance():
    n, k = 31, 20.0
    levels = O.build_hierarchy(2, n, 0.3, TG, WF, k=k)
    b = I.random_source(2, n, 12)
    x, info = O.fgmres(levels[0].apply_h, lambda v: O.vcycle(levels, v), b, tol=1e-9, restart=4)
    assert info.converged and info.restarts >= 2
    assert np.linalg.norm(b - levels[0].apply_h(x)) / np.linalg.norm(b) <= 1e-9


@pytest.mark.parametrize("dim,n", [(2, 31), (3, 15)])
def test_manufactured_solution(dim, n):
    """u* quadratic in the complex coordinates of the ECS grid: the scheme is exact
    on it, so the discrete solution of H u = -Laplacian u* - phi u* is u* itself."""
    k = 7.0
    u, mlap = quad_manufactured(dim, n, 0.0)
    b = mlap - k * k * u
    levels = O.build_hierarchy(dim, n, 0.3, TG, WF, k=k)
    x, info = O.fgmres(levels[0].apply_h, lambda v: O.vcycle(levels, v), b, tol=1e-12)
    assert info.converged
    assert np.linalg.norm(x - u) / np.linalg.norm(u) < 1e-9


def test_zero_source_returns_zero():
    levels = O.build_hierarchy(2, 15, 0.3, TG, WF, k=5.0)
    b = np.zeros((15, 15), dtype=np.complex128)
    x, info = O.fgmres(levels[0].apply_h, lambda v: O.vcycle(levels, v), b, tol=1e-8)
    assert info.converged and info.iters == 0 and not np.any(x)
