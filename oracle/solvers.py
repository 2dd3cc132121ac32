"""Textbook Krylov and Chebyshev iterations (oracle; test infrastructure).

Sec. 5.1: the linear systems are solved by preconditioned CG with a
matrix-free operator; for singular (all-Neumann or periodic) Poisson problems
the right-hand side and every operator product are projected onto the space of
vectors with zero mean; the Chebyshev iteration needs only the matrix diagonal
and operator products, with eigenvalue estimates from an initial CG run.
"""
import numpy as np


def project_mean(v):
    """Projection onto vectors with zero (Euclidean) mean: v - (1^T v / N) 1."""
    return v - v.mean()


def cg(apply, b, x0=None, rtol=1e-10, maxit=10000, precond=None, zero_mean=False, flexible=False):
    """Preconditioned CG (Hestenes-Stiefel form); ``flexible`` uses the
    Polak-Ribiere beta  z_new^T (r_new - r_old) / (z_old^T r_old).

    Stops when ||b - A x||_2 <= rtol ||b||_2 (the recursively updated residual).
    Returns (x, iterations, relative residual)."""
    b = np.asarray(b, dtype=np.float64)
    if zero_mean:
        b = project_mean(b)
    x = np.zeros_like(b) if x0 is None else np.array(x0, dtype=np.float64)

    def A(v):
        y = apply(v)
        return project_mean(y) if zero_mean else y

    M = precond if precond is not None else (lambda r: r.copy())
    r = b - A(x)
    bnorm = np.linalg.norm(b)
    if bnorm == 0.0:
        return x, 0, 0.0
    if np.linalg.norm(r) <= rtol * bnorm:
        return x, 0, np.linalg.norm(r) / bnorm
    z = M(r)
    p = z.copy()
    rz = r @ z
    for it in range(1, maxit + 1):
        Ap = A(p)
        pAp = p @ Ap
        if not pAp > 0.0:
            raise FloatingPointError("CG breakdown: p^T A p <= 0")
        alpha = rz / pAp
        x += alpha * p
        r_old = r.copy() if flexible else None
        r -= alpha * Ap
        relres = np.linalg.norm(r) / bnorm
        if relres <= rtol:
            return x, it, relres
        z = M(r)
        rz_new = r @ z
        beta = ((r - r_old) @ z) / rz if flexible else rz_new / rz
        rz = rz_new
        p = z + beta * p
    return x, maxit, relres


def lanczos_max_eig(apply, diag, v0, steps=20):
    """Largest eigenvalue of D^-1 A from ``steps`` Jacobi-PCG iterations on A x = v0
    (Lanczos tridiagonal from the CG coefficients, Sec. 5.1: eigenvalue estimates
    through an initial CG solution)."""
    x = np.zeros_like(v0)
    r = v0.copy()
    z = r / diag
    p = z.copy()
    rz = r @ z
    alphas, betas = [], []
    for _ in range(steps):
        Ap = apply(p)
        pAp = p @ Ap
        if pAp <= 0:
            break
        alpha = rz / pAp
        x += alpha * p
        r -= alpha * Ap
        z = r / diag
        rz_new = r @ z
        beta = rz_new / rz
        alphas.append(alpha)
        betas.append(beta)
        rz = rz_new
        p = z + beta * p
        if rz <= 0:
            break
    m = len(alphas)
    T = np.zeros((m, m))
    for i in range(m):
        T[i, i] = 1.0 / alphas[i] + (betas[i - 1] / alphas[i - 1] if i > 0 else 0.0)
        if i + 1 < m:
            T[i, i + 1] = T[i + 1, i] = np.sqrt(betas[i]) / alphas[i]
    return float(np.linalg.eigvalsh(T).max())


def chebyshev(apply, diag, b, degree, lmin, lmax):
    """``degree`` steps of the Chebyshev iteration for A x = b preconditioned by
    D = diag(A), starting from x = 0, with the spectrum of D^-1 A taken in
    [lmin, lmax] (three-term recurrence of the Chebyshev acceleration, Saad,
    "Iterative methods for sparse linear systems", Alg. 12.1; Varga).  The first
    step needs no operator product, so ``degree`` steps use degree-1 products."""
    theta = 0.5 * (lmax + lmin)
    delta = 0.5 * (lmax - lmin)
    sigma = theta / delta
    rho = 1.0 / sigma
    r = b.copy()
    d = (r / diag) / theta
    x = np.zeros_like(b)
    for step in range(degree):
        x = x + d
        if step == degree - 1:
            break
        r = r - apply(d)
        rho_new = 1.0 / (2.0 * sigma - rho)
        d = rho_new * rho * d + (2.0 * rho_new / delta) * (r / diag)
        rho = rho_new
    return x


def chebyshev_from(apply, diag, b, x0, degree, lmin, lmax):
    """``degree`` Chebyshev steps for A x = b preconditioned by D = diag(A),
    from the initial guess x0 (None: zero; then the first step needs no
    operator product).  Same recurrence as ``chebyshev``; with x0 the first
    residual is b - A x0."""
    theta = 0.5 * (lmax + lmin)
    delta = 0.5 * (lmax - lmin)
    sigma = theta / delta
    rho = 1.0 / sigma
    if x0 is None:
        x = np.zeros_like(b)
        r = b.copy()
    else:
        x = np.array(x0, dtype=np.float64)
        r = b - apply(x)
    d = (r / diag) / theta
    for step in range(degree):
        x = x + d
        if step == degree - 1:
            break
        r = r - apply(d)
        rho_new = 1.0 / (2.0 * sigma - rho)
        d = rho_new * rho * d + (2.0 * rho_new / delta) * (r / diag)
        rho = rho_new
    return x
