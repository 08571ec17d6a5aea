"""Host model of the Krylov refinement's algebra (flexible GMRES as the library's
refined_solve runs it): right preconditioning by an inexact, slightly nonlinear inverse,
classical Gram-Schmidt applied twice, the complex Givens rotation
    c = |a| / nu,  s = (a / |a|) conj(b) / nu,  rho = (a / |a|) nu,  nu = sqrt(|a|^2 + |b|^2),
restarts every m steps and back substitution.  Checked against numpy's solve of the same
complex system: the rotation zeroes the subdiagonal, the residual estimate |g_{j+1}| equals
the true residual of the update, and the iteration reaches FP64-level accuracy where plain
refinement with the same preconditioner stalls."""
import numpy as np


def givens(a, b):
    if a == 0:
        return 0.0, 1.0 + 0j, b
    ph = a / abs(a)
    nu = np.sqrt(abs(a) ** 2 + abs(b) ** 2)
    return abs(a) / nu, ph * np.conj(b) / nu, ph * nu


def fgmres(A, b, x, prec, m=16, max_steps=60, tol=1e-13, check=None):
    n = b.size
    bnorm = np.linalg.norm(b)
    used, prev = 0, 0.0
    restart = 0
    while used < max_steps:
        r = b - A @ x
        worst = np.linalg.norm(r) / bnorm
        if worst <= tol or (restart > 0 and worst > 0.5 * prev):
            break
        prev = worst
        beta = np.linalg.norm(r)
        V = np.zeros((m + 1, n), complex)
        Z = np.zeros((m, n), complex)
        H = np.zeros((m + 1, m), complex)
        g = np.zeros(m + 1, complex)
        cs, sn = np.zeros(m), np.zeros(m, complex)
        V[0] = r / beta
        g[0] = beta
        k = 0
        for j in range(m):
            if used >= max_steps:
                break
            Z[j] = prec(V[j])
            used += 1
            w = A @ Z[j]
            h1 = V[: j + 1].conj() @ w
            w = w - h1 @ V[: j + 1]
            h2 = V[: j + 1].conj() @ w
            w = w - h2 @ V[: j + 1]
            hn = np.linalg.norm(w)
            H[: j + 1, j] = h1 + h2
            H[j + 1, j] = hn
            for i in range(j):
                a, c = H[i, j], H[i + 1, j]
                H[i, j] = cs[i] * a + sn[i] * c
                H[i + 1, j] = -np.conj(sn[i]) * a + cs[i] * c
            cs[j], sn[j], H[j, j] = givens(H[j, j], H[j + 1, j])
            H[j + 1, j] = 0
            g[j + 1] = -np.conj(sn[j]) * g[j]
            g[j] = cs[j] * g[j]
            k = j + 1
            if hn > 0:
                V[j + 1] = w / hn
            if check is not None:
                check(A, b, x, Z[:k], H[:k, :k], g[: k + 1])
            if abs(g[j + 1]) <= 0.5 * tol * bnorm or hn == 0:
                break
        y = np.zeros(k, complex)
        for i in range(k - 1, -1, -1):
            t = g[i] - H[i, i + 1:k] @ y[i + 1:k]
            y[i] = t / H[i, i] if H[i, i] != 0 else 0
        x = x + y @ Z[:k]
        restart += 1
    return x, used, np.linalg.norm(b - A @ x) / bnorm


def _system(n, seed):
    rng = np.random.default_rng(seed)
    # a complex symmetric, indefinite system A = Q diag(lam) Q^T with real orthogonal Q
    Q, _ = np.linalg.qr(rng.standard_normal((n, n)))
    lam = rng.uniform(0.5, 2.0, n) * np.exp(1j * rng.uniform(0, np.pi, n))
    b = rng.standard_normal(n) + 1j * rng.standard_normal(n)
    return (Q * lam) @ Q.T, b, Q, lam


def _fp32_inverse(Q, lam, bad):
    # an inverse that resolves a few modes poorly (lam_i taken as lam_i f_i: the error
    # contraction 1 - 1/f_i of plain refinement is near 1 in modulus there), applied in
    # single precision (slightly nonlinear)
    mu = lam.copy()
    mu[: len(bad)] *= np.asarray(bad)
    P32 = ((Q / mu) @ Q.T).astype(np.complex64)
    return lambda v: (P32 @ v.astype(np.complex64)).astype(np.complex128)


def test_givens_zeroes_the_subdiagonal_and_keeps_the_norm():
    rng = np.random.default_rng(0)
    for _ in range(100):
        a = complex(*rng.standard_normal(2)) * 10 ** rng.uniform(-3, 3)
        b = abs(rng.standard_normal()) * 10 ** rng.uniform(-3, 3)
        c, s, rho = givens(a, b)
        G = np.array([[c, s], [-np.conj(s), c]])
        out = G @ np.array([a, b])
        assert abs(out[1]) <= 1e-12 * abs(rho)
        assert abs(out[0] - rho) <= 1e-12 * abs(rho)
        assert abs(G @ G.conj().T - np.eye(2)).max() < 1e-12


def test_residual_estimate_equals_the_true_residual():
    A, b, Q, lam = _system(80, 1)
    prec = _fp32_inverse(Q, lam, [0.5, 3.0])

    def check(A, b, x, Z, R, g):
        k = R.shape[0]
        y = np.linalg.solve(np.triu(R), g[:k])
        true = np.linalg.norm(b - A @ (x + y @ Z))
        assert abs(true - abs(g[k])) <= 1e-8 * np.linalg.norm(b) + 1e-6 * true

    fgmres(A, b, np.zeros_like(b), prec, m=16, max_steps=16, check=check)


def test_fgmres_converges_where_plain_refinement_stalls():
    A, b, Q, lam = _system(120, 2)
    prec = _fp32_inverse(Q, lam, [0.5, 0.51 + 0.1j, 0.52 - 0.08j])
    x_ref = np.linalg.solve(A, b)
    # plain refinement with the same preconditioner stalls well above the tolerance
    x = prec(b)
    ratios = []
    for _ in range(30):
        r = b - A @ x
        ratios.append(np.linalg.norm(r) / np.linalg.norm(b))
        x = x + prec(r)
    assert min(ratios) > 1e-8
    x, used, rel = fgmres(A, b, np.zeros_like(b), prec, m=16, max_steps=60)
    assert rel <= 1e-13, (rel, used)
    assert np.linalg.norm(x - x_ref) <= 1e-9 * np.linalg.norm(x_ref)
