"""The delayed re-orthogonalisation recurrence of the mixed subdomain cycles
(k_dcgs_dots / k_dcgs_update), written out in numpy exactly as the kernels
form it, against the textbook Arnoldi process with two classical Gram-Schmidt
passes: both must build the same Krylov space, so flexible GMRES over either
reaches the same residual at every step.  A dropped 1/gamma in the next
vector (norms growing geometrically), a wrong sign in the coefficients or a
missing gamma_{j-1} in the lagged Hessenberg column fails here.  Plain numpy,
no GPU."""
import numpy as np
import pytest

pytestmark = pytest.mark.filterwarnings("ignore::RuntimeWarning")


def _problem(n=300, seed=0):
    r = np.random.default_rng(seed)
    A = r.standard_normal((n, n)) / np.sqrt(n) + 2 * np.eye(n) + 1j * r.standard_normal((n, n)) / np.sqrt(n)
    M = np.diag(1 + r.random(n))
    b = r.standard_normal(n) + 1j * r.standard_normal(n)
    return A, M, b


def _residuals(H, Z, A, b, ks):
    beta = np.linalg.norm(b)
    out = []
    for k in ks:
        e1 = np.zeros(k + 1, complex)
        e1[0] = beta
        y = np.linalg.lstsq(H[:k + 1, :k], e1, rcond=None)[0]
        out.append(np.linalg.norm(b - A @ (Z[:k].T @ y)) / beta)
    return np.array(out)


def dcgs_kernels(A, M, b, m, dtype):
    """Steps 0..m as the kernels run them: u_j in basis slot j, z_j = M u_j,
    w = A z_j; one dot pass (s, bb, c1, c2); gamma_j, d_j; column j-1 final
    with gamma_{j-1}; the update pass writes v_j and u_{j+1}."""
    n = len(b)
    U = np.zeros((m + 1, n), dtype)
    Z = np.zeros((m, n), dtype)
    H = np.zeros((m + 1, m), complex)
    U[0] = (b / np.linalg.norm(b)).astype(dtype)
    pre, gprev = None, 1.0
    for j in range(m + 1):
        u = U[j].copy()
        last = j == m
        if not last:
            Z[j] = (M @ u).astype(dtype)
            w = (A @ Z[j]).astype(dtype)
        else:
            w = np.zeros(n, dtype)
        V = U[:j]
        s, bb = V.conj() @ u, V.conj() @ w
        c1, c2 = np.vdot(u, u).real, np.vdot(u, w)
        gamma = 1.0 if j == 0 else np.sqrt(c1 - np.sum(np.abs(s) ** 2))
        if j > 0:
            H[:j, j - 1] = pre + gprev * s
            H[j, j - 1] = gprev * gamma
        if last:
            break
        d = (c2 - np.vdot(s, bb)) / gamma
        pre, gprev = np.concatenate([bb, [d]]), gamma
        alpha = -s / gamma
        beta_k = -(bb - s * d / gamma) / gamma
        U[j] = (u / gamma + alpha @ V).astype(dtype)
        U[j + 1] = (w / gamma - (d / gamma ** 2) * u + beta_k @ V).astype(dtype)
    return H, Z, U


def cgs2(A, M, b, m, dtype):
    n = len(b)
    V = np.zeros((m + 1, n), dtype)
    Z = np.zeros((m, n), dtype)
    H = np.zeros((m + 1, m), complex)
    V[0] = (b / np.linalg.norm(b)).astype(dtype)
    for j in range(m):
        Z[j] = (M @ V[j]).astype(dtype)
        w = (A @ Z[j]).astype(dtype)
        h1 = V[:j + 1].conj() @ w
        w = (w - h1 @ V[:j + 1]).astype(dtype)
        h2 = V[:j + 1].conj() @ w
        w = (w - h2 @ V[:j + 1]).astype(dtype)
        H[:j + 1, j] = h1 + h2
        H[j + 1, j] = np.linalg.norm(w)
        V[j + 1] = (w / H[j + 1, j]).astype(dtype)
    return H, Z, V


@pytest.mark.parametrize("dtype,tol", [(np.complex128, 1e-9), (np.complex64, 2e-2)])
def test_same_residual_history_as_cgs2(dtype, tol):
    A, M, b = _problem()
    m = 40
    ks = [5, 10, 20, 30, 40]
    Hd, Zd, _ = dcgs_kernels(A, M, b, m, dtype)
    Hc, Zc, _ = cgs2(A, M, b, m, dtype)
    rd, rc = _residuals(Hd, Zd, A, b, ks), _residuals(Hc, Zc, A, b, ks)
    assert rc[-1] < 1e-5                       # the problem converges within the window
    assert np.all(np.abs(rd / rc - 1) <= tol), (rd, rc)


def test_basis_stays_orthonormal_and_next_vectors_bounded():
    A, M, b = _problem(seed=1)
    m = 40
    H, Z, U = dcgs_kernels(A, M, b, m, np.complex64)
    V = U[:m].astype(np.complex128)
    assert np.linalg.norm(V.conj() @ V.T - np.eye(m)) < 1e-5
    # |u_{j+1}| is about h_{j+1,j} (the division by gamma_j): bounded by ||A M||
    assert np.linalg.norm(U[m]) < 10 * np.linalg.norm(A @ M, 2)
    # the flexible Arnoldi relation A Z = V H holds for every finished column
    lhs = A @ Z[:m - 1].T
    rhs = U[:m].T.astype(np.complex128) @ H[:m, :m - 1]
    assert np.linalg.norm(lhs - rhs) <= 1e-5 * np.linalg.norm(lhs)


def test_without_the_gamma_scaling_the_norms_grow():
    """The recurrence without 1/gamma_j in u_{j+1} (the next vector keeps the
    scale of w): its norms grow geometrically, which is what the scaling
    prevents."""
    A, M, b = _problem(seed=2)
    n, m = len(b), 30
    U = np.zeros((m + 1, n), complex)
    U[0] = b / np.linalg.norm(b)
    norms = []
    for j in range(m):
        u = U[j].copy()
        w = A @ (M @ u)
        V = U[:j]
        s, bb = V.conj() @ u, V.conj() @ w
        gamma = 1.0 if j == 0 else np.sqrt(np.vdot(u, u).real - np.sum(np.abs(s) ** 2))
        d = (np.vdot(u, w) - np.vdot(s, bb)) / gamma
        U[j] = u / gamma - (s / gamma) @ V
        U[j + 1] = w - (d / gamma) * u - (bb - s * d / gamma) @ V
        norms.append(np.linalg.norm(U[j + 1]))
    assert norms[-1] > 1e6 * norms[0]
