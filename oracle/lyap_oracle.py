"""CPU oracle for f(v) = trace(E X(v)) of parametrized Lyapunov equations.

TEST INFRASTRUCTURE. Only the test suite, the package smoke check and the
benchmark's CPU-baseline leg may import or call this module. The GPU library
never routes through it, and it shares no code with the library.

What it computes (paper §1, eqs. (Ljap jdba 1) and (formA), written in the
transposed convention of the library's API):

    A(v) = A0 - U diag(v) V^T,
    A(v)^T X + X A(v) = -G G^T,
    f(v) = trace(E X(v)).

The paper's method (§2.1) reaches the exact solution of this equation: the
Sherman-Morrison-Woodbury split and the recycled Krylov solve only change how
X(v) is obtained. So the oracle is the definition itself, solved plainly for
every v, in float64:

* n <= 8: the Kronecker form (I (x) A^T + A^T (x) I) vec X = -vec(GG^T) by a
  dense LU (the brute-force reading of the Kronecker equations of §2.1);
* exact rational arithmetic (``fractions``) for rational input at n <= 4;
* otherwise Bartels-Stewart (cited in §1 as the naive per-v solver): a
  complex Schur form A^T = Z T Z^H (library step), the transformed equation
  T Y + Y T^H = -Z^H C Z solved column by column from the last column
  backwards with triangular solves, then X = Z Y Z^H.

The gradient uses the adjoint equation A Y + Y A^T = -E (E symmetrised):
df/dv_i = -2 V_i^T Y X U_i, which follows from differentiating the
equation above with dA/dv_i = -U_i V_i^T.

Pins (tests/test_oracle.py): single-oscillator closed forms, the paper's
closed-form seed solution for the modal chain (§3.1, with its (1,1) entry
corrected), a scalar case, brute force and exact arithmetic on tiny inputs,
orthogonal-similarity and scaling invariance, duality, symmetry and
positive semi-definiteness, and the gradient against central differences.
"""
from __future__ import annotations

import math
from fractions import Fraction

import numpy as np
import scipy.linalg as sla

KRON_MAX_N = 8


def param_matrix(A0, U, V, v):
    """A(v) = A0 - U diag(v) V^T (eq. (formA), transposed convention)."""
    v = np.asarray(v, dtype=np.float64)
    return np.asarray(A0, dtype=np.float64) - (np.asarray(U) * v[None, :]) @ np.asarray(V).T


def lyap_kron(A, C):
    """Solve A^T X + X A = -C from its n^2 x n^2 Kronecker form (dense LU)."""
    A = np.asarray(A, dtype=np.float64)
    n = A.shape[0]
    I = np.eye(n)
    K = np.kron(I, A.T) + np.kron(A.T, I)  # acts on column-major vec(X)
    x = np.linalg.solve(K, -np.asarray(C, dtype=np.float64).ravel(order="F"))
    return x.reshape((n, n), order="F")


def lyap_exact(A, C):
    """Same Kronecker system in exact rational arithmetic (Gauss-Jordan).

    ``A`` and ``C`` are nested lists (or arrays) of ints/Fractions; returns an
    n x n list of Fractions. Meant for n <= 4.
    """
    n = len(A)
    A = [[Fraction(A[i][j]) for j in range(n)] for i in range(n)]
    C = [[Fraction(C[i][j]) for j in range(n)] for i in range(n)]
    N = n * n
    # unknown index of X[i][j] in column-major vec: j*n + i
    M = [[Fraction(0)] * (N + 1) for _ in range(N)]
    for i in range(n):
        for j in range(n):
            row = j * n + i
            # (A^T X)_{ij} = sum_l A[l][i] X[l][j]
            for l in range(n):
                M[row][j * n + l] += A[l][i]
            # (X A)_{ij} = sum_l X[i][l] A[l][j]
            for l in range(n):
                M[row][l * n + i] += A[l][j]
            M[row][N] = -C[i][j]
    for col in range(N):
        piv = next(r for r in range(col, N) if M[r][col] != 0)
        M[col], M[piv] = M[piv], M[col]
        p = M[col][col]
        M[col] = [x / p for x in M[col]]
        for r in range(N):
            if r != col and M[r][col] != 0:
                f = M[r][col]
                M[r] = [a - f * b for a, b in zip(M[r], M[col])]
    X = [[Fraction(0)] * n for _ in range(n)]
    for i in range(n):
        for j in range(n):
            X[i][j] = M[j * n + i][N]
    return X


def lyap_bartels_stewart(A, C):
    """Solve A^T X + X A = -C for real A, C by Bartels-Stewart.

    With the complex Schur form A^T = Z T Z^H (T upper triangular) and real A,
    A = Z T^H Z^H, so Y = Z^H X Z satisfies T Y + Y T^H = -F, F = Z^H C Z.
    Column j of Y T^H is sum_{l >= j} conj(T[j, l]) Y[:, l]; hence
        (T + conj(T[j, j]) I) Y[:, j] = -F[:, j] - sum_{l > j} conj(T[j, l]) Y[:, l],
    solved for j = n-1, ..., 0.
    """
    A = np.asarray(A, dtype=np.float64)
    C = np.asarray(C, dtype=np.float64)
    n = A.shape[0]
    T, Z = sla.schur(A.T.astype(np.complex128), output="complex")
    F = Z.conj().T @ C @ Z
    Y = np.zeros((n, n), dtype=np.complex128)
    d = np.diag(T).copy()
    Ts = T.copy()
    for j in range(n - 1, -1, -1):
        rhs = -F[:, j]
        if j + 1 < n:
            rhs = rhs - Y[:, j + 1 :] @ np.conj(T[j, j + 1 :])
        np.fill_diagonal(Ts, d + np.conj(d[j]))  # Ts = T + conj(T[j, j]) I
        Y[:, j] = sla.solve_triangular(Ts, rhs, lower=False)
    X = Z @ Y @ Z.conj().T
    return X.real


def lyap_solve(A, C, method: str = "auto"):
    if method == "auto":
        method = "kron" if A.shape[0] <= KRON_MAX_N else "bs"
    if method == "kron":
        return lyap_kron(A, C)
    if method == "bs":
        return lyap_bartels_stewart(A, C)
    raise ValueError(method)


def trace_product(E, X):
    """trace(E X) = sum_ij E_ji X_ij, summed with math.fsum."""
    return math.fsum((np.asarray(E).T * np.asarray(X)).ravel().tolist())


def solve(A0, U, V, G, E, v, method: str = "auto"):
    """Return (f, X) for one parameter vector v."""
    A = param_matrix(A0, U, V, v)
    C = np.asarray(G) @ np.asarray(G).T
    X = lyap_solve(A, C, method)
    return trace_product(E, X), X


def trace_EX(A0, U, V, G, E, v, method: str = "auto"):
    return solve(A0, U, V, G, E, v, method)[0]


def gradient(A0, U, V, G, E, v, method: str = "auto"):
    """Return (f, df/dv) via the adjoint equation A Y + Y A^T = -sym(E)."""
    A = param_matrix(A0, U, V, v)
    C = np.asarray(G) @ np.asarray(G).T
    X = lyap_solve(A, C, method)
    Es = 0.5 * (np.asarray(E) + np.asarray(E).T)
    Y = lyap_solve(A.T, Es, method)  # (A^T)^T Y + Y A^T = -Es
    U = np.asarray(U)
    V = np.asarray(V)
    g = np.array([-2.0 * (V[:, i] @ Y @ X @ U[:, i]) for i in range(U.shape[1])])
    return trace_product(E, X), g


def check_solution(A, C, X):
    """Diagnostics of one solve: relative asymmetry, backward error (the
    normwise form used in §2.2's backward-error proposition) and the smallest
    eigenvalue of sym(X) relative to ||X||."""
    nx = np.linalg.norm(X)
    asym = np.linalg.norm(X - X.T) / nx
    R = A.T @ X + X @ A + C
    berr = np.linalg.norm(R) / (2 * np.linalg.norm(A) * nx + np.linalg.norm(C))
    mineig = np.linalg.eigvalsh(0.5 * (X + X.T)).min() / nx
    return dict(asym=asym, backward_error=berr, min_eig_rel=mineig)


def sweep(problem, vs, method: str = "auto"):
    """f(v) for every row of ``vs`` (plain loop, one solve per v)."""
    return np.array(
        [trace_EX(problem.A0, problem.U, problem.V, problem.G, problem.E, v, method) for v in vs]
    )
