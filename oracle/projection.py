"""CPU oracle of the projection framework for large parametrized Lyapunov
equations (paper §2.2: eqs. (EK_def) and (param_projected), the backward
error proposition, Algorithm 1).

TEST INFRASTRUCTURE. Only the test suite, the package smoke check and the
benchmark's CPU-baseline leg may import or call this module. The GPU library
never routes through it, and it shares no code with the library.

Convention. The library's API writes A(v) = A0 - U diag(v) V^T and
A(v)^T X + X A(v) = -G G^T. §2.2 works with the transposed matrices:

    A_p(v) = A0p - B_l D(v) B_r^T,   A0p = A0^T,  B_l = V,  B_r = U,

and with the change X_d(v) = X(v) - X0 from the seed solution
A0p X0 + X0 A0p^T = -G G^T, which solves eq. (Lyap_deltaX):

    A_p(v) X_d + X_d A_p(v)^T = P (I2 (x) D(v)) P^T,   P = [X0 B_r, B_l]
    (eq. (rhs_newexpression)), I2 (x) D = [[0, D], [D, 0]].

Steps, in the paper's order:

* One extended Krylov space for every v (eq. (EK_def)): block j of the
  orthonormal basis adds A0p^(j-1) P and A0p^(-j) P. The first block is an
  orthonormal basis of [P, A0p^{-1} P] (so P = V_1 G); each further block
  takes A0p times the first half and A0p^{-1} times the second half of the
  latest block, orthogonalised against all blocks by block Gram-Schmidt,
  twice (the construction of Simoncini 2007, which §2.2 cites).
  Solves with A0p reuse one stored LU factorisation (Assumption 3).
* T_m = V_m^T A0p V_m, B_{l,m} = V_m^T B_l, B_{r,m} = V_m^T B_r, written
  as their definitions.
* The projected equation (param_projected)
      (T_m - B_{l,m} D B_{r,m}^T) Y + Y (T_m - B_{l,m} D B_{r,m}^T)^T
          = E_1 G (I2 (x) D) G^T E_1^T
  by LAPACK's Bartels-Stewart solver (a library step; lyap_oracle's own
  solver is pinned against it).
* The backward error Delta_{m,v} by the backward error proposition (cheap:
  no n-sized work per v) and by its definition (the full n x n residual).
* f(v) = trace(E X0) + trace((V_m^T E V_m) Y_m(v)); for E = I the second
  term is trace(Y_m) (the trace identity at the end of §2.2).
* Algorithm 1: grow the space until every v meets the backward-error bound.

The paper assumes full-rank blocks and points to standard deflation
otherwise. The oracle deflates: a new direction whose size after
orthogonalisation is below RANK_TOL of its candidate's is dropped, the
halves of a block (A0p- and A0p^{-1}-directions) deflate separately, and an
empty block ends the space (the projected solution is then exact).
"""
from __future__ import annotations

import math

import numpy as np
import scipy.linalg as sla

from .lyap_oracle import lyap_solve, trace_product

# Directions of a new block whose norm after orthogonalisation falls below
# this fraction of the largest candidate column are already in the space.
RANK_TOL = 1e-13


def seed_quantities(A0, U, V, G, E, X0=None):
    """A0p, B_l, B_r, X0, P and f(X0) in the convention of §2.2.

    X0 may be given when it is already known (a closed form pinned
    separately); otherwise Bartels-Stewart solves the seed equation.
    """
    A0 = np.asarray(A0, dtype=np.float64)
    A0p = A0.T.copy()
    Bl = np.asarray(V, dtype=np.float64)
    Br = np.asarray(U, dtype=np.float64)
    G = np.asarray(G, dtype=np.float64)
    if X0 is None:
        X0 = lyap_solve(A0, G @ G.T)  # A0^T X0 + X0 A0 = -G G^T, i.e. A0p X0 + X0 A0p^T = -G G^T
    X0 = np.asarray(X0, dtype=np.float64)
    P = np.hstack([X0 @ Br, Bl])
    return dict(A0p=A0p, Bl=Bl, Br=Br, X0=X0, P=P, f0=trace_product(E, X0))


def i2_kron(v):
    """I2 (x) D(v) = [[0, D], [D, 0]] (eq. (rhs_newexpression))."""
    v = np.asarray(v, dtype=np.float64)
    k = v.size
    M = np.zeros((2 * k, 2 * k))
    M[:k, k:] = np.diag(v)
    M[k:, :k] = np.diag(v)
    return M


def _new_directions(W, blocks):
    """Orthonormal directions of Range(W) outside the span of ``blocks``.

    Block Gram-Schmidt against every block, twice, then an SVD: directions
    whose size after the projection is below RANK_TOL of the largest
    candidate column are already in the space and are dropped (deflation).
    """
    ref = max(np.linalg.norm(W, axis=0).max(initial=0.0), 1e-300)
    for _ in range(2):
        for Qb in blocks:
            if Qb.shape[1]:
                W = W - Qb @ (Qb.T @ W)
    if W.shape[1] == 0:
        return W
    Uw, sig, _ = np.linalg.svd(W, full_matrices=False)
    return Uw[:, sig > RANK_TOL * ref]


class ExtendedKrylov:
    """Orthonormal basis of EK_m(A0p, P), one block per expansion (eq. (EK_def)).

    Each block keeps its two halves apart: the directions reached by A0p
    (first ``split`` columns) and those reached by A0p^{-1}. The next block
    applies A0p to the first half and A0p^{-1} to the second, so a half that
    deflates stops growing while the other goes on.
    """

    def __init__(self, A0p, P):
        self.A = np.asarray(A0p, dtype=np.float64)
        self.n = self.A.shape[0]
        self.lu = sla.lu_factor(self.A)  # Assumption 3: one stored LU of A0
        P = np.asarray(P, dtype=np.float64)
        self.s = P.shape[1]
        Q1 = _new_directions(P, [])
        Q2 = _new_directions(sla.lu_solve(self.lu, P), [Q1])
        self.blocks = [np.hstack([Q1, Q2])]
        self.split = [Q1.shape[1]]
        self.G = self.blocks[0].T @ P  # P = V_1 G (P lies in the first half)

    @property
    def dim(self) -> int:
        return sum(b.shape[1] for b in self.blocks)

    def expand(self):
        """Append block j+1 from [A0p V_j^(1), A0p^{-1} V_j^(2)]."""
        last, sp = self.blocks[-1], self.split[-1]
        Q1 = _new_directions(self.A @ last[:, :sp], self.blocks)
        Q2 = _new_directions(sla.lu_solve(self.lu, last[:, sp:]), self.blocks + [Q1])
        self.blocks.append(np.hstack([Q1, Q2]))
        self.split.append(Q1.shape[1])

    def basis(self, m: int):
        """V_m: the first m blocks."""
        return np.hstack(self.blocks[:m])

    def ensure(self, blocks: int):
        while len(self.blocks) < blocks:
            self.expand()


def projected_matrices(ek: ExtendedKrylov, m: int, Bl, Br):
    """T_m, the last block row of the Arnoldi relation, B_{l,m}, B_{r,m}."""
    ek.ensure(m + 1)
    Vm = ek.basis(m)
    AV = ek.A @ Vm
    Tm = Vm.T @ AV
    Vnext = ek.blocks[m]
    Em_T = Vnext.T @ AV  # E_m^T underline(T)_m = V_{m+1}-block^T A0p V_m
    return dict(Vm=Vm, Tm=Tm, EmT=Em_T, Blm=Vm.T @ Bl, Brm=Vm.T @ Br)


def solve_projected(pm: dict, G, v):
    """Y_m(v) from the projected equation (param_projected)."""
    v = np.asarray(v, dtype=np.float64)
    M = pm["Tm"] - (pm["Blm"] * v[None, :]) @ pm["Brm"].T
    d = M.shape[0]
    E1G = np.zeros((d, G.shape[1]))
    E1G[: G.shape[0], :] = G
    Q = E1G @ i2_kron(v) @ E1G.T
    # M Y + Y M^T = Q: LAPACK's Bartels-Stewart (real Schur form, trsyl),
    # which lyap_oracle's own solver is pinned against
    return sla.solve_continuous_lyapunov(M, Q)


def offline_norms(A0p, Bl, Br):
    """||A0||_F, (B_r^T B_l) o (B_r^T B_l) and a = diag(B_r^T A0p B_l) (backward error proposition)."""
    BB = Br.T @ Bl
    return dict(normA0=np.linalg.norm(A0p), H=BB * BB, a=np.diag(Br.T @ A0p @ Bl).copy())


def backward_error_cheap(pm: dict, Y, G, v, off: dict):
    """Delta_{m,v} by the backward error proposition: no n-sized work."""
    v = np.asarray(v, dtype=np.float64)
    num = math.sqrt(2.0) * np.linalg.norm(pm["EmT"] @ Y)
    normA2 = off["normA0"] ** 2 + v @ off["H"] @ v - 2.0 * off["a"] @ v
    den = 2.0 * math.sqrt(max(normA2, 0.0)) * np.linalg.norm(Y) + np.linalg.norm(G @ i2_kron(v) @ G.T)
    return num / den


def backward_error_full(sq: dict, pm: dict, Y, v):
    """Delta_{m,v} from its definition, with the full n x n residual."""
    v = np.asarray(v, dtype=np.float64)
    Av = sq["A0p"] - (sq["Bl"] * v[None, :]) @ sq["Br"].T
    X = pm["Vm"] @ Y @ pm["Vm"].T
    rhs = sq["P"] @ i2_kron(v) @ sq["P"].T
    R = Av @ X + X @ Av.T - rhs
    return np.linalg.norm(R) / (2.0 * np.linalg.norm(Av) * np.linalg.norm(X) + np.linalg.norm(rhs))


def trace_value(sq: dict, pm: dict, Y, E):
    """f(v) = trace(E X0) + trace((V_m^T E V_m) Y_m)."""
    Vm = pm["Vm"]
    return sq["f0"] + trace_product(Vm.T @ np.asarray(E) @ Vm, Y)


def eksm_sweep(A0, U, V, G, E, vs, eps: float, m_max: int, X0=None):
    """Algorithm 1 over the ordered parameter set ``vs``.

    For m = 1, 2, ... (while m < m_max): build the next block, then go
    through the remaining v in order. A v whose backward error meets eps is
    evaluated and leaves the set; the first v that does not ends the pass
    and the space grows. Returns (f, m_used, delta) per v; v that never met
    eps keep f = nan and m_used = 0.
    """
    sq = seed_quantities(A0, U, V, G, E, X0)
    off = offline_norms(sq["A0p"], sq["Bl"], sq["Br"])
    ek = ExtendedKrylov(sq["A0p"], sq["P"])
    vs = np.asarray(vs, dtype=np.float64)
    f = np.full(len(vs), np.nan)
    m_used = np.zeros(len(vs), dtype=int)
    delta = np.full(len(vs), np.nan)
    remaining = list(range(len(vs)))
    m = 1
    while m < m_max and remaining:
        pm = projected_matrices(ek, m, sq["Bl"], sq["Br"])
        while remaining:
            i = remaining[0]
            Y = solve_projected(pm, ek.G, vs[i])
            d = backward_error_cheap(pm, Y, ek.G, vs[i], off)
            if d <= eps:
                f[i] = trace_value(sq, pm, Y, E)
                m_used[i] = m
                delta[i] = d
                remaining.pop(0)
            else:
                break
        m += 1
    return f, m_used, delta
