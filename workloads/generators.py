"""Synthetic problem generators (paper §3 application models, §4 sweeps).

Every generator returns a :class:`Problem` in the convention used by the
library and the oracle:

    A(v)^T X + X A(v) = -G G^T,     A(v) = A0 - U diag(v) V^T,
    f(v) = trace(E X(v)).

The paper writes the same family transposed (§1, eqs. (Ljap jdba 1) and
(formA)): A_p(v) X + X A_p(v)^T = -Q with A_p = A0^T, B_l = V, B_r = U,
Q = G G^T. For the damped vibrational system the energy integral of §3.1
yields the form above directly with A(v) the phase-space matrix of eq.
(MatrixA).

Nothing here solves a Lyapunov equation; the only linear algebra is the
modal transformation that defines the application model (eq. (MatrixPhi)).
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np
import scipy.linalg as sla


@dataclass
class Problem:
    """One seed: fixed matrices of a parametrized Lyapunov family.

    Arrays are float64. ``A0`` is n x n, ``U`` and ``V`` are n x k, ``G`` is
    n x g and ``E`` is n x n (symmetric).
    """

    name: str
    A0: np.ndarray
    U: np.ndarray
    V: np.ndarray
    G: np.ndarray
    E: np.ndarray
    meta: dict = field(default_factory=dict)

    @property
    def n(self) -> int:
        return self.A0.shape[0]

    @property
    def k(self) -> int:
        return self.U.shape[1]

    @property
    def g(self) -> int:
        return self.G.shape[1]


def config_rngs(count: int = 5):
    """Independent generators per workload: SeedSequence(0) spawned."""
    return [np.random.default_rng(s) for s in np.random.SeedSequence(0).spawn(count)]


def haar_orthogonal(rng: np.random.Generator, n: int) -> np.ndarray:
    """Haar-distributed orthogonal matrix (QR of a Gaussian, sign-fixed)."""
    z = rng.standard_normal((n, n))
    q, r = np.linalg.qr(z)
    q *= np.sign(np.diag(r))[None, :]
    return q


def generic_dense(p: Problem, rng: np.random.Generator) -> Problem:
    """Apply an orthogonal similarity S to (A0, U, V, G, E).

    f(v) is unchanged (X -> S X S^T), but the block structure of the modal
    matrices is hidden, so a solver cannot exploit it.
    """
    S = haar_orthogonal(rng, p.n)
    return Problem(
        name=p.name + "+dense",
        A0=S @ p.A0 @ S.T,
        U=S @ p.U,
        V=S @ p.V,
        G=S @ p.G,
        E=S @ p.E @ S.T,
        meta=dict(p.meta, similarity="haar"),
    )


def mass_spring_chain(
    springs,
    alpha: float,
    dampers,
    masses=None,
    energy_modes: int | None = None,
) -> Problem:
    """Damped chain of m masses between two fixed walls (§3.1).

    * ``springs``: m+1 stiffnesses k_0..k_m; spring i joins mass i-1 and i
      (walls at both ends), so K is tridiagonal.
    * Internal damping is the critical fraction of eq. (Ccrit), which the
      modal basis of eq. (MatrixPhi) turns into alpha*Omega.
    * ``dampers``: 1-based mass indices of grounded external dampers, so
      B = [e_i1, ..., e_ik] and C_ext(v) = B diag(v) B^T (eq. (Cext)).
    * State y = [Omega Phi^{-1} x ; Phi^{-1} xdot] (eq. (MatrixA)):
      A0 = [[0, Omega], [-Omega, -alpha Omega]], U = V = [0 ; Phi^T B].
    * G = I. E = I, or, with ``energy_modes = s``, the projector onto the
      first s modal displacements (a reading of eq. (matrix Z)).
    """
    springs = np.asarray(springs, dtype=np.float64)
    m = springs.size - 1
    if masses is None:
        masses = np.ones(m)
    masses = np.asarray(masses, dtype=np.float64)
    K = np.zeros((m, m))
    for i in range(m):
        K[i, i] = springs[i] + springs[i + 1]
        if i + 1 < m:
            K[i, i + 1] = K[i + 1, i] = -springs[i + 1]
    minv_half = 1.0 / np.sqrt(masses)
    w2, S = np.linalg.eigh(minv_half[:, None] * K * minv_half[None, :])
    Phi = minv_half[:, None] * S  # Phi^T K Phi = Omega^2, Phi^T M Phi = I
    omega = np.sqrt(w2)
    n = 2 * m
    A0 = np.zeros((n, n))
    A0[:m, m:] = np.diag(omega)
    A0[m:, :m] = -np.diag(omega)
    A0[m:, m:] = -alpha * np.diag(omega)
    k = len(dampers)
    B = np.zeros((m, k))
    for c, d in enumerate(dampers):
        if not 1 <= d <= m:
            raise ValueError("damper position out of range")
        B[d - 1, c] = 1.0
    U = np.zeros((n, k))
    U[m:, :] = Phi.T @ B
    E = np.eye(n)
    if energy_modes is not None:
        E = np.zeros((n, n))
        E[np.arange(energy_modes), np.arange(energy_modes)] = 1.0
    return Problem(
        name=f"chain{m}",
        A0=A0,
        U=U,
        V=U.copy(),
        G=np.eye(n),
        E=E,
        meta=dict(omega=omega, alpha=alpha, dampers=list(dampers), masses=m),
    )


def two_row_masses(d: int) -> np.ndarray:
    """Masses of Ex. 1's two-row system, eq. (mass-Config), as printed for
    d = 1000: m_i = (2d + 1 - 2i)/10 for i <= 500, (i - 500)/10 + 100 for
    501 <= i <= 1000, 160 for 1001 <= i <= 2d (the printed range starts at
    1000, which the second range already covers), and m_{2d+1} = 175."""
    i = np.arange(1, 2 * d + 1, dtype=np.float64)
    m = np.where(i <= 500, (2 * d + 1 - 2 * i) / 10.0, np.where(i <= 1000, (i - 500) / 10.0 + 100.0, 160.0))
    m = np.append(m, 175.0)
    if np.any(m <= 0):
        raise ValueError("eq. (mass-Config) gives non-positive masses for this d")
    return m


def two_row_system(d: int, i1: int, i2: int, s: int, alpha: float = 0.04,
                   stiffness=(40.0, 20.0, 30.0)) -> Problem:
    """Ex. 1: two rows of d masses joined to a last mass (2d + 1 masses).

    * K: row r has springs of stiffness k_r, with the first mass of the row
      tied to the wall and the last tied to mass 2d + 1, which a spring k_3
      ties to the wall (the block matrix printed with the example).
    * Critical internal damping (eq. (Ccrit)), modal state of eq. (MatrixA):
      A_p = [[0, Omega], [-Omega, -alpha Omega]].
    * Dampers, eq. (damping-geometry): B = [e_i1, e_(i1+d/10) - e_(i1+d/10+d),
      e_i2] (1-based mass indices), B_l = B_r = [0; Phi^T B].
    * Q = eq. (matrix Z) with s modes: 1/(2s) on the first s modal
      displacements and velocities. E = I (average total energy = trace X).

    The paper writes A_p X + X A_p^T = -Q; the API's A(v)^T X + X A(v) = -G G^T
    takes A0 = A_p^T, U = B_r, V = B_l and G G^T = Q.
    """
    if d % 10:
        raise ValueError("d must be a multiple of 10 (damper offset d/10)")
    k1, k2, k3 = stiffness
    masses = two_row_masses(d)
    nm = 2 * d + 1
    K = np.zeros((nm, nm))
    for r, kr in ((0, k1), (1, k2)):
        o = r * d
        for i in range(d):
            K[o + i, o + i] = 2.0 * kr
            if i + 1 < d:
                K[o + i, o + i + 1] = K[o + i + 1, o + i] = -kr
        K[o + d - 1, nm - 1] = K[nm - 1, o + d - 1] = -kr
    K[nm - 1, nm - 1] = k1 + k2 + k3
    w2, Phi = sla.eigh(K, np.diag(masses))  # Phi^T K Phi = Omega^2, Phi^T M Phi = I, ascending
    omega = np.sqrt(w2)
    n = 2 * nm
    Ap = np.zeros((n, n))
    Ap[:nm, nm:] = np.diag(omega)
    Ap[nm:, :nm] = -np.diag(omega)
    Ap[nm:, nm:] = -alpha * np.diag(omega)
    B = np.zeros((nm, 3))
    B[i1 - 1, 0] = 1.0
    B[i1 + d // 10 - 1, 1] = 1.0
    B[i1 + d // 10 + d - 1, 1] = -1.0
    B[i2 - 1, 2] = 1.0
    Bm = np.zeros((n, 3))
    Bm[nm:, :] = Phi.T @ B
    G = np.zeros((n, 2 * s))
    G[np.arange(s), np.arange(s)] = 1.0
    G[nm + np.arange(s), s + np.arange(s)] = 1.0
    G /= np.sqrt(2.0 * s)
    return Problem(
        name=f"tworow{d}_{i1}_{i2}",
        A0=Ap.T.copy(),
        U=Bm,
        V=Bm.copy(),
        G=G,
        E=np.eye(n),
        meta=dict(omega=omega, alpha=alpha, d=d, i1=i1, i2=i2, s=s),
    )


def erdos_renyi_edges(rng: np.random.Generator, nodes: int, p: float):
    iu = np.triu_indices(nodes, 1)
    keep = rng.random(iu[0].size) < p
    return np.stack([iu[0][keep], iu[1][keep]], axis=1)


def multi_agent(
    rng: np.random.Generator,
    agents: int = 256,
    p: float = 0.05,
    tunable_edges: int = 8,
    gain: float = 0.3,
) -> Problem:
    """Output-synchronising agents on an Erdos-Renyi graph (§3.2, Ex. 2 data).

    Each agent has state dimension 4, A_agent = blkdiag(Abar, Abar) with
    Abar = [[-10, 5], [5, -8]], output row c = [1, 1, -1, 1]/2 and gain
    kappa; B^(i) = c^T, K^(i) = kappa, C^(i) = c, so the coupling block is
    S = kappa c^T c. ``tunable_edges`` edges of the graph are taken out of
    the base Laplacian and become the parameters: with
    u_e = (e_i - e_j) (x) sqrt(kappa) c^T,

        A(w) = I (x) A_agent - L_base (x) S - sum_e w_e u_e u_e^T,

    i.e. A0 = I (x) A_agent - L_base (x) S and U = V = [u_e]. The H2 target
    of §3.2 is trace(EE^T X) with A^T X + X A = -C^T C, so G = C^T =
    I (x) c^T and E = I.
    """
    Abar = np.array([[-10.0, 5.0], [5.0, -8.0]])
    A_agent = np.kron(np.eye(2), Abar)
    c = np.array([[1.0, 1.0, -1.0, 1.0]]) / 2.0
    S = gain * (c.T @ c)
    edges = erdos_renyi_edges(rng, agents, p)
    if edges.shape[0] < tunable_edges:
        raise ValueError("graph has too few edges")
    pick = rng.choice(edges.shape[0], tunable_edges, replace=False)
    tun = edges[np.sort(pick)]
    base = np.delete(edges, pick, axis=0)
    L = np.zeros((agents, agents))
    for i, j in base:
        L[i, i] += 1
        L[j, j] += 1
        L[i, j] -= 1
        L[j, i] -= 1
    A0 = np.kron(np.eye(agents), A_agent) - np.kron(L, S)
    n = 4 * agents
    U = np.zeros((n, tunable_edges))
    for col, (i, j) in enumerate(tun):
        e = np.zeros(agents)
        e[i] = 1.0
        e[j] = -1.0
        U[:, col] = np.kron(e, np.sqrt(gain) * c[0])
    G = np.kron(np.eye(agents), c.T)
    return Problem(
        name=f"agents{agents}",
        A0=A0,
        U=U,
        V=U.copy(),
        G=G,
        E=np.eye(n),
        meta=dict(edges=tun.tolist(), agents=agents, p=p),
    )


def order_nearest_neighbour(vs: np.ndarray) -> np.ndarray:
    """Greedy nearest-neighbour path through log(v), from the smallest v.

    The recycled solver of §2.1 assumes consecutive parameter vectors vary
    slowly; this ordering presents a random sweep that way.
    """
    lv = np.log(vs)
    n = lv.shape[0]
    left = np.ones(n, dtype=bool)
    cur = int(np.argmin(lv.sum(axis=1)))
    order = [cur]
    left[cur] = False
    for _ in range(n - 1):
        d = np.where(left, ((lv - lv[cur]) ** 2).sum(axis=1), np.inf)
        cur = int(np.argmin(d))
        order.append(cur)
        left[cur] = False
    return vs[np.array(order)]


def _log_uniform(rng, lo, hi, shape):
    return np.exp(rng.uniform(np.log(lo), np.log(hi), size=shape))


def workload_small_fp64(dense: bool = False):
    """50 unit masses (n=100), unit springs, alpha=0.04, dampers at masses
    10 and 35, G = E = I; v on a linear 10 x 10 grid over [0.1, 10]^2."""
    rng = config_rngs()[0]
    p = mass_spring_chain(np.ones(51), 0.04, [10, 35])
    if dense:
        p = generic_dense(p, rng)
    g = np.linspace(0.1, 10.0, 10)
    vs = np.array([(a, b) for a in g for b in g])
    return p, vs


def workload_precision(dense: bool = True, count: int = 1000, ordered: bool = True):
    """400 unit masses (n=800), 401 springs U[0.5, 2], alpha=0.04, two dampers
    at distinct random masses; v log-uniform on [1e-2, 1e2]^2."""
    rng = config_rngs()[1]
    springs = rng.uniform(0.5, 2.0, 401)
    dampers = sorted((rng.choice(400, 2, replace=False) + 1).tolist())
    p = mass_spring_chain(springs, 0.04, dampers)
    vs = _log_uniform(rng, 1e-2, 1e2, (count, 2))
    if dense:
        p = generic_dense(p, rng)
    if ordered:
        vs = order_nearest_neighbour(vs)
    return p, vs


def workload_serving_seeds(dense: bool = True, sizes=(200, 400, 800, 1600)):
    """Eight seeds: unit-spring chains of 200/400/800/1600 masses, two each,
    rank k in {2, 3, 4} drawn per seed, dampers at random masses."""
    rng = config_rngs()[2]
    seeds = []
    for m in sizes:
        for _ in range(2):
            k = int(rng.integers(2, 5))
            dampers = sorted((rng.choice(m, k, replace=False) + 1).tolist())
            p = mass_spring_chain(np.ones(m + 1), 0.04, dampers)
            if dense:
                p = generic_dense(p, rng)
            seeds.append(p)
    return seeds


def workload_serving_requests(seeds, rate_hz: float, count: int, per_request: int = 64, seed: int = 0):
    """Poisson arrivals: list of (arrival_s, seed_index, v[per_request, k])."""
    rng = np.random.default_rng(np.random.SeedSequence([0, 3, seed]))
    t = 0.0
    out = []
    for _ in range(count):
        t += rng.exponential(1.0 / rate_hz)
        si = int(rng.integers(0, len(seeds)))
        k = seeds[si].k
        out.append((t, si, _log_uniform(rng, 0.1, 10.0, (per_request, k))))
    return out


def workload_differentiation(dense: bool = True, count: int = 256):
    """1000 unit masses (n=2000), unit springs, four dampers at random masses,
    E = projector on the first 100 modal displacements; v log-uniform on
    [0.1, 10]^4."""
    rng = config_rngs()[3]
    dampers = sorted((rng.choice(1000, 4, replace=False) + 1).tolist())
    p = mass_spring_chain(np.ones(1001), 0.04, dampers, energy_modes=100)
    vs = _log_uniform(rng, 0.1, 10.0, (count, 4))
    if dense:
        p = generic_dense(p, rng)
    return p, vs


def workload_multi_agent(count: int = 512):
    """256 agents (n=1024), ER(p=0.05) graph, 8 tunable edge weights,
    weights uniform on [0.1, 5]."""
    rng = config_rngs()[4]
    p = multi_agent(rng)
    ws = rng.uniform(0.1, 5.0, (count, 8))
    return p, ws


def chain_stiffness(springs) -> np.ndarray:
    """Tridiagonal stiffness of a fixed-fixed chain: spring i joins masses
    i-1 and i (walls at both ends), m + 1 springs for m masses."""
    springs = np.asarray(springs, dtype=np.float64)
    m = springs.size - 1
    K = np.zeros((m, m))
    for i in range(m):
        K[i, i] = springs[i] + springs[i + 1]
        if i + 1 < m:
            K[i, i + 1] = K[i + 1, i] = -springs[i + 1]
    return K


def rayleigh_chain(springs, masses, alpha: float, beta: float, dampers) -> Problem:
    """Damped chain with internal Rayleigh damping C_int = alpha M + beta K
    (eq. (Cprop)) in the physical linearisation y = [x; xdot] (eq. (MatrixAA)).

    Paper convention (§3.1): A_p(v) = A0p - B_l D(v) B_r^T with
        A0p = [[0, I], [-M^-1 K, -alpha I - beta M^-1 K]],
        B_l = [0; M^-1 B],  B_r = [0; B],
    and Q = diag(K^-1, M^-1) (the energy-norm measure). The API's family
    takes A0 = A0p^T, U = B_r, V = B_l and G with G G^T = Q
    (G = blockdiag(chol(K^-1), chol(M^-1))); E = I gives the total average
    energy. ``dampers`` are 1-based mass indices of grounded dampers.
    """
    K = chain_stiffness(springs)
    m = K.shape[0]
    masses = np.asarray(masses, dtype=np.float64)
    if masses.size != m:
        raise ValueError("one mass per chain node")
    Minv = np.diag(1.0 / masses)
    A0p = np.zeros((2 * m, 2 * m))
    A0p[:m, m:] = np.eye(m)
    A0p[m:, :m] = -Minv @ K
    A0p[m:, m:] = -alpha * np.eye(m) - beta * Minv @ K
    k = len(dampers)
    B = np.zeros((m, k))
    for c, d in enumerate(dampers):
        if not 1 <= d <= m:
            raise ValueError("damper position out of range")
        B[d - 1, c] = 1.0
    Br = np.zeros((2 * m, k))
    Br[m:, :] = B
    Bl = np.zeros((2 * m, k))
    Bl[m:, :] = Minv @ B
    G = np.zeros((2 * m, 2 * m))
    G[:m, :m] = np.linalg.cholesky(np.linalg.inv(K))
    G[m:, m:] = np.diag(1.0 / np.sqrt(masses))
    return Problem(
        name=f"rayleigh{m}",
        A0=A0p.T.copy(),
        U=Br,
        V=Bl,
        G=G,
        E=np.eye(2 * m),
        meta=dict(K=K, masses=masses, alpha=alpha, beta=beta, dampers=list(dampers)),
    )


def workload_rayleigh(masses: int = 60, dense: bool = False, count: int = 64):
    """Rayleigh-damped chain: `masses` masses U[1, 3], springs U[0.5, 2],
    alpha = 0.05, beta = 0.01, three dampers at random masses; v
    log-uniform on [0.1, 10]^3, nearest-neighbour ordered."""
    rng = np.random.default_rng(np.random.SeedSequence([0, 6]))
    springs = rng.uniform(0.5, 2.0, masses + 1)
    mvals = rng.uniform(1.0, 3.0, masses)
    dampers = sorted((rng.choice(masses, 3, replace=False) + 1).tolist())
    p = rayleigh_chain(springs, mvals, 0.05, 0.01, dampers)
    vs = order_nearest_neighbour(_log_uniform(rng, 0.1, 10.0, (count, 3)))
    if dense:
        p = generic_dense(p, rng)
    return p, vs


def _matlab_range(a: float, b: float) -> list:
    """The integers a:b of a colon expression with unit step (a, b may be
    fractional; an empty list when b < a)."""
    lo = int(np.ceil(a - 1e-12))
    return list(range(lo, int(np.floor(b + 1e-12)) + 1))


def ex3_laplacian(m: int) -> np.ndarray:
    """Laplacian of Ex. 3's communication graph (Algorithm 2), 1-based.

    The graph starts as a wheel: the ring 1 - 2 - ... - (m-1) - 1 and a hub m
    joined to every ring node. Ring edges (r, r+1) for r in the list r are
    removed (r = m - 1 names the closing edge (1, m - 1)), and the spokes of
    the nodes in the list h are removed; the Laplacian is the degree matrix
    minus the adjacency.
    """
    r = (_matlab_range(m / 20 + m / 50, m / 10) + _matlab_range(m / 4 + m / 20, m / 4 + m / 10)
         + _matlab_range(m / 2 + m / 20 + 2, m / 2 + m / 20 + m / 50)
         + _matlab_range(m / 2 + m / 10 + 2, m / 2 + m / 10 + m / 20) + _matlab_range(m - m / 10, m - m / 20))
    h = (_matlab_range(1, m / 20) + _matlab_range(m / 10 + m / 40, m / 10 + m / 20)
         + _matlab_range(m / 2, m / 2 + m / 20) + [m - 1])
    adj = np.zeros((m + 1, m + 1))  # 1-based; row/column 0 unused
    for i in range(1, m - 1):
        adj[i, i + 1] = 1.0
        adj[i, m] = 1.0
    adj[1, m - 1] = 1.0
    adj[m - 1, m] = 1.0
    for ri in r:
        if ri == m - 1:
            adj[1, m - 1] = 0.0
        else:
            adj[ri, ri + 1] = 0.0
    for hi in h:
        adj[hi, m] = 0.0
    adj = adj[1:, 1:]
    adj = adj + adj.T
    return np.diag(adj.sum(axis=1)) - adj


def agent_network(L: np.ndarray):
    """Ex. 2 / Ex. 3 agents on the graph with Laplacian L (§3.2): 2 x 2 agent
    state A_i = [[-10, 5], [5, -8]], gain K_i = diag(0.3, 0.2),
    B_i = C_i^T = [[1, 1], [-1, 1]]; blocks A_ij = delta_ij A_i -
    l_ij B_i K_i C_j. Returns (A, C) with C = blockdiag(C_i)."""
    Ai = np.array([[-10.0, 5.0], [5.0, -8.0]])
    Bi = np.array([[1.0, 1.0], [-1.0, 1.0]])
    Ki = np.diag([0.3, 0.2])
    Ci = Bi.T
    m = L.shape[0]
    A = np.kron(np.eye(m), Ai) - np.kron(L, Bi @ Ki @ Ci)
    C = np.kron(np.eye(m), Ci)
    return A, C


def ex3_problem(m: int = 200, k_index: int = 41) -> Problem:
    """Ex. 3: m agents on the Algorithm 2 graph, a rank-4 change of the
    off-diagonal entries of two consecutive agents' diagonal blocks.

    For the odd 1-based state index k (1 <= k <= 2m - 3), B_l and B_r are
    zero except rows k..k+3: B_l there is the permutation [[0,1,0,0],
    [1,0,0,0],[0,0,0,1],[0,0,1,0]] and B_r the identity. The paper's family
    A_p(v) = A - B_l diag(v1, v1, v2, v2) B_r^T with Q = C^T C and E = I;
    the API's parameter vector is (v1, v1, v2, v2), A0 = A^T = A,
    U = B_r, V = B_l, G = C^T.
    """
    if k_index % 2 != 1 or not 1 <= k_index <= 2 * m - 3:
        raise ValueError("k must be odd and in [1, 2m - 3]")
    A, C = agent_network(ex3_laplacian(m))
    n = 2 * m
    Bl = np.zeros((n, 4))
    Br = np.zeros((n, 4))
    Bl[k_index - 1:k_index + 3, :] = np.array([[0, 1, 0, 0], [1, 0, 0, 0], [0, 0, 0, 1], [0, 0, 1, 0]], float)
    Br[k_index - 1:k_index + 3, :] = np.eye(4)
    return Problem(name=f"ex3_{m}_{k_index}", A0=A.T.copy(), U=Br, V=Bl, G=C.T.copy(), E=np.eye(n),
                   meta=dict(m=m, k_index=k_index))


def ex3_grid() -> np.ndarray:
    """Ex. 3's parameter grid: v1, v2 in -4.9:0.5:14.6 (40 values each), in
    serpentine order (consecutive pairs differ in one coordinate by 0.5);
    rows are the API's vectors (v1, v1, v2, v2)."""
    g = -4.9 + 0.5 * np.arange(40)
    rows = []
    for a, v1 in enumerate(g):
        for v2 in (g if a % 2 == 0 else g[::-1]):
            rows.append((v1, v1, v2, v2))
    return np.array(rows)


def stable_mask(p: Problem, vs) -> np.ndarray:
    """True where A(v) = A0 - U diag(v) V^T is Hurwitz (rightmost eigenvalue
    in the open left half plane; unstable members are discarded, §4).

    For a symmetric, negative definite A0 and a symmetric change
    U diag(v) V^T = S M(v) S^T supported on a few rows S (Ex. 3), -A(v) is
    positive definite iff I + W^(1/2) M(v) W^(1/2) is, with
    W = S^T (-A0)^-1 S: a congruence (see the test), so each v costs a
    small eigenproblem. Otherwise the eigenvalues of A(v) are computed.
    """
    vs = np.asarray(vs, dtype=np.float64)
    A0, U, V = p.A0, p.U, p.V
    rows = np.nonzero(np.any(U != 0, axis=1) | np.any(V != 0, axis=1))[0]
    sym = np.allclose(A0, A0.T) and np.linalg.eigvalsh(A0).max() < 0
    if sym:
        M0 = [(U[rows] * v[None, :]) @ V[rows].T for v in vs]
        sym = all(np.allclose(M, M.T) for M in M0)
    out = np.zeros(len(vs), dtype=bool)
    if sym:
        S = np.zeros((A0.shape[0], rows.size))
        S[rows, np.arange(rows.size)] = 1.0
        W = S.T @ np.linalg.solve(-A0, S)
        wv, wq = np.linalg.eigh(W)
        Wh = (wq * np.sqrt(wv)) @ wq.T
        for i, M in enumerate(M0):
            # A(v) = A0 - S M S^T, so -A(v) = -A0 + S M S^T
            out[i] = np.linalg.eigvalsh(np.eye(rows.size) + Wh @ M @ Wh).min() > 0
        return out
    for i, v in enumerate(vs):
        out[i] = np.linalg.eigvals(A0 - (U * v[None, :]) @ V.T).real.max() < 0
    return out


EX3_POSITIONS = (41, 121, 201, 281)  # the positions k of Ex. 3's table


def workload_ex3(k_index: int = 41, m: int = 200):
    """Ex. 3 sweep for one perturbation position: the stable members of the
    40 x 40 grid, in serpentine order. Over the four positions of Ex. 3's
    table (EX3_POSITIONS) 356 of the 6,400 grid points are unstable."""
    p = ex3_problem(m, k_index)
    vs = ex3_grid()
    return p, vs[stable_mask(p, vs)]
