"""Ex. 1's two-row mechanical model (workloads.two_row_system), checked
against an independent construction from its spring list (paper §4, Ex. 1:
the stiffness matrix printed with the example, eq. (mass-Config), eq.
(damping-geometry), eq. (matrix Z))."""
import numpy as np
import scipy.linalg as sla

from workloads import two_row_masses, two_row_system


def springs_to_K(d, k1, k2, k3):
    """K from the springs: row r: wall - mass 1 - ... - mass d - mass 2d+1, and
    mass 2d+1 - wall (1-based masses; row 2 is masses d+1..2d)."""
    nm = 2 * d + 1
    K = np.zeros((nm, nm))

    def spring(i, j, k):  # 0-based masses, j = None: wall
        K[i, i] += k
        if j is not None:
            K[j, j] += k
            K[i, j] -= k
            K[j, i] -= k

    for r, kr in ((0, k1), (1, k2)):
        o = r * d
        spring(o, None, kr)
        for i in range(d - 1):
            spring(o + i, o + i + 1, kr)
        spring(o + d - 1, nm - 1, kr)
    spring(nm - 1, None, k3)
    return K


def test_masses_as_printed():
    m = two_row_masses(1000)
    assert m.size == 2001
    np.testing.assert_allclose(m[[0, 499, 500, 999, 1000, 1999, 2000]],
                               [199.9, 100.1, 100.1, 150.0, 160.0, 160.0, 175.0])


def test_model_against_spring_list():
    d, s = 500, 7
    p = two_row_system(d, 40, 900, s)
    nm = 2 * d + 1
    K = springs_to_K(d, 40.0, 20.0, 30.0)
    M = np.diag(two_row_masses(d))
    w2, Phi = sla.eigh(K, M)
    np.testing.assert_allclose(p.meta["omega"], np.sqrt(w2), rtol=1e-10)
    # A_p = A0^T in the modal form of eq. (MatrixA) with critical-fraction damping
    Ap = p.A0.T
    om = np.sqrt(w2)
    np.testing.assert_allclose(np.diag(Ap[:nm, nm:]), om, rtol=1e-10)
    np.testing.assert_allclose(np.diag(Ap[nm:, :nm]), -om, rtol=1e-10)
    np.testing.assert_allclose(np.diag(Ap[nm:, nm:]), -0.04 * om, rtol=1e-10)
    # dampers of eq. (damping-geometry): diag(Phi^T B B^T Phi) is independent of eigenvector signs
    B = np.zeros((nm, 3))
    B[40 - 1, 0] = 1.0
    B[40 + d // 10 - 1, 1] = 1.0
    B[40 + d // 10 + d - 1, 1] = -1.0
    B[900 - 1, 2] = 1.0
    ref = np.diag(Phi.T @ B @ B.T @ Phi)
    got = np.diag(p.U[nm:] @ p.U[nm:].T)
    np.testing.assert_allclose(got, ref, rtol=1e-8, atol=1e-14 * ref.max())
    assert np.all(p.U[:nm] == 0) and np.array_equal(p.U, p.V)
    # Q = G G^T = eq. (matrix Z): 1/(2s) on the first s modal displacements and velocities
    Q = p.G @ p.G.T
    expect = np.zeros(2 * nm)
    expect[:s] = expect[nm:nm + s] = 1.0 / (2 * s)
    np.testing.assert_allclose(Q, np.diag(expect), atol=1e-15)
