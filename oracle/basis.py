"""1D building blocks of the discretization (Section 2 of the paper).

Test infrastructure: see ``oracle/__init__.py``.

* Nodal basis: Lagrange polynomials on the Legendre-Gauss-Lobatto (GL) nodes of
  degree p, i.e. the end points plus the roots of P'_p (Section 2, nodal basis).
* Quadrature: Gauss-Legendre with p+1 points (Section 2, "Gaussian quadrature
  with p+1 points per coordinate direction").

Both rules are computed here with the Golub-Welsch eigenvalue method from the
three-term recurrences of the Legendre and Jacobi(1,1) polynomials, on the
reference interval [0,1] (the paper's reference element is [0,1]^d).
"""
import numpy as np


def gauss_legendre(n):
    """n-point Gauss-Legendre rule on [0,1]: (points ascending, weights).

    Golub-Welsch: the points are eigenvalues of the symmetric Jacobi matrix of
    the Legendre recurrence, off-diagonal b_j = j / sqrt(4 j^2 - 1); the weight
    of a point is 2 * (first eigenvector component)^2 on [-1,1].
    """
    if n < 1:
        raise ValueError("n >= 1")
    j = np.arange(1, n, dtype=np.float64)
    off = j / np.sqrt(4.0 * j * j - 1.0)
    T = np.diag(off, 1) + np.diag(off, -1)
    lam, V = np.linalg.eigh(T)
    w = 2.0 * V[0, :] ** 2
    order = np.argsort(lam)
    t, w = lam[order], w[order]
    # symmetrise against eigen-solver noise (rule is exactly symmetric)
    t = 0.5 * (t - t[::-1])
    w = 0.5 * (w + w[::-1])
    return 0.5 * (t + 1.0), 0.5 * w


def gauss_lobatto(n):
    """n GL nodes on [0,1] (n >= 2): 0, roots of P'_{n-1}, 1.

    The interior nodes are the Gauss-Jacobi(1,1) points of degree n-2, obtained
    as eigenvalues of the Jacobi matrix with off-diagonal
    b_j^2 = j (j+2) / ((2j+1)(2j+3)).
    """
    if n < 2:
        raise ValueError("n >= 2")
    m = n - 2
    if m > 0:
        j = np.arange(1, m, dtype=np.float64)
        off = np.sqrt(j * (j + 2.0) / ((2.0 * j + 1.0) * (2.0 * j + 3.0)))
        T = np.diag(off, 1) + np.diag(off, -1)
        inner = np.sort(np.linalg.eigvalsh(T))
        inner = 0.5 * (inner - inner[::-1])
    else:
        inner = np.zeros(0)
    t = np.concatenate([[-1.0], inner, [1.0]])
    return 0.5 * (t + 1.0)


def lagrange_values(nodes, x):
    """L[a, j] = l_j(x_a) for the Lagrange basis on ``nodes`` (product formula)."""
    nodes = np.asarray(nodes, dtype=np.float64)
    x = np.atleast_1d(np.asarray(x, dtype=np.float64))
    n = len(nodes)
    L = np.ones((len(x), n))
    for j in range(n):
        for m in range(n):
            if m != j:
                L[:, j] *= (x - nodes[m]) / (nodes[j] - nodes[m])
    return L


def lagrange_derivatives(nodes, x):
    """L'[a, j] = l_j'(x_a): derivative of the product formula term by term."""
    nodes = np.asarray(nodes, dtype=np.float64)
    x = np.atleast_1d(np.asarray(x, dtype=np.float64))
    n = len(nodes)
    D = np.zeros((len(x), n))
    for j in range(n):
        for m in range(n):
            if m == j:
                continue
            term = np.full(len(x), 1.0 / (nodes[j] - nodes[m]))
            for r in range(n):
                if r != j and r != m:
                    term *= (x - nodes[r]) / (nodes[j] - nodes[r])
            D[:, j] += term
    return D


def tensor_basis(nodes, pts):
    """Values V[p, i] and reference gradients G[b, p, i] of the 3D tensor basis.

    Node index i = ix + n*(iy + n*iz) (x fastest); N_i(xi) = l_ix(xi_0) l_iy(xi_1)
    l_iz(xi_2) (Section 2, tensor-product shape functions).  ``pts`` is (P,3).
    """
    pts = np.asarray(pts, dtype=np.float64)
    n = len(nodes)
    Lv = [lagrange_values(nodes, pts[:, d]) for d in range(3)]
    Ld = [lagrange_derivatives(nodes, pts[:, d]) for d in range(3)]
    P = len(pts)
    V = np.einsum("pi,pj,pk->pkji", Lv[0], Lv[1], Lv[2]).reshape(P, n ** 3)
    G = np.empty((3, P, n ** 3))
    G[0] = np.einsum("pi,pj,pk->pkji", Ld[0], Lv[1], Lv[2]).reshape(P, n ** 3)
    G[1] = np.einsum("pi,pj,pk->pkji", Lv[0], Ld[1], Lv[2]).reshape(P, n ** 3)
    G[2] = np.einsum("pi,pj,pk->pkji", Lv[0], Lv[1], Ld[2]).reshape(P, n ** 3)
    return V, G


def tensor_points(x1d):
    """All 3D tensor points (x fastest) of a 1D point set: array (n^3, 3)."""
    n = len(x1d)
    z, y, x = np.meshgrid(x1d, x1d, x1d, indexing="ij")
    return np.stack([x.ravel(), y.ravel(), z.ravel()], axis=1).reshape(n ** 3, 3)


def tensor_weights(w1d):
    """Tensor quadrature weights matching ``tensor_points`` ordering."""
    return np.einsum("k,j,i->kji", w1d, w1d, w1d).ravel()
