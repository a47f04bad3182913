"""FP64 CPU oracle of the Tutte initializer (App. A, "Tutte's Energy").

TEST INFRASTRUCTURE ONLY, like oracle/admm.py: only the test-suite, the smoke
check and the CPU-baseline leg of the benchmark may import it.

E_T(W) = sum over the mesh edges (i, j) of |W_i - W_j|^2 / |V_i - V_j|, minimized
with the boundary vertices held at given positions.  E_T is quadratic, so the
minimizer solves one sparse linear system: for every interior vertex i,
sum_j c_ij (W_i - W_j) = 0 with c_ij = 1 / |V_i - V_j| over the edges at i.
The paper uses its minimizers as initial maps (flip-free in 2D with a convex
boundary, Tutte's theorem; not in general for tetrahedra).
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as sla


def mesh_edges(T: np.ndarray) -> np.ndarray:
    """Every edge of the elements once, as (i, j) with i < j."""
    T = np.asarray(T, np.int64)
    k = T.shape[1]
    pairs = [np.sort(T[:, [a, b]], axis=1) for a in range(k) for b in range(a + 1, k)]
    return np.unique(np.concatenate(pairs, 0), axis=0)


def tutte_energy(V: np.ndarray, T: np.ndarray, W: np.ndarray) -> float:
    """E_T(W) summed edge by edge, as the definition writes it."""
    e = mesh_edges(T)
    c = 1.0 / np.linalg.norm(V[e[:, 0]] - V[e[:, 1]], axis=1)
    d = W[e[:, 0]] - W[e[:, 1]]
    return float(np.sum(c * np.sum(d * d, axis=1)))


def tutte(V, T, boundary, boundary_pos) -> np.ndarray:
    """Minimizer of E_T with W[boundary] = boundary_pos (n x d)."""
    V = np.asarray(V, np.float64)
    n = V.shape[0]
    boundary = np.asarray(boundary, np.int64)
    boundary_pos = np.asarray(boundary_pos, np.float64)
    e = mesh_edges(T)
    c = 1.0 / np.linalg.norm(V[e[:, 0]] - V[e[:, 1]], axis=1)
    # the gradient of E_T is 2 L W with L the weighted graph Laplacian
    rows = np.concatenate([e[:, 0], e[:, 1], e[:, 0], e[:, 1]])
    cols = np.concatenate([e[:, 0], e[:, 1], e[:, 1], e[:, 0]])
    vals = np.concatenate([c, c, -c, -c])
    L = sp.csr_matrix((vals, (rows, cols)), shape=(n, n))
    fixed = np.zeros(n, bool)
    fixed[boundary] = True
    inner = np.nonzero(~fixed)[0]
    W = np.zeros((n, boundary_pos.shape[1]))
    W[boundary] = boundary_pos
    if len(inner):
        A = L[inner][:, inner].tocsc()
        rhs = -(L[inner][:, boundary] @ boundary_pos)
        lu = sla.splu(A)
        W[inner] = lu.solve(np.ascontiguousarray(rhs))
    return W
