"""FP64 reference gradient of a loss through the variable-coefficient solve.

TEST INFRASTRUCTURE ONLY: imported by ``tests/``.  The CUDA library never uses
it, and it shares no code with the library's autograd path (which assembles
the operator with torch operations and scatters the gradient on the GPU).

Problem (the differentiation workload): cell-centred finite volumes for
-div(exp(theta) grad u) = f on the unit square with u = 0 on the boundary, on
m x m cells; the face coefficient between cells a and b is the harmonic mean
k_f = 2 k_a k_b / (k_a + k_b) of k = exp(theta); a boundary face of cell a
contributes 2 k_a to the diagonal (the wall at half a cell).  The loss is
L(theta) = 1/2 ||u(theta) - u_obs||^2.

Gradient by the adjoint method, written out by hand:
  A u = f,   A^T lam = u - u_obs,   dL/dA_ij = -lam_i u_j   (dA: A's entries)
  face f = (a, b):  A_aa += k_f, A_bb += k_f, A_ab = A_ba = -k_f, so
      dL/dk_f = dL/dA_aa + dL/dA_bb - dL/dA_ab - dL/dA_ba
              = -(lam_a - lam_b)(u_a - u_b)
  dk_f/dtheta_a = k_f k_b / (k_a + k_b),  dk_f/dtheta_b = k_f k_a / (k_a + k_b)
  boundary face of cell a: dL/d(2 k_a) = dL/dA_aa = -lam_a u_a, d(2 k_a)/dtheta_a = 2 k_a.
Solves are sparse direct (scipy's SuperLU) in FP64.
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla


def faces(m: int):
    idx = np.arange(m * m).reshape(m, m)
    a = np.concatenate([idx[:, :-1].ravel(), idx[:-1, :].ravel()])
    b = np.concatenate([idx[:, 1:].ravel(), idx[1:, :].ravel()])
    nb = np.zeros((m, m))
    nb[:, 0] += 1
    nb[:, -1] += 1
    nb[0, :] += 1
    nb[-1, :] += 1
    return a, b, nb.ravel()


def operator(m: int, theta: np.ndarray) -> sp.csr_matrix:
    """The FV matrix, assembled face by face."""
    k = np.exp(theta)
    a, b, nb = faces(m)
    kf = 2.0 * k[a] * k[b] / (k[a] + k[b])
    n = m * m
    diag = np.zeros(n)
    np.add.at(diag, a, kf)
    np.add.at(diag, b, kf)
    diag += 2.0 * k * nb
    rows = np.concatenate([a, b, np.arange(n)])
    cols = np.concatenate([b, a, np.arange(n)])
    vals = np.concatenate([-kf, -kf, diag])
    return sp.csr_matrix((vals, (rows, cols)), shape=(n, n))


def loss_and_grad(m: int, theta: np.ndarray, f: np.ndarray, u_obs: np.ndarray):
    """(L, dL/dtheta, u) by the adjoint formulas above."""
    k = np.exp(theta)
    A = operator(m, theta).tocsc()
    lu = spla.splu(A)
    u = lu.solve(f)
    r = u - u_obs
    lam = lu.solve(r, trans="T")
    a, b, nb = faces(m)
    dLdkf = -(lam[a] - lam[b]) * (u[a] - u[b])
    g = np.zeros(m * m)
    np.add.at(g, a, dLdkf * (2.0 * k[a] * k[b] / (k[a] + k[b])) * k[b] / (k[a] + k[b]))
    np.add.at(g, b, dLdkf * (2.0 * k[a] * k[b] / (k[a] + k[b])) * k[a] / (k[a] + k[b]))
    g += (-lam * u) * 2.0 * k * nb
    return 0.5 * float(r @ r), g, u


def loss(m: int, theta: np.ndarray, f: np.ndarray, u_obs: np.ndarray) -> float:
    u = spla.spsolve(operator(m, theta).tocsc(), f)
    r = u - u_obs
    return 0.5 * float(r @ r)
