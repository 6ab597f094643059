"""Dense FP64 reference of the global-step iteration used on the GPU.

TEST INFRASTRUCTURE ONLY.

Sec. 5 of the paper solves the global system A x = b (A = H + dH,
Eq. (global) with collision springs) by a reduced solve in span(U) followed
by A-Jacobi relaxation of the remaining high-frequency residual:

  Eq. (subspace_collision):  (U^T A U) q = U^T r,   r = b - A x
  Eq. (uu):                  U^T dH U = sum_c w_c U_c U_c^T  (dH diagonal)
  Eq. (high_frequency_residual):  A dx = r - A U q, relaxed by Jacobi.

Reading used here and on the GPU: the correction is taken about the current
iterate x (a two-level correction, as the paper's Sec. 2 multigrid remark
describes) rather than about the rest shape X; with exact eigenvectors and
the rest iterate the two coincide.  The reduced matrix is formed from the U
actually used, so it need not be diagonal.
"""
import numpy as np


def reduced_matrix(U, H, contact_w=None):
    """U^T H U + sum_c w_c U_c U_c^T (Eq. (subspace_collision) with Eq. (uu))."""
    A0 = U.T @ (H @ U)
    if contact_w is not None:
        nz = np.nonzero(contact_w)[0]
        Uc = U[nz]
        A0 = A0 + (Uc * contact_w[nz][:, None]).T @ Uc
    return A0


def subspace_correction(U, H, contact_w, r):
    """delta0 = U q with (U^T A U) q = U^T r; returns (delta0, q)."""
    Ar = reduced_matrix(U, H, contact_w)
    g = U.T @ r
    q = np.linalg.solve(Ar, g)
    return U @ q, q


def jacobi(H, contact_w, r, delta0, sweeps, omega, free):
    """delta_{k+1} = delta_k + omega D^-1 (r - A delta_k) on free rows,
    D = diag(A), A = H + diag(contact_w); pinned rows stay 0."""
    d = H.diagonal() + (contact_w if contact_w is not None else 0.0)
    delta = delta0.copy()
    for _ in range(sweeps):
        Ad = H @ delta
        if contact_w is not None:
            Ad = Ad + contact_w[:, None] * delta
        delta = delta + omega * (r - Ad) / d[:, None]
        delta[~free] = 0.0
    return delta
