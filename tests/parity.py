"""Shared comparison helpers for the GPU parity tests (no method arithmetic)."""
import numpy as np

U_TOL = 1e-10


def u_tol(R):
    """Bar for U = (R^T R)^{-1}: 1e-10 relative, widened to 1e-15 * kappa(R^T R)
    when the kept fibers are ill-conditioned (both sides then carry errors of
    order kappa * 2^-53; the oracle's rank-one updates more than a Cholesky)."""
    if R.shape[1] == 0:
        return U_TOL
    R = np.asarray(R, dtype=np.float64)
    kappa = np.linalg.cond(R.T @ R)
    return max(U_TOL, 1e-15 * kappa)


def u_residual(U, R):
    """||U (R^T R) - I||_F with the exact Gram matrix (a property at any size)."""
    R = np.asarray(R, dtype=np.float64)
    G = R.T @ R
    return np.linalg.norm(U @ G - np.eye(G.shape[0]))


def rel_fro(a, b):
    nb = np.linalg.norm(b)
    return np.linalg.norm(a - b) / (nb if nb > 0 else 1.0)


def error_tol(precision, e_ref):
    """Stated bar for the relative error: 1e-10 relative (FP64 path) or 1e-4
    (FP32-bulk path); below 1e-8 the bar is absolute (1e-12 / 1e-6)."""
    if precision == 0:
        return 1e-12 if e_ref < 1e-8 else 1e-10 * e_ref
    return 1e-6 if e_ref < 1e-8 else 1e-4 * e_ref


def tie_margin(ratios, eps):
    """Smallest distance of a residual ratio ||res||/||x|| to eps (reading A14)."""
    r = np.asarray(ratios, dtype=np.float64)
    return float(np.min(np.abs(r - eps))) if r.size else np.inf


def error_tol_real(e_ref, R):
    """Bar for the error of real-valued tensors.  The Gram matrix of real
    values is not exact, so the Q-form (Q = R L^{-T} from its Cholesky
    factor) loses orthogonality in proportion to kappa(R^T R): its error is
    within 4 n u kappa(R^T R) (n = rows of R, u = 2^-53; the factor covers
    the Gram's and the factorization's backward errors), on top of the
    FP64 bar (reading A29)."""
    R = np.asarray(R, dtype=np.float64)
    kappa = np.linalg.cond(R.T @ R) if R.shape[1] else 1.0
    return max(error_tol(0, e_ref), 4.0 * R.shape[0] * 2.0 ** -53 * kappa)
