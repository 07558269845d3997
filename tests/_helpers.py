"""Shared test helpers: error metrics and small conveniences (no method
arithmetic beyond the comparison metric itself)."""
import numpy as np


def omega_floor(cell):
    """c_T,min |q|_min / 2: the scale below which frequencies are compared
    in absolute terms (the acoustic branches vanish at Gamma)."""
    A = np.array([cell.h1, cell.h2], float)
    qm = 2 * np.pi * np.linalg.inv(A)
    qmin = min(np.linalg.norm(qm[:, 0]), np.linalg.norm(qm[:, 1]))
    if getattr(cell, "stiffness", None) is not None:
        # slowest shear-like speed: smallest eigenvalue of the Voigt stiffness over rho
        c2 = min(np.linalg.eigvalsh(C)[0] / r for C, r in zip(cell.stiffness, cell.rho))
        return np.sqrt(c2) * qmin / 2
    return np.sqrt(np.min(cell.mu / cell.rho)) * qmin / 2


def omega_rel_err(w, w_ref, floor):
    """Relative frequency error measured on lambda = omega^2:
    |lambda - lambda_ref| / (2 max(lambda_ref, floor^2)), which equals
    |d omega| / omega for omega >> floor and stays meaningful at omega = 0
    where only absolute accuracy in lambda exists."""
    lam, lref = np.asarray(w) ** 2, np.asarray(w_ref) ** 2
    return np.abs(lam - lref) / (2 * np.maximum(lref, floor ** 2))


def field_tables(cell):
    """Per-pixel fields 1/(lam+mu), 1/mu, rho of a cell, (3, P*P)."""
    ph = cell.phase.reshape(-1).astype(np.int64)
    return np.array([(1 / (cell.lam + cell.mu))[ph], (1 / cell.mu)[ph], cell.rho[ph]])
