"""Test-side metrics: canonical angles (Definition 3.1) and friends."""
import numpy as np


def orth(X):
    q, _ = np.linalg.qr(np.asarray(X, dtype=np.float64))
    return q


def sine(U, V):
    """||sin Theta(U, V)||_2 for subspaces of equal dimension (Definition 3.1):
    the largest singular value of (I - Q_U Q_U^T) Q_V."""
    Qu, Qv = orth(U), orth(V)
    P = Qv - Qu @ (Qu.T @ Qv)
    return float(np.linalg.norm(P, 2))


def chi(a, b):
    """Relative gap chi(a, b) = |a - b| / sqrt(|a b|) (Section 3.1)."""
    return abs(a - b) / np.sqrt(abs(a * b))
