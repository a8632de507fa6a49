"""FP64 CPU oracle for principal coordinates analysis of a distance matrix.

TEST INFRASTRUCTURE ONLY: used by the tests and the benchmark to check the
GPU ordination; the product library never imports or calls anything here.

The paper (Sections I and II) places the UniFrac distance matrix in the usual
analysis pipeline, where it is ordinated by principal coordinates analysis
(PCoA).  Classical PCoA, written out from its definition:

    A = -1/2 (D o D)                       (element-wise square)
    B = J A J,   J = I - (1/n) 1 1^T       (double centring)
    B = U diag(lambda) U^T                 (symmetric eigendecomposition)
    coordinates = U_k diag(sqrt(max(lambda_k, 0)))

for the k largest eigenvalues.  Parity pinned: planar configurations are
recovered exactly (their distances reproduced, the non-zero eigenvalues equal
the squared singular values of the centred points, the rest zero), and the
eigenvalues sum to trace(B) = (1/n) sum_{i<j} d_ij^2.
"""
from __future__ import annotations

import numpy as np


def double_centred(D: np.ndarray) -> np.ndarray:
    """B = -1/2 J (D o D) J in FP64, formed with explicit matrix products."""
    D = np.asarray(D, dtype=np.float64)
    n = D.shape[0]
    A = -0.5 * D * D
    J = np.eye(n) - np.ones((n, n)) / n
    return J @ A @ J


def pcoa(D: np.ndarray, k: int) -> tuple[np.ndarray, np.ndarray]:
    """(eigenvalues, coordinates) of the k largest eigenvalues of B, in
    descending order; coordinates [n, k] = U_k sqrt(max(lambda_k, 0))."""
    B = double_centred(D)
    w, V = np.linalg.eigh(B)
    idx = np.argsort(w)[::-1][:k]
    lam = w[idx]
    coords = V[:, idx] * np.sqrt(np.maximum(lam, 0.0))
    return lam, coords
