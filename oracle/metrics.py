"""Error measures for completion and truncated SVDs (CPU oracle; test
infrastructure).

* ``completion_error``: ||P_Phi(X) - P_Phi(M)||_F / ||P_Phi(M)||_F, the stopping
  quantity of Alg. 2 / Alg. 6.
* ``mae``: eq. (10), mean absolute error over a set of entries.
* ``rmse``: root-mean-square error over a set of entries (held-out quality).
* ``sigma_rel_err``: max_j |s_j - t_j| / t_j.
* ``max_principal_angle``: largest principal angle between two subspaces of
  equal dimension, atan2(||Qb - Qa Qa^T Qb||_2, sigma_min(Qa^T Qb)) for
  orthonormal bases (the sine and cosine forms together stay accurate for
  both small and large angles).
"""
from __future__ import annotations

import numpy as np


def completion_error(x_on_phi: np.ndarray, m_on_phi: np.ndarray) -> float:
    return float(np.linalg.norm(np.asarray(x_on_phi, np.float64) - m_on_phi) / np.linalg.norm(m_on_phi))


def mae(pred: np.ndarray, truth: np.ndarray) -> float:
    return float(np.mean(np.abs(np.asarray(pred, np.float64) - truth)))


def rmse(pred: np.ndarray, truth: np.ndarray) -> float:
    d = np.asarray(pred, np.float64) - truth
    return float(np.sqrt(np.mean(d * d)))


def sigma_rel_err(s: np.ndarray, t: np.ndarray) -> float:
    s = np.asarray(s, np.float64)
    t = np.asarray(t, np.float64)
    return float(np.max(np.abs(s - t) / np.abs(t))) if t.size else 0.0


def max_principal_angle(A: np.ndarray, B: np.ndarray) -> float:
    Qa, _ = np.linalg.qr(np.asarray(A, np.float64))
    Qb, _ = np.linalg.qr(np.asarray(B, np.float64))
    C = Qa.T @ Qb
    cos_min = np.linalg.svd(C, compute_uv=False).min()
    sin_max = np.linalg.norm(Qb - Qa @ C, 2)
    return float(np.arctan2(sin_max, cos_min))
