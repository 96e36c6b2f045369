"""Shared helpers for the GPU parity tests (error metrics, context setup)."""
import numpy as np


def rel_vec(a, b):
    """Per-particle relative error |a - b| / |b| of [n, 3] vectors."""
    return np.linalg.norm(np.asarray(a) - np.asarray(b), axis=-1) / np.linalg.norm(np.asarray(b), axis=-1)


def rel_scalar(a, b):
    return np.abs(np.asarray(a) - np.asarray(b)) / np.abs(np.asarray(b))


def kappa(m, x, v, eps, idx):
    """Cancellation factor sum_j |m_j r_ij / s^3| / |a_i| for the sampled i
    (numpy, FP64; used only to explain a worst-case miss)."""
    out = np.empty(len(idx))
    for k, i in enumerate(idx):
        r = x - x[i]
        s2 = (r * r).sum(1) + eps * eps
        s2[i] = np.inf
        terms = m[:, None] * r / s2[:, None] ** 1.5
        out[k] = np.linalg.norm(terms, axis=1).sum() / np.linalg.norm(terms.sum(0))
    return out


def gpu_forces(nb, precision, m, x, v, eps, idx, tuning=None, t=0.0):
    N = len(m)
    with nb.NBody(N, precision, 0) as s:
        s.set_params(eps, 0.01, 2.0 ** -22, 2.0 ** -3)
        s.set_j_particles(0, m, x, v)
        if tuning:
            s.set_tuning(**tuning)
        s.predict(t)
        return s.compute_forces(np.asarray(idx, dtype=np.int32))
