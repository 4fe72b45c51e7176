"""Fundamental solutions as dense 3x3 blocks (oracle side, FP64).

stokeslet  Sec. 2.1 eq. stokeslet:   S(r) = (I/|r| + r r^T/|r|^3) / (8 pi mu)
rotlet     Sec. 2.3 (rotlet R):      R(r) = [[0, r3, -r2], [-r3, 0, r1], [r2, -r1, 0]] / (8 pi mu |r|^3)
dipole     Sec. 2.3 eq. doublet:     D(r) = (-I/|r|^3 + 3 r r^T/|r|^5) / (4 pi)   (no viscosity, as printed)

Each function takes r of shape (..., 3) and returns blocks of shape (..., 3, 3) so
that u = block @ strength.
"""
import math

import numpy as np


def _norm(r):
    return np.sqrt(np.sum(r * r, axis=-1))


def stokeslet(r, visc=1.0):
    r = np.asarray(r, dtype=np.float64)
    n = _norm(r)[..., None, None]
    eye = np.eye(3)
    rr = r[..., :, None] * r[..., None, :]
    return (eye / n + rr / n ** 3) / (8.0 * math.pi * visc)


def rotlet(r, visc=1.0):
    r = np.asarray(r, dtype=np.float64)
    n = _norm(r)[..., None, None]
    z = np.zeros(r.shape[:-1])
    m = np.stack([
        np.stack([z, r[..., 2], -r[..., 1]], axis=-1),
        np.stack([-r[..., 2], z, r[..., 0]], axis=-1),
        np.stack([r[..., 1], -r[..., 0], z], axis=-1),
    ], axis=-2)
    return m / (8.0 * math.pi * visc * n ** 3)


def dipole(r):
    r = np.asarray(r, dtype=np.float64)
    n = _norm(r)[..., None, None]
    eye = np.eye(3)
    rr = r[..., :, None] * r[..., None, :]
    return (-eye / n ** 3 + 3.0 * rr / n ** 5) / (4.0 * math.pi)


def block_matrix(targets, sources, kind, visc=1.0):
    """Dense (3 nt, 3 ns) matrix whose (i, j) 3x3 block is kind(x_i - y_j)."""
    targets = np.asarray(targets, dtype=np.float64).reshape(-1, 3)
    sources = np.asarray(sources, dtype=np.float64).reshape(-1, 3)
    nt, ns = targets.shape[0], sources.shape[0]
    if nt == 0 or ns == 0:
        return np.zeros((3 * nt, 3 * ns))
    r = targets[:, None, :] - sources[None, :, :]
    if kind == "S":
        b = stokeslet(r, visc)
    elif kind == "R":
        b = rotlet(r, visc)
    elif kind == "D":
        b = dipole(r)
    else:
        raise ValueError(kind)
    return b.transpose(0, 2, 1, 3).reshape(3 * nt, 3 * ns)
