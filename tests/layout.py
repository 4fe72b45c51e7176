"""Conversions between the oracle's strength order and the library's (test glue only).

Oracle, per sphere: [S: proxies then image nodes | R: image nodes | D: image nodes] x 3.
Library, per sphere: [proxies x 3 | per image node: S(3) R(3) D(3)].
"""
import numpy as np


def oracle_to_lib(disc, lam_list):
    out = []
    for k, sp in enumerate(disc.spheres):
        N, ni = sp.proxy.shape[0], sp.image.shape[0]
        l = np.asarray(lam_list[k])
        f = l[:3 * (N + ni)].reshape(-1, 3)
        t = l[3 * (N + ni):3 * (N + 2 * ni)].reshape(-1, 3)
        d = l[3 * (N + 2 * ni):].reshape(-1, 3)
        out.append(f[:N].ravel())
        out.append(np.concatenate([f[N:], t, d], axis=1).ravel())
    return np.concatenate(out)


def lib_to_oracle(disc, lam):
    out, off = [], 0
    for sp in disc.spheres:
        N, ni = sp.proxy.shape[0], sp.image.shape[0]
        prox = lam[off:off + 3 * N].reshape(-1, 3)
        img = lam[off + 3 * N:off + 3 * N + 9 * ni].reshape(-1, 9)
        off += 3 * N + 9 * ni
        out.append(np.concatenate([prox.ravel(), img[:, 0:3].ravel(), img[:, 3:6].ravel(), img[:, 6:9].ravel()]))
    return out
