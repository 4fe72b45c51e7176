"""Dense and matrix-free FP64 solvers for the MFS system (oracle side).

Notation follows the paper: collocation nodes x_i^(k), sources y^(k) of types S, R, D,
target-from-source blocks G^(kk') = [G_S, G_R, G_D] (Sec. 2.3, the stresslet column
block is empty because N_T = 0 in the final recipe, Sec. 5.1), left row scaling
W = diag(sqrt(w_i) I_3) (Sec. 5.1 remark left-precond) and one-body blocks
B_k = W_k G^(kk) with truncated pseudo-inverse B_k^+ = V Sigma^+ U^T (Sec. 2.2).

Reading of how the left scaling combines with the one-body right preconditioner
(the paper uses both but does not spell out the product): the scaled system
W G lambda = W b (eq. lq2) is preconditioned exactly as eq. resistance, i.e.
B_k := W_k G^(kk), mu_k = B_k lambda_k, off-diagonal blocks W_k G^(kk') B_k'^+,
right-hand side W b.  Velocities are always evaluated unscaled, u = G lambda.

Unknown ordering inside one sphere: [S: proxies then image nodes | R: image nodes |
D: image nodes], three components per source.  Rows: three components per node.
"""
from __future__ import annotations

from dataclasses import dataclass
import math

import numpy as np
import scipy.linalg

from . import kernels
from .geometry import Discretisation


# ---------------------------------------------------------------- building blocks

def source_sets(disc: Discretisation, k: int):
    """Positions of the Stokeslets, rotlets and potential dipoles of sphere k (eq. lin_comb)."""
    sp = disc.spheres[k]
    return np.concatenate([sp.proxy, sp.image], axis=0), sp.image, sp.image


def n_unknowns(disc: Discretisation, k: int) -> int:
    """3 N^(k), eq. Nk with N_S = N + n_img, N_R = N_D = n_img, N_T = 0 (Sec. 5.1)."""
    sp = disc.spheres[k]
    return 3 * (sp.proxy.shape[0] + 3 * sp.image.shape[0])


def n_rows(disc: Discretisation, k: int) -> int:
    return 3 * disc.spheres[k].colloc.shape[0]


def target_from_source(disc: Discretisation, targets, kp: int) -> np.ndarray:
    """Unscaled G(targets, sources of sphere kp) = [G_S, G_R, G_D]."""
    S, R, D = source_sets(disc, kp)
    mu = disc.params.visc
    return np.hstack([kernels.block_matrix(targets, S, "S", mu),
                      kernels.block_matrix(targets, R, "R", mu),
                      kernels.block_matrix(targets, D, "D", mu)])


def row_scale(disc: Discretisation, k: int) -> np.ndarray:
    """Diagonal of W_k: sqrt(w_i) repeated for the three velocity components."""
    w = disc.spheres[k].weight
    if not disc.params.left_precond:
        w = np.ones_like(w)
    return np.repeat(np.sqrt(w), 3)


def scaled_block(disc: Discretisation, k: int, kp: int) -> np.ndarray:
    """W_k G^(kk')."""
    return row_scale(disc, k)[:, None] * target_from_source(disc, disc.spheres[k].colloc, kp)


# ---------------------------------------------------------------- boundary data

@dataclass
class Background:
    """Background flow u_inf(x) = U + E x + omega x x (Sec. 1 eq. bc; Sec. 4 Ex. 2)."""
    U: np.ndarray = None
    E: np.ndarray = None
    omega: np.ndarray = None

    def __call__(self, x):
        u = np.zeros_like(x)
        if self.U is not None:
            u = u + np.asarray(self.U)[None, :]
        if self.E is not None:
            u = u + x @ np.asarray(self.E).T
        if self.omega is not None:
            u = u + np.cross(np.asarray(self.omega)[None, :], x)
        return u


def boundary_velocity(disc, k, x, v, omega, background=None):
    """eq. bc: u_bc = v_k + omega_k x (x - c_k) - u_inf(x)."""
    c = disc.spheres[k].centre
    u = np.asarray(v[k])[None, :] + np.cross(np.asarray(omega[k])[None, :], x - c[None, :])
    if background is not None:
        u = u - background(x)
    return u


def rhs(disc, v, omega, background=None) -> list:
    """W b per sphere, b = u_bc at the collocation nodes (eq. lq, eq. lq2)."""
    out = []
    for k, sp in enumerate(disc.spheres):
        u = boundary_velocity(disc, k, sp.colloc, v, omega, background)
        out.append(row_scale(disc, k) * u.reshape(-1))
    return out


# ---------------------------------------------------------------- one-body factors

@dataclass
class OneBody:
    U: np.ndarray   # (3M, r)
    s: np.ndarray   # (r,)
    V: np.ndarray   # (3N, r)


def one_body_factor(B: np.ndarray, eps_trunc: float) -> OneBody:
    """Thin SVD B = U Sigma V^T, singular values below eps_trunc * sigma_max dropped (Sec. 2.2, App. A.1)."""
    U, s, Vt = np.linalg.svd(B, full_matrices=False)
    keep = s >= eps_trunc * s[0]
    return OneBody(U=U[:, keep], s=s[keep], V=Vt[keep].T)


def one_body_factors(disc: Discretisation) -> list:
    return [one_body_factor(scaled_block(disc, k, k), disc.params.eps_trunc)
            for k in range(len(disc.spheres))]


def pinv_apply(f: OneBody, mu: np.ndarray) -> np.ndarray:
    """eq. transform: lambda_hat = V (Sigma^+ (U^T mu)), the two factors applied in turn."""
    t = f.U.T @ mu
    t = t / (f.s[:, None] if t.ndim == 2 else f.s)
    return f.V @ t


# ---------------------------------------------------------------- the preconditioned operator

class Operator:
    """G_hat of eq. resistance, applied in the paper's three steps (Sec. 2.2)."""

    def __init__(self, disc: Discretisation, factors=None, cache_blocks=True):
        self.disc = disc
        self.P = len(disc.spheres)
        self.f = factors if factors is not None else one_body_factors(disc)
        self.rows = [n_rows(disc, k) for k in range(self.P)]
        self.cols = [n_unknowns(disc, k) for k in range(self.P)]
        self.roff = np.concatenate([[0], np.cumsum(self.rows)])
        self.blocks = None
        if cache_blocks:
            self.blocks = [[scaled_block(disc, k, kp) for kp in range(self.P)] for k in range(self.P)]

    @property
    def n(self):
        return int(self.roff[-1])

    def split(self, x):
        return [x[self.roff[k]:self.roff[k + 1]] for k in range(self.P)]

    def block(self, k, kp):
        return self.blocks[k][kp] if self.blocks is not None else scaled_block(self.disc, k, kp)

    def apply(self, mu):
        mus = self.split(mu)
        # step 1, eq. transform
        lam_hat = [pinv_apply(self.f[k], mus[k]) for k in range(self.P)]
        out = []
        for k in range(self.P):
            # step 2, eq. uAll: all-to-all interaction including the self block
            u_all = sum(self.block(k, kp) @ lam_hat[kp] for kp in range(self.P))
            # step 3: replace the self interaction B lambda_hat by the identity
            out.append(u_all - self.block(k, k) @ lam_hat[k] + mus[k])
        return np.concatenate(out, axis=0)

    def dense(self):
        """G_hat assembled by applying the three steps to the unit vectors."""
        return self.apply(np.eye(self.n))

    def strengths(self, mu):
        """lambda = B^+ mu per sphere, after convergence (Sec. 2.2)."""
        return [pinv_apply(self.f[k], m) for k, m in enumerate(self.split(mu))]


# ---------------------------------------------------------------- solvers

def gmres(apply, b, tol=1e-10, restart=300, max_iter=3000, x0=None):
    """Restarted GMRES with modified Gram-Schmidt Arnoldi and Givens rotations (Saad 2003, Alg. 6.9)."""
    n = b.shape[0]
    x = np.zeros(n) if x0 is None else x0.copy()
    bnorm = np.linalg.norm(b)
    if bnorm == 0.0:
        return x, 0, 0.0
    iters = 0
    while True:
        r = b - apply(x)
        beta = np.linalg.norm(r)
        if beta / bnorm <= tol or iters >= max_iter:
            return x, iters, beta / bnorm
        m = restart
        Q = np.zeros((n, m + 1))
        H = np.zeros((m + 1, m))
        cs = np.zeros(m)
        sn = np.zeros(m)
        g = np.zeros(m + 1)
        g[0] = beta
        Q[:, 0] = r / beta
        j_used = 0
        for j in range(m):
            w = apply(Q[:, j])
            for i in range(j + 1):
                H[i, j] = np.dot(Q[:, i], w)
                w = w - H[i, j] * Q[:, i]
            H[j + 1, j] = np.linalg.norm(w)
            if H[j + 1, j] > 0:
                Q[:, j + 1] = w / H[j + 1, j]
            for i in range(j):
                t = cs[i] * H[i, j] + sn[i] * H[i + 1, j]
                H[i + 1, j] = -sn[i] * H[i, j] + cs[i] * H[i + 1, j]
                H[i, j] = t
            den = math.hypot(H[j, j], H[j + 1, j])
            cs[j], sn[j] = H[j, j] / den, H[j + 1, j] / den
            H[j, j] = den
            H[j + 1, j] = 0.0
            g[j + 1] = -sn[j] * g[j]
            g[j] = cs[j] * g[j]
            iters += 1
            j_used = j + 1
            if abs(g[j + 1]) / bnorm <= tol or iters >= max_iter:
                break
        y = scipy.linalg.solve_triangular(H[:j_used, :j_used], g[:j_used])
        x = x + Q[:, :j_used] @ y


@dataclass
class Solution:
    lam: list            # per sphere strengths, ordering [S | R | D] x 3 components
    mu: np.ndarray = None
    iters: int = 0
    rel_residual: float = 0.0


class DenseSystem:
    """O2: dense G_hat (eq. resistance) assembled from the three steps, LU-factored once."""

    def __init__(self, disc, op=None):
        self.disc = disc
        self.op = op or Operator(disc)
        self.A = self.op.dense()
        self.lu = scipy.linalg.lu_factor(self.A)

    def solve(self, v, omega, background=None) -> Solution:
        b = np.concatenate(rhs(self.disc, v, omega, background))
        mu = scipy.linalg.lu_solve(self.lu, b)
        res = np.linalg.norm(self.A @ mu - b) / max(np.linalg.norm(b), 1e-300)
        return Solution(lam=self.op.strengths(mu), mu=mu, iters=0, rel_residual=res)


def solve_o2(disc, v, omega, background=None, op=None) -> Solution:
    """O2: dense LU solve of eq. resistance (see DenseSystem)."""
    return DenseSystem(disc, op).solve(v, omega, background)


def solve_o3(disc, v, omega, background=None, op=None, tol=1e-10, restart=300) -> Solution:
    """O3: matrix-free GMRES on eq. resistance with the three-step apply."""
    op = op or Operator(disc)
    b = np.concatenate(rhs(disc, v, omega, background))
    mu, it, rr = gmres(op.apply, b, tol=tol, restart=restart)
    return Solution(lam=op.strengths(mu), mu=mu, iters=it, rel_residual=rr)


def solve_o1(disc, v, omega, background=None) -> Solution:
    """O1: the plain method, dense least squares W G lambda = W b (eq. lq2) by Householder QR."""
    P = len(disc.spheres)
    A = np.vstack([np.hstack([scaled_block(disc, k, kp) for kp in range(P)]) for k in range(P)])
    b = np.concatenate(rhs(disc, v, omega, background))
    Q, R = np.linalg.qr(A, mode="reduced")
    lam = scipy.linalg.solve_triangular(R, Q.T @ b)
    cols = np.concatenate([[0], np.cumsum([n_unknowns(disc, k) for k in range(P)])])
    res = np.linalg.norm(A @ lam - b) / max(np.linalg.norm(b), 1e-300)
    return Solution(lam=[lam[cols[k]:cols[k + 1]] for k in range(P)], rel_residual=res)


# ---------------------------------------------------------------- outputs

def split_strengths(disc, k, lam_k):
    sp = disc.spheres[k]
    nS = sp.proxy.shape[0] + sp.image.shape[0]
    nI = sp.image.shape[0]
    f = lam_k[:3 * nS].reshape(-1, 3)
    t = lam_k[3 * nS:3 * (nS + nI)].reshape(-1, 3)
    d = lam_k[3 * (nS + nI):].reshape(-1, 3)
    return f, t, d


def forces_torques(disc, lam):
    """Sec. 2.3 remark: F = sum f_alpha, T = sum t_alpha + sum (y_alpha - c) x f_alpha."""
    P = len(disc.spheres)
    F = np.zeros((P, 3))
    T = np.zeros((P, 3))
    for k in range(P):
        f, t, _ = split_strengths(disc, k, lam[k])
        yS, _, _ = source_sets(disc, k)
        F[k] = f.sum(axis=0)
        T[k] = t.sum(axis=0) + np.cross(yS - disc.spheres[k].centre[None, :], f).sum(axis=0)
    return F, T


def velocity(disc, lam, x, chunk=2048):
    """u(x) = sum over all spheres of G(x, sources) lambda (unscaled), eq. lin_comb."""
    x = np.asarray(x, dtype=np.float64).reshape(-1, 3)
    u = np.zeros(x.shape[0] * 3)
    for s in range(0, x.shape[0], chunk):
        xs = x[s:s + chunk]
        acc = np.zeros(xs.shape[0] * 3)
        for kp in range(len(disc.spheres)):
            acc += target_from_source(disc, xs, kp) @ lam[kp]
        u[3 * s:3 * s + acc.shape[0]] = acc
    return u.reshape(-1, 3)


def residual_max(disc, lam, v, omega, background=None):
    """eq. residual: max over check points of eq. residual_x."""
    worst = 0.0
    for k in range(len(disc.spheres)):
        x = disc.check[k]
        u = velocity(disc, lam, x)
        ubc = boundary_velocity(disc, k, x, v, omega, background)
        nb = np.linalg.norm(ubc, axis=1)
        err = np.linalg.norm(u - ubc, axis=1) / np.where(nb > 0, nb, 1.0)
        worst = max(worst, float(err.max()))
    return worst


def resistance_matrix(disc, system=None):
    """6P x 6P matrix mapping (v, omega) to (F, T), from 6P unit solves with O2."""
    P = len(disc.spheres)
    system = system or DenseSystem(disc)
    Rm = np.zeros((6 * P, 6 * P))
    for j in range(6 * P):
        v = np.zeros((P, 3))
        om = np.zeros((P, 3))
        k, c = divmod(j, 6)
        if c < 3:
            v[k, c] = 1.0
        else:
            om[k, c - 3] = 1.0
        sol = system.solve(v, om)
        F, T = forces_torques(disc, sol.lam)
        Rm[:, j] = np.concatenate([np.concatenate([F[i], T[i]]) for i in range(P)])
    return Rm


# ---------------------------------------------------------------- mobility (bordered system)
#
# The paper solves the resistance problem and defers the mobility problem (forces and torques
# given, rigid velocities unknown) to another paper.  Reading used here: the rigid velocities
# U_k = (V_k, Omega_k) become unknowns of eq. bc, and the force/torque of each sphere, taken
# from lambda = B^+ mu by the Sec. 2.3 remark, is prescribed:
#   G_hat mu - W (V_k + Omega_k x (x - c_k)) = -W u_inf(x)          (collocation rows)
#   s_F F_k(B_k^+ mu_k) = s_F F_k^given,  s_T T_k(B_k^+ mu_k) = s_T T_k^given
# with s_F = 1/(6 pi mu a), s_T = 1/(8 pi mu a^3) so that the border rows carry velocity scale.

def rigid_block(disc, k) -> np.ndarray:
    """(3 M_k, 6) matrix of the rigid velocity V + Omega x (x - c_k) at the nodes of sphere k."""
    sp = disc.spheres[k]
    r = sp.colloc - sp.centre[None, :]
    m = r.shape[0]
    out = np.zeros((m, 3, 6))
    out[:, :, :3] = np.eye(3)[None, :, :]
    # Omega x r = [[0, r3, -r2], [-r3, 0, r1], [r2, -r1, 0]] Omega
    out[:, 0, 4], out[:, 0, 5] = r[:, 2], -r[:, 1]
    out[:, 1, 3], out[:, 1, 5] = -r[:, 2], r[:, 0]
    out[:, 2, 3], out[:, 2, 4] = r[:, 1], -r[:, 0]
    return out.reshape(3 * m, 6)


def ft_functional(disc, k) -> np.ndarray:
    """(6, 3 N_k) matrix taking lambda_k to (F_k, T_k) (Sec. 2.3 remark)."""
    sp = disc.spheres[k]
    yS, _, _ = source_sets(disc, k)
    nS, nI = yS.shape[0], sp.image.shape[0]
    out = np.zeros((6, n_unknowns(disc, k)))
    for j in range(nS):
        out[0:3, 3 * j:3 * j + 3] = np.eye(3)
        r = yS[j] - sp.centre
        # (r x f) = [[0, -r3, r2], [r3, 0, -r1], [-r2, r1, 0]] f
        out[3:6, 3 * j:3 * j + 3] = np.array([[0, -r[2], r[1]], [r[2], 0, -r[0]], [-r[1], r[0], 0]])
    for j in range(nI):
        col = 3 * (nS + j)
        out[3:6, col:col + 3] = np.eye(3)
    return out


class MobilitySystem:
    """Dense bordered mobility system (reading above), LU-factored once."""

    def __init__(self, disc, op=None):
        self.disc = disc
        self.op = op or Operator(disc)
        P = len(disc.spheres)
        a, mu_v = disc.radius, disc.params.visc
        self.sF, self.sT = 1.0 / (6 * math.pi * mu_v * a), 1.0 / (8 * math.pi * mu_v * a ** 3)
        n = self.op.n
        A = np.zeros((n + 6 * P, n + 6 * P))
        A[:n, :n] = self.op.dense()
        for k in range(P):
            rows = slice(self.op.roff[k], self.op.roff[k + 1])
            A[rows, n + 6 * k:n + 6 * k + 6] = -row_scale(disc, k)[:, None] * rigid_block(disc, k)
            f = self.op.f[k]
            # FT(B^+ mu_k) with B^+ applied as its two factors
            ftb = ((ft_functional(disc, k) @ f.V) / f.s[None, :]) @ f.U.T
            ftb[:3] *= self.sF
            ftb[3:] *= self.sT
            A[n + 6 * k:n + 6 * k + 6, rows] = ftb
        self.A = A
        self.lu = scipy.linalg.lu_factor(A)

    def solve(self, F, T, background=None):
        disc, op = self.disc, self.op
        P = len(disc.spheres)
        n = op.n
        b = np.zeros(n + 6 * P)
        if background is not None:
            zero = np.zeros((P, 3))
            # -W u_inf: the boundary data of a fixed sphere in the background flow
            b[:n] = np.concatenate(rhs(disc, zero, zero, background))
        for k in range(P):
            b[n + 6 * k:n + 6 * k + 3] = self.sF * np.asarray(F[k])
            b[n + 6 * k + 3:n + 6 * k + 6] = self.sT * np.asarray(T[k])
        x = scipy.linalg.lu_solve(self.lu, b)
        mu = x[:n]
        U = x[n:].reshape(P, 6)
        return U[:, :3].copy(), U[:, 3:].copy(), Solution(lam=op.strengths(mu), mu=mu)
