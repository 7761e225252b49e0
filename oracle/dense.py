"""Dense NumPy formulation of the same timestep, for brute-force cross-checks.

Test infrastructure only. This second implementation shares nothing with the
C oracle except the model it follows (Sec. 3.1 of the paper): it keeps every
voxel (solids included) in dense arrays, streams with ``np.roll`` and finds
bounce-back links from rolled solid masks instead of a neighbour table, and
builds its own lattice tables. Agreement of the two on small lattices pins
the oracle's indexing, streaming, bounce-back, periodic wrap and gradient.

It takes the same readings as the oracle (see its header): the gradient
stencil C = sum_q 18 t_q xi_q phi(x + xi_q), solids contribute phi_s and the
outside of a non-periodic face contributes 0, u = j in the equilibria.
"""
from __future__ import annotations

import numpy as np

# Eq. d3q19 with the same in-group sign order as the oracle's table
_XI = np.array([
    (0, 0, 0),
    (1, 0, 0), (-1, 0, 0), (0, 1, 0), (0, -1, 0), (0, 0, 1), (0, 0, -1),
    (1, 1, 0), (-1, -1, 0), (1, -1, 0), (-1, 1, 0),
    (1, 0, 1), (-1, 0, -1), (1, 0, -1), (-1, 0, 1),
    (0, 1, 1), (0, -1, -1), (0, 1, -1), (0, -1, 1)], dtype=np.int64)
_OPP = np.array([0] + [q + 1 if q % 2 else q - 1 for q in range(1, 19)])
_T = np.array([1 / 3] + [1 / 18] * 6 + [1 / 36] * 12)
_W = np.array([1 / 3] + [1 / 9] * 6)


def _moment_matrix():
    x, y, z = (_XI[:, a].astype(float) for a in range(3))
    c2 = x * x + y * y + z * z
    rows = [
        np.ones(19), 19 * c2 - 30, (21 * c2 ** 2 - 53 * c2 + 24) / 2,
        x, (5 * c2 - 9) * x, y, (5 * c2 - 9) * y, z, (5 * c2 - 9) * z,
        3 * x * x - c2, (3 * c2 - 5) * (3 * x * x - c2),
        y * y - z * z, (3 * c2 - 5) * (y * y - z * z),
        x * y, y * z, x * z,
        (y * y - z * z) * x, (z * z - x * x) * y, (x * x - y * y) * z]
    M = np.array(rows)
    Minv = np.linalg.inv(M)
    return M, Minv


_M, _MINV = _moment_matrix()


class DenseLBM:
    """Dense-grid color LBM. Arrays are indexed [q, z, y, x]."""

    def __init__(self, labels, affinity, periodic, tau_a, tau_b, alpha, beta, force):
        self.pore = (np.asarray(labels) == 0)
        self.phis = np.where(self.pore, 0.0, np.asarray(affinity, dtype=np.float64))
        self.periodic = tuple(int(p) for p in periodic)
        self.tau_a, self.tau_b = tau_a, tau_b
        self.alpha, self.beta = alpha, beta
        self.F = np.asarray(force, dtype=np.float64)
        nz, ny, nx = self.pore.shape
        self.shape = (nz, ny, nx)
        # pad one layer of wall (phi_s = 0, not pore) on each non-periodic axis
        self.pad = [(1, 1) if not self.periodic[2 - ax] else (0, 0) for ax in range(3)]
        self.f = np.zeros((19,) + self.shape)
        self.A = np.zeros((7,) + self.shape)
        self.B = np.zeros((7,) + self.shape)

    def _padded(self, a, fill):
        return np.pad(a, self.pad, mode="constant", constant_values=fill)

    def _unpad(self, a):
        sl = tuple(slice(p[0], a.shape[i] - p[1]) for i, p in enumerate(self.pad))
        return a[sl]

    def _shift(self, a, c, fill):
        """b(x) = a(x + c) with periodic wrap or wall fill."""
        ap = self._padded(a, fill)
        b = np.roll(ap, shift=(-c[2], -c[1], -c[0]), axis=(0, 1, 2))
        return self._unpad(b)

    def init_fluids(self, phi0):
        phi0 = np.asarray(phi0, dtype=np.float64)
        Na = np.where(self.pore, 0.5 * (1 + phi0), 0.0)
        Nb = np.where(self.pore, 0.5 * (1 - phi0), 0.0)
        self.f = _T[:, None, None, None] * self.pore[None].astype(float)
        self.A = _W[:, None, None, None] * Na[None]
        self.B = _W[:, None, None, None] * Nb[None]

    def step(self):
        pore = self.pore
        Na = self.A.sum(0)
        Nb = self.B.sum(0)
        N = Na + Nb
        with np.errstate(invalid="ignore", divide="ignore"):
            phi = np.where(N > 0, (Na - Nb) / np.where(N > 0, N, 1.0), 0.0)
        phi_all = np.where(pore, phi, self.phis)
        C = np.zeros((3,) + self.shape)
        for q in range(1, 19):
            nb = self._shift(phi_all, _XI[q], 0.0)
            C += 18.0 * _T[q] * _XI[q][:, None, None, None] * nb[None]
        cmag = np.sqrt((C * C).sum(0))
        n = np.where(cmag > 0, C / np.where(cmag > 0, cmag, 1.0), 0.0)
        rho = self.f.sum(0)
        j = np.einsum("qa,qzyx->azyx", _XI.astype(float), self.f)
        jj = (j * j).sum(0)
        ac = self.alpha * cmag
        m = np.einsum("kq,qzyx->kzyx", _M, self.f)
        meq = np.zeros_like(m)
        jx, jy, jz = j
        nx, ny, nz = n
        meq[0] = rho
        meq[1] = -11 * rho + 19 * jj - ac
        meq[2] = 3 * rho - 5.5 * jj
        meq[3], meq[5], meq[7] = jx, jy, jz
        meq[4], meq[6], meq[8] = -2 / 3 * jx, -2 / 3 * jy, -2 / 3 * jz
        meq[9] = 2 * jx * jx - jy * jy - jz * jz + 0.5 * ac * (2 * nx * nx - ny * ny - nz * nz)
        meq[10] = -0.5 * (2 * jx * jx - jy * jy - jz * jz)
        meq[11] = jy * jy - jz * jz + 0.5 * ac * (ny * ny - nz * nz)
        meq[12] = -0.5 * (jy * jy - jz * jz)
        meq[13] = jx * jy + 0.5 * ac * nx * ny
        meq[14] = jy * jz + 0.5 * ac * ny * nz
        meq[15] = jx * jz + 0.5 * ac * nx * nz
        tau = self.tau_b + (self.tau_a - self.tau_b) * 0.5 * (1 + phi)
        s_nu = 1.0 / tau
        s_m = 8 * (2 - s_nu) / (8 - s_nu)
        S = np.zeros((19,) + self.shape)
        for k in (1, 2, 9, 10, 11, 12, 13, 14, 15):
            S[k] = s_nu
        for k in (4, 6, 8, 16, 17, 18):
            S[k] = s_m
        fpost = self.f + np.einsum("qk,kzyx->qzyx", _MINV, S * (meq - m))
        fpost += 3 * _T[:, None, None, None] * np.einsum("qa,a->q", _XI.astype(float), self.F)[:, None, None, None]
        udotxi = np.einsum("qa,azyx->qzyx", _XI[:7].astype(float), j)
        ndotxi = np.einsum("qa,azyx->qzyx", _XI[:7].astype(float), n)
        with np.errstate(invalid="ignore", divide="ignore"):
            xa = np.where(N > 0, Nb / np.where(N > 0, N, 1.0), 0.0)
            xb = np.where(N > 0, Na / np.where(N > 0, N, 1.0), 0.0)
        Apost = _W[:, None, None, None] * Na * (1 + 4.5 * udotxi + self.beta * xa * ndotxi)
        Bpost = _W[:, None, None, None] * Nb * (1 + 4.5 * udotxi - self.beta * xb * ndotxi)
        fpost *= pore
        Apost *= pore
        Bpost *= pore
        self.f = self._stream(fpost, 19)
        self.A = self._stream(Apost, 7)
        self.B = self._stream(Bpost, 7)

    def _stream(self, post, Q):
        pore = self.pore
        out = np.zeros_like(post)
        out[0] = post[0]
        for q in range(1, Q):
            c = _XI[q]
            # arrival from the pore upstream of x: post_q(x - c)
            out[q] += self._shift(post[q], -c, 0.0) * pore
            # halfway bounce-back: the target x + c is not a pore
            target_pore = self._shift(pore.astype(float), c, 0.0)
            out[_OPP[q]] += post[q] * (1.0 - target_pore) * pore
        return out

    def site_values(self, a):
        """Flatten [Q, z, y, x] to [Q, N] in lexicographic pore order."""
        return a[:, self.pore]
