"""The least-squares operator A, the full-box operator A^c and the plain inverse Z*.

Paper passages followed:
* Sec. 2.2 Eqs. (matrix_entries)-(circulant_system): A^c (L x N), A^c_ij =
  phi_per(x_i - c_j), applied here as a circulant convolution on the L-grid:
  A^c a = IDFT_L( Ghat * tile_s(DFT_N a) ), which is the block-diagonalisation
  B = P Pi A^c F of Sec. 3.1 Eq. (blockdiagonal_system) written without the
  permutation Pi (the s polyphase blocks are the s aliases k + qN of each
  frequency k).
* Sec. 2.3: A = R Pi A^c (rows of the kept points), E = R^dagger (zero fill).
* Sec. 3.1 Eq. (B_pinv): the pseudo-inverse is diagonal per alias group;
  Z* = F B^dagger P E (Sec. 3.2.2) becomes, per frequency k of the N-grid,
      ahat(k) = sum_q Ghat(k+qN) Y(k+qN) / S_k,  S_k = sum_q Ghat(k+qN)^2,
  with Y = DFT_L(E y) and a = IDFT_N(ahat).
* Sec. 5.1 Eqs. (circulant_system_2d), (B_pinv_2d): 2D is the tensor product;
  the coefficient index is j = jx*Ny + jy and the grid index i = ix*Ly + iy
  (x-major), as in the paper's j = (m-1) N^y + n.
* Sec. 6.1 Example 6.1 (the ODE u'' + k0^2 u = g on [-1, 1] with Dirichlet rows
  at the end points): 1D interior rows -(phi'' + k0^2 phi) / (2 eps^2), boundary
  rows phi_j(x_b) times the weight, Z* with zero columns for those rows.
* Sec. 6.2 (Ai_2d_bvp and the three-term splitting of A^ic): the Helmholtz
  rows are -(phi''_x phi_y + phi_x phi''_y + k0^2 phi_x phi_y) divided by
  2 eps^2 (the normalisation of Example 6.1 read as a division, so the rows
  have O(1) entries; k0 = 0 is the Poisson operator), and Z* = [F B^dagger P E, 0]
  has zero columns for the boundary rows.

* Sec. 6.3 (the flower-domain Helmholtz problem: du/dn = 0 on the outer
  boundary, u = 0 on the inner one): a boundary point with a nonzero unit
  normal n gives a Neumann row n . grad phi_j(p_b), the sum over dimensions
  of n_d times the product of phi' in dimension d and phi in the others.

Reading of the Neumann rows: the paper does not say how it scales them.  They
are divided by eps (the derivative of phi is O(eps)), so that their entries
are O(1) like the normalised interior rows, and then multiplied by the
boundary weight like the Dirichlet rows; the data du/dn is scaled the same way.

Reading of the symbol truncation: S_k^{-1} is replaced by 0 when
S_k <= tau_sym^2 * max S (tau_sym = 0 gives the exact pseudo-inverse).
"""
import os

import numpy as np
import scipy.fft as sfft

from . import rbf

# The DFTs of Sec. 3.1 (F, and the per-dimension transforms of Sec. 5.1) are
# library FFTs; they run on every host core (the transform is the same one
# numpy.fft computes, up to rounding).
WORKERS = os.cpu_count() or 1


class Operator:
    """A^c, A and Z* for one problem (approximation or Poisson collocation)."""

    def __init__(self, grid, mask, kind="approx", boundary=None, weight=1.0, tau_sym=0.0, k0=0.0, normals=None):
        self.grid = grid
        self.dim = grid.dim
        self.n = tuple(int(v) for v in grid.n)
        self.s = tuple(int(v) for v in grid.s)
        self.L = grid.L
        self.N = grid.N
        self.Ltot = grid.Ltot
        self.eps = grid.eps
        self.kind = kind
        self.k0 = float(k0)
        self.mask = np.asarray(mask).reshape(-1).astype(np.uint8)
        assert self.mask.size == self.Ltot
        self.idx = np.flatnonzero(self.mask)          # compact index map (S1)
        self.M = self.idx.size
        self.boundary = None if boundary is None else np.asarray(boundary, dtype=np.float64)
        self.Mb = 0 if self.boundary is None else self.boundary.shape[0]
        self.weight = float(weight)
        # (Mb, dim) outward unit normals; a zero row keeps the Dirichlet row
        self.normals = None if normals is None else np.asarray(normals, dtype=np.float64).reshape(self.Mb, self.dim)
        self.neumann = (np.zeros(self.Mb, bool) if self.normals is None
                        else np.any(self.normals != 0.0, axis=1))
        self.G0 = rbf.grid_symbols(grid, 0)
        if kind == "poisson":
            self.G2 = rbf.grid_symbols(grid, 2)
        self.Ghat = self._full_symbol()               # on the L-grid, shape self.L
        S = self._fold(self.Ghat ** 2)
        thr = tau_sym * tau_sym * S.max()
        self.S = S
        self.Sinv = np.where(S > thr, 1.0 / np.where(S > 0, S, 1.0), 0.0)

    # ------------------------------------------------------------------ symbols
    def _full_symbol(self):
        if self.dim == 1:
            if self.kind == "approx":
                return self.G0[0].copy()
            return -(self.G2[0] + self.k0 ** 2 * self.G0[0]) / (2.0 * self.eps ** 2)
        gx, gy = self.G0
        if self.kind == "approx":
            return np.outer(gx, gy)
        hx, hy = self.G2
        return -(np.outer(hx, gy) + np.outer(gx, hy) + self.k0 ** 2 * np.outer(gx, gy)) / (2.0 * self.eps ** 2)

    def _fold(self, F):
        """Sum an L-grid array over each alias group {k + qN}: result on the N-grid."""
        if self.dim == 1:
            return F.reshape(self.s[0], self.n[0], *F.shape[1:]).sum(axis=0)
        sx, sy = self.s
        nx, ny = self.n
        return F.reshape(sx, nx, sy, ny, *F.shape[2:]).sum(axis=(0, 2))

    def _tile(self, F):
        if self.dim == 1:
            return np.tile(F, (self.s[0],) + (1,) * (F.ndim - 1))
        return np.tile(F, (self.s[0], self.s[1]) + (1,) * (F.ndim - 2))

    # ------------------------------------------------------------ FFT operators
    def _to_grid(self, v, shape):
        return v.reshape(*shape, v.shape[-1])

    def Ac(self, a):
        """A^c a on the full L-grid; a is (N, ncol); returns (Ltot, ncol)."""
        a = np.asarray(a, dtype=np.float64)
        a2 = self._to_grid(a, self.n)
        axes = tuple(range(self.dim))
        ah = sfft.fftn(a2, axes=axes, workers=WORKERS)
        G = self.Ghat.reshape(*self.L, 1)
        v = sfft.ifftn(G * self._tile(ah), axes=axes, workers=WORKERS).real
        return v.reshape(self.Ltot, -1)

    def boundary_rows(self, a):
        """w * A^b a: Dirichlet rows phi_j(p_b) (Sec. 6.1, 6.2) and Neumann rows
        n . grad phi_j(p_b) / eps (Sec. 6.3) at the boundary points."""
        a = np.asarray(a, dtype=np.float64)
        F = self._boundary_factors()
        if self.dim == 1:
            (B, dB), = F
            out = B @ a
            if self.neumann.any():
                nb = self.neumann
                out[nb] = (self.normals[nb, 0][:, None] * (dB[nb] @ a)) / self.eps
            return self.weight * out
        (Bx, dBx), (By, dBy) = F
        a2 = a.reshape(self.n[0], self.n[1], -1)

        def sep(X, Y):
            return np.einsum("bjc,bj->bc", np.einsum("bi,ijc->bjc", X, a2), Y)

        out = sep(Bx, By)
        if self.neumann.any():
            nb = self.neumann
            nx, ny = self.normals[nb, 0][:, None], self.normals[nb, 1][:, None]
            out[nb] = (nx * sep(dBx[nb], By[nb]) + ny * sep(Bx[nb], dBy[nb])) / self.eps
        return self.weight * out

    def _boundary_factors(self):
        """Per dimension, phi_per and phi_per' between the boundary points and
        the centers: two (Mb, n_d) arrays (Eq. periodic_rbf, image by image)."""
        out = []
        for d in range(self.dim):
            T = self.grid.T[d]
            c = -T + np.arange(self.n[d]) * (2.0 * T / self.n[d])
            P = rbf.image_count(self.eps, T)
            diff = self.boundary[:, d][:, None] - c[None, :]
            acc = np.zeros_like(diff)
            dacc = np.zeros_like(diff)
            for p in range(-P, P + 1):
                acc += rbf.phi(diff - 2.0 * p * T, self.eps)
                dacc += rbf.dphi(diff - 2.0 * p * T, self.eps)
            out.append((acc, dacc))
        return out

    def collocation_rhs(self, f, g):
        """b = [f / (2 eps^2); w g], the Neumann entries of g (du/dn) also divided
        by eps: the row scalings above applied to the data (f: (M, c), g: (Mb, c))."""
        g = self.weight * np.asarray(g, dtype=np.float64).copy()
        g[self.neumann] /= self.eps
        return np.concatenate([np.asarray(f, dtype=np.float64) / (2.0 * self.eps ** 2), g], axis=0)

    def boundary_dense(self):
        """The boundary block w * A^b as a dense (Mb, N) matrix, row by row."""
        F = self._boundary_factors()
        if self.dim == 1:
            (B, dB), = F
            Ab = B.copy()
            nb = self.neumann
            if nb.any():
                Ab[nb] = self.normals[nb, 0][:, None] * dB[nb] / self.eps
            return self.weight * Ab
        (Bx, dBx), (By, dBy) = F
        Ab = (Bx[:, :, None] * By[:, None, :]).reshape(self.Mb, -1)
        nb = self.neumann
        if nb.any():
            nx, ny = self.normals[nb, 0][:, None, None], self.normals[nb, 1][:, None, None]
            Ab[nb] = ((nx * dBx[nb][:, :, None] * By[nb][:, None, :] +
                       ny * Bx[nb][:, :, None] * dBy[nb][:, None, :]) / self.eps).reshape(nb.sum(), -1)
        return self.weight * Ab

    def A(self, a):
        """Rows of the least-squares matrix: kept grid rows, then boundary rows."""
        v = self.Ac(a)[self.idx]
        if self.Mb:
            v = np.concatenate([v, self.boundary_rows(a)], axis=0)
        return v

    def extend(self, y):
        """E y: zero fill of the kept rows onto the L-grid (boundary rows dropped)."""
        y = np.asarray(y, dtype=np.float64)
        out = np.zeros((self.Ltot, y.shape[1]))
        out[self.idx] = y[: self.M]
        return out

    def Zstar_grid(self, yL):
        """pinv(A^c) applied to a full L-grid array (Ltot, ncol) -> (N, ncol)."""
        axes = tuple(range(self.dim))
        Y = sfft.fftn(self._to_grid(yL, self.L), axes=axes, workers=WORKERS)
        G = self.Ghat.reshape(*self.L, 1)
        ah = self._fold(G * Y) * self.Sinv.reshape(*self.n, 1)
        return sfft.ifftn(ah, axes=axes, workers=WORKERS).real.reshape(self.N, -1)

    def Zstar(self, y):
        """Z* y = F B^dagger P E y (zero columns for boundary rows)."""
        return self.Zstar_grid(self.extend(y))

    # ------------------------------------------------------------ dense forms
    def Ac_dense(self):
        """A^c formed entry by entry from the periodised samples (tiny sizes)."""
        mats = []
        for d in range(self.dim):
            Ld, nd, sd = self.L[d], self.n[d], self.s[d]
            i = np.arange(Ld)[:, None]
            j = np.arange(nd)[None, :]
            g0 = rbf.periodised_samples(Ld, self.grid.T[d], self.eps, 0)
            m0 = g0[(i - sd * j) % Ld]
            if self.kind == "poisson":
                g2 = rbf.periodised_samples(Ld, self.grid.T[d], self.eps, 2)
                mats.append((m0, g2[(i - sd * j) % Ld]))
            else:
                mats.append((m0, None))
        if self.dim == 1:
            if self.kind == "approx":
                return mats[0][0]
            return -(mats[0][1] + self.k0 ** 2 * mats[0][0]) / (2.0 * self.eps ** 2)
        (ax0, ax2), (ay0, ay2) = mats
        if self.kind == "approx":
            return np.kron(ax0, ay0)
        return -(np.kron(ax2, ay0) + np.kron(ax0, ay2) + self.k0 ** 2 * np.kron(ax0, ay0)) / (2.0 * self.eps ** 2)

    def A_dense(self):
        A = self.Ac_dense()[self.idx]
        if self.Mb:
            A = np.concatenate([A, self.boundary_dense()], axis=0)
        return A

    def Zstar_dense(self, rcond=1e-14):
        """Definition form: pinv(A^c) E, with zero columns for the boundary rows."""
        Zc = np.linalg.pinv(self.Ac_dense(), rcond=rcond)
        Z = Zc[:, self.idx]
        if self.Mb:
            Z = np.concatenate([Z, np.zeros((self.N, self.Mb))], axis=1)
        return Z
