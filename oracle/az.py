"""Algorithm 1 (AZ) and the direct truncated-SVD least-squares solve, in FP64.

Algorithm 1 (Sec. 3.2.1), with Z* from Sec. 3.2.2 and the randomised low-rank
step of Sec. 3.2.3 ("Low-rank solver for Ax=b": r+p matrix-vector products,
then an SVD of the resulting tall matrix):

  step 1   solve (I - A Z*) A x2 = (I - A Z*) b
           as x2 = R u, u = TSVD_tau(Y) (I - A Z*) b,  Y = (I - A Z*) A R,
           R a random N x k matrix (oracle.philox.rademacher);
  step 2   x1 = Z* (b - A x2);
  step 3   x = x1 + x2.

The truncated SVD keeps the singular values sigma_i > tau * sigma_1 (the
threshold is a parameter; the paper does not fix one).  Reading for the
degenerate case: singular values at the rounding level of A R
(sigma_i <= 1e-13 ||A R||_F) are treated as zero, so that when Omega is the whole
box (Y = 0 up to rounding, rank 0) step 1 returns x2 = 0 and AZ reduces to Z*.

Refinement (not in the paper's Algorithm 1; it is the one step of residual-based
iterative refinement the GPU path performs): r = b - A x in FP64, then
x <- x + AZ(r) with the same R and the same factorisation of Y.

``direct_tsvd`` is the dense comparison: the SVD of the whole M x N matrix A,
truncated at tau * sigma_1 (the "backslash" column of the paper's figures is
played by this solve).
"""
import numpy as np

from .philox import rademacher


class AZ:
    """Reference AZ loop for one Operator (see oracle.operators)."""

    def __init__(self, op, k: int, seed: int, tau: float = 1e-12, chunk: int = 0):
        """chunk > 0 forms the sketch `chunk` columns at a time (the columns are
        independent; this only bounds the host memory of the FFTs)."""
        self.op = op
        self.k = k
        self.seed = seed
        self.tau = tau
        self.R = rademacher(op.N, k, seed)
        step = chunk if chunk > 0 else k
        self.Y = np.empty((op.M + op.Mb, k))
        ar2 = 0.0
        for c0 in range(0, k, step):
            AR = op.A(self.R[:, c0:c0 + step])
            # Y = (I - A Z*) A R, one column per random vector (Sec. 3.2.3).
            self.Y[:, c0:c0 + step] = AR - op.A(op.Zstar(AR))
            ar2 += float(np.sum(AR * AR))
            del AR
        U, sig, Vt = np.linalg.svd(self.Y, full_matrices=False)
        self.sig = sig
        floor = 1e-13 * np.sqrt(ar2)
        self.rank = int(np.sum(sig > max(tau * sig[0], floor)))
        r = self.rank
        self.U = U[:, :r]
        self.Vs = Vt[:r].T / sig[:r]

    def step1(self, b):
        """x2 = R TSVD(Y)^+ (I - A Z*) b."""
        g = b - self.op.A(self.op.Zstar(b))
        u = self.Vs @ (self.U.T @ g)
        return self.R @ u

    def solve_once(self, b):
        x2 = self.step1(b)
        x1 = self.op.Zstar(b - self.op.A(x2))
        return x1 + x2

    def solve(self, b, refine: int = 0):
        b = np.asarray(b, dtype=np.float64)
        if b.ndim == 1:
            b = b[:, None]
        x = self.solve_once(b)
        for _ in range(refine):
            x = x + self.solve_once(b - self.op.A(x))
        return x


def relres(op, x, b):
    """||A x - b|| / ||b|| per right-hand side."""
    b = np.asarray(b, dtype=np.float64)
    if b.ndim == 1:
        b = b[:, None]
    x = np.asarray(x, dtype=np.float64).reshape(op.N, -1)
    return np.linalg.norm(op.A(x) - b, axis=0) / np.linalg.norm(b, axis=0)


def direct_tsvd(A, b, tau: float = 1e-12):
    """Dense truncated-SVD least squares: x = V_r S_r^{-1} U_r^T b."""
    U, sig, Vt = np.linalg.svd(A, full_matrices=False)
    r = int(np.sum(sig > tau * sig[0]))
    b = np.asarray(b, dtype=np.float64)
    if b.ndim == 1:
        b = b[:, None]
    return Vt[:r].T @ ((U[:, :r].T @ b) / sig[:r, None]), r
