"""Gaussian RBF, periodisation and the diagonal symbols (FP64).

Paper passages:
* Sec. 2.1 Eq. (rbf): phi(r) = exp(-eps^2 r^2).
* Sec. 2.1 Eq. (periodic_rbf): phi_per(x) = sum_m phi(x - 2 m T).
* Sec. 2.2 Eqs. (set_centers), (set_Xtilde): centers c_j = -T + j 2T/N and grid
  x_i = -T + i 2T/L, L = s N (0-based j, i here).
* Sec. 2.2 Eq. (matrix_entries): A^c_ij = phi_per(x_i - c_j).  Because
  x_i - c_j = (i - s j) h_L, A^c_ij = g((i - s j) mod L) with the periodised
  samples g(m) = sum_p phi((m + p L) h_L), m in Z_L.
* Lemma 4.2 and Sec. 3.1 Eq. (explicit_d): the diagonals of B are DFTs of the
  kernel sampled on the (shifted) grids.  Written on the oversampled grid this is
  one real, even sequence  Ghat = DFT_L(g)  (unnormalised DFT); the paper's d_i
  are its entries regrouped by the permutation Pi.
* Sec. 6.1 Example 6.1: phi''(r) = -2 eps^2 exp(-eps^2 r^2) (1 - 2 eps^2 r^2).
* Sec. 6.3 (the flower-domain Helmholtz problem, du/dn = 0 on the outer
  boundary): Neumann rows need the first derivative, the derivative of
  Eq. (rbf): phi'(r) = -2 eps^2 r exp(-eps^2 r^2).

Reading of the image sum (periodic_rbf is an infinite sum): it is truncated at
|p| <= p_max with p_max chosen so that the first omitted image is below 1e-300
of the kernel's peak; ``tests/test_oracle_rbf.py`` pins this against a much
larger p_max and against a brute-force double loop.
"""
import numpy as np


def phi(r, eps):
    """Gaussian RBF, Eq. (rbf)."""
    return np.exp(-(eps * r) ** 2)


def dphi(r, eps):
    """First derivative of the Gaussian RBF (for Neumann rows, Sec. 6.3)."""
    e2 = eps * eps
    return -2.0 * e2 * r * np.exp(-e2 * r * r)


def d2phi(r, eps):
    """Second derivative of the Gaussian RBF (Example 6.1)."""
    e2 = eps * eps
    return -2.0 * e2 * np.exp(-e2 * r * r) * (1.0 - 2.0 * e2 * r * r)


def image_count(eps: float, T: float) -> int:
    """Images |p| <= p_max needed so that exp(-(eps*(2T p_max - T))^2) < 1e-300."""
    # The farthest point of the box from a center is at distance <= 2T; the
    # p-th image is at distance >= (2|p|-1) T from any point of the box.
    p = 1
    while (eps * (2 * p - 1) * T) ** 2 < 700.0:
        p += 1
    return p + 1


def periodised_samples(L: int, T: float, eps: float, deriv: int = 0) -> np.ndarray:
    """g(m) = sum_p f((m + p L) h_L) for m = 0..L-1, f = phi (deriv=0) or phi''."""
    hL = 2.0 * T / L
    f = phi if deriv == 0 else d2phi
    P = image_count(eps, T)
    m = np.arange(L, dtype=np.float64)
    # Use the symmetric representative m -> m - L for m > L/2 so the sum is
    # taken around the nearest image; the set of images summed is the same.
    m = np.where(m > L / 2, m - L, m)
    g = np.zeros(L)
    for p in range(-P, P + 1):
        g += f((m + p * L) * hL, eps)
    return g


def symbol(L: int, T: float, eps: float, deriv: int = 0) -> np.ndarray:
    """Ghat = DFT_L(g): real and even (imaginary part is rounding only)."""
    G = np.fft.fft(periodised_samples(L, T, eps, deriv))
    return G.real.copy()


def grid_symbols(grid, deriv: int = 0):
    """Per-dimension symbols of a workloads.Grid (tuple of 1D arrays)."""
    return tuple(symbol(grid.L[d], grid.T[d], grid.eps, deriv) for d in range(grid.dim))
