"""Pins for oracle.rbf: brute-force periodisation, Poisson-summation closed form."""
import math

import numpy as np
import pytest

from oracle import rbf


def test_d2phi_matches_finite_difference():
    eps = 3.7
    x = np.linspace(-1.3, 1.3, 41)
    hh = 1e-4
    fd = (rbf.phi(x + hh, eps) - 2 * rbf.phi(x, eps) + rbf.phi(x - hh, eps)) / hh ** 2
    assert np.allclose(rbf.d2phi(x, eps), fd, rtol=1e-5, atol=1e-5)


@pytest.mark.parametrize("deriv", [0, 2])
def test_periodised_samples_bruteforce(deriv):
    # Eq. periodic_rbf summed with many more images, one sample at a time.
    L, T, eps = 24, 1.0, 5.0
    f = rbf.phi if deriv == 0 else rbf.d2phi
    g = rbf.periodised_samples(L, T, eps, deriv)
    hL = 2 * T / L
    ref = []
    for m in range(L):
        acc = 0.0
        for p in range(-40, 41):
            acc += float(f((m * hL) - 2 * T * p, eps))
        ref.append(acc)
    ref = np.array(ref)
    assert np.abs(g - ref).max() <= 1e-14 * np.abs(ref).max()


def test_image_truncation_converged():
    for (L, T, eps) in [(64, 1.0, 16.0), (30, 1.5, 2.0), (512, 1.0, 128.0)]:
        P = rbf.image_count(eps, T)
        hL = 2 * T / L
        m = np.arange(L)
        m = np.where(m > L / 2, m - L, m)
        extra = sum(rbf.phi((m + p * L) * hL, eps) for p in list(range(-P - 10, -P)) + list(range(P + 1, P + 11)))
        assert np.all(np.abs(extra) < 1e-290)


def _closed_form(L, T, eps, deriv):
    # Proof of Lemma 4.3: the DFT of equispaced samples of a Gaussian is the
    # periodic summation of its continuous Fourier transform (Poisson summation).
    hL = 2 * T / L
    a = eps * hL
    f = np.arange(L) / L
    out = np.zeros(L)
    for m in range(-8, 9):
        t = f + m
        gauss = math.sqrt(math.pi) / a * np.exp(-(math.pi * t / a) ** 2)
        if deriv == 0:
            out += gauss
        else:
            out += -(2 * math.pi * t / hL) ** 2 * gauss
    return out


@pytest.mark.parametrize("L,T,epsh_L,deriv", [(512, 1.0, 0.5, 0), (256, 1.5, 0.5, 0),
                                               (64, 1.0, 0.1637, 0), (300, 1.0, 1.0, 0),
                                               (512, 1.0, 0.5, 2), (128, 1.0, 0.3, 2)])
def test_symbol_poisson_closed_form(L, T, epsh_L, deriv):
    eps = epsh_L / (2 * T / L)
    G = rbf.symbol(L, T, eps, deriv)
    cf = _closed_form(L, T, eps, deriv)
    scale = np.abs(cf).max()
    assert np.abs(G - cf).max() <= 1e-13 * scale


def test_symbol_real_even():
    L, T, eps = 400, 1.0, 150.0
    Gc = np.fft.fft(rbf.periodised_samples(L, T, eps))
    assert np.abs(Gc.imag).max() < 1e-12 * np.abs(Gc.real).max()
    G = rbf.symbol(L, T, eps)
    assert np.allclose(G[1:], G[1:][::-1], rtol=0, atol=1e-13 * G.max())
    assert np.all(G > 0)
