"""Pins for the oracle's finite-difference Laplacian (Sec. 5: twelfth-order
central differences on a periodic cell)."""
from fractions import Fraction

import numpy as np
import pytest

from oracle import fd, hamiltonian


def _weights_by_moment_solve(n):
    """Central second-derivative weights from the moment conditions
    sum_p w_|p| p^(2q) = 2 delta_{q,1}, q = 0..n, solved exactly in rationals
    (an independent route to the closed form)."""
    A = [[Fraction(1 if p == 0 else 2) * Fraction(p) ** (2 * q) if not (p == 0 and q == 0)
          else Fraction(1) for p in range(n + 1)] for q in range(n + 1)]
    b = [Fraction(2 if q == 1 else 0) for q in range(n + 1)]
    # Gauss-Jordan elimination in exact arithmetic.
    m = len(b)
    for c in range(m):
        piv = next(r for r in range(c, m) if A[r][c] != 0)
        A[c], A[piv] = A[piv], A[c]
        b[c], b[piv] = b[piv], b[c]
        for r in range(m):
            if r != c and A[r][c] != 0:
                f = A[r][c] / A[c][c]
                A[r] = [x - f * y for x, y in zip(A[r], A[c])]
                b[r] -= f * b[c]
    return [b[i] / A[i][i] for i in range(m)]


@pytest.mark.parametrize("order", [2, 4, 8, 12])
def test_weights_match_exact_moment_solution(order):
    w = fd.fd_weights(order)
    exact = _weights_by_moment_solve(order // 2)
    np.testing.assert_allclose(w, [float(x) for x in exact], rtol=1e-14, atol=0)


def test_twelfth_order_exactness_and_no_more():
    w = fd.fd_weights(12)
    p = np.arange(-6, 7)
    wp = w[np.abs(p)]
    for d in range(14):
        target = 2.0 if d == 2 else 0.0
        assert abs(np.sum(wp * p.astype(float) ** d) - target) < 1e-9 * 6.0 ** d
    assert abs(np.sum(wp * p.astype(float) ** 14)) > 1.0


def test_convergence_order_on_periodic_sine():
    errs = []
    for n in (24, 48):
        h = 2 * np.pi / n
        x = np.arange(n) * h
        u = np.sin(3 * x)
        L = fd.laplacian_1d(n, h, 12)
        errs.append(np.max(np.abs(L @ u + 9 * np.sin(3 * x))))
    rate = np.log2(errs[0] / errs[1])
    assert 11.0 < rate < 13.5


def _symbol(theta, w):
    return -w[0] - 2.0 * sum(w[p] * np.cos(p * theta) for p in range(1, len(w)))


def test_plane_wave_eigenvector_noncubic_grid():
    """A plane wave on a 5 x 7 x 9 grid with different spacings is an
    eigenvector of the assembled Laplacian with the FD symbol per axis,
    which pins the index order k = i + nx j + nx ny l."""
    nx, ny, nz = 5, 7, 9
    hx, hy, hz = 0.3, 0.45, 0.6
    w = fd.fd_weights(12)
    Lap = fd.laplacian_3d(nx, ny, nz, hx, hy, hz, 12)
    mx, my, mz = 2, 3, 1
    l, j, i = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    tx, ty, tz = 2 * np.pi * mx / nx, 2 * np.pi * my / ny, 2 * np.pi * mz / nz
    u = np.cos(tx * i + ty * j + tz * l).ravel()
    lam = -(_symbol(tx, w) / hx ** 2 + _symbol(ty, w) / hy ** 2 + _symbol(tz, w) / hz ** 2)
    np.testing.assert_allclose(Lap @ u, lam * u, atol=1e-11 * np.abs(lam))


@pytest.mark.parametrize("n,L", [(6, 4.0), (8, 5.3)])
def test_free_electron_dispersion(n, L):
    """V = 0, no projectors: spectrum of H equals {1/2 sum_a s(2 pi m_a/n)/h^2}."""
    h = L / n
    w = fd.fd_weights(12)
    H = hamiltonian.hamiltonian_dense(n, L, np.zeros(n ** 3))
    lam = np.linalg.eigvalsh(H)
    s1 = np.array([_symbol(2 * np.pi * m / n, w) for m in range(n)]) / h ** 2
    analytic = np.sort(0.5 * (s1[:, None, None] + s1[None, :, None] + s1[None, None, :]).ravel())
    np.testing.assert_allclose(lam, analytic, atol=1e-11 * analytic.max())
    assert abs(lam[0]) < 1e-11


def test_dense_laplacian_against_loop_brute_force():
    """Assemble -1/2 Lap + V on a 5 x 5 x 5 grid by explicit loops over grid
    points and neighbours and compare with the Kronecker assembly."""
    n, L = 5, 3.0
    h = L / n
    w = fd.fd_weights(12)
    rng = np.random.default_rng(3)
    V = rng.normal(size=n ** 3)
    B = np.zeros((n ** 3, n ** 3))
    for l in range(n):
        for j in range(n):
            for i in range(n):
                k = i + n * j + n * n * l
                B[k, k] += -0.5 * 3 * w[0] / h ** 2 + V[k]
                for p in range(1, 7):
                    for s in (p, -p):
                        for kk in ((i + s) % n + n * j + n * n * l,
                                   i + n * ((j + s) % n) + n * n * l,
                                   i + n * j + n * n * ((l + s) % n)):
                            B[k, kk] += -0.5 * w[p] / h ** 2
    H = hamiltonian.hamiltonian_dense(n, L, V)
    np.testing.assert_allclose(H, B, atol=1e-12)
