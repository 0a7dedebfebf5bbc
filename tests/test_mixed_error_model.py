"""CPU check of the error model behind the last Cholesky QR pass of the
mixed path, which forms X + X G (G = R^-1 - I of the nearly orthonormal
block's factor, R^T R = I + E) from BF16 pieces: the piece products left out
(order k in the pieces, 2^-9k relative each) cost about 2 2^-9k |G| per
element, so one piece of each operand suffices when |E|_F <= 1.6e-5 and two
pieces (three products) when |E|_F <= 2.6e-3, both within 3e-8 of the
exact X R^-1; one piece at the larger deviation does not.  BF16 rounding
(round to nearest even, 8 significant bits) is emulated in numpy; the
products and sums are exact (FP64), as the argument assumes."""
import numpy as np
import pytest
import scipy.linalg as sla


def _bf16(x):
    u = np.asarray(x, dtype=np.float32).view(np.uint32).astype(np.uint64)
    u = (u + 0x7FFF + ((u >> 16) & 1)) & 0xFFFF0000
    return u.astype(np.uint32).view(np.float32).astype(np.float64)


def _pieces(x, k):
    out, r = [], np.asarray(x, dtype=np.float64)
    for _ in range(k):
        p = _bf16(r)
        out.append(p)
        r = r - p
    return out


def _block(N, Ns, e_frob, seed):
    """An FP32 block X1 with |X1^T X1 - I|_F close to e_frob."""
    rng = np.random.default_rng(seed)
    Q, _ = np.linalg.qr(rng.normal(size=(N, Ns)))
    P = rng.normal(size=(Ns, Ns))
    P = 0.5 * (P + P.T)
    P *= 0.5 * e_frob / np.linalg.norm(P)
    X1 = (Q @ (np.eye(Ns) + P)).astype(np.float32).astype(np.float64)
    return X1


def _last_pass(X1, k):
    Ns = X1.shape[1]
    E = X1.T @ X1 - np.eye(Ns)
    R = np.linalg.cholesky(np.eye(Ns) + E).T
    Rinv = sla.solve_triangular(R, np.eye(Ns))
    G = Rinv - np.eye(Ns)
    exact = X1 @ Rinv
    xs, gs = _pieces(X1, k), _pieces(G, k)
    corr = sum(xs[a] @ gs[b] for a in range(k) for b in range(k) if a + b < k)
    return np.linalg.norm(E), np.max(np.abs(X1 + corr - exact)) / np.max(np.abs(exact))


@pytest.mark.parametrize("seed", [0, 1])
def test_one_piece_within_fp32_at_small_deviation(seed):
    e, err = _last_pass(_block(3000, 96, 1.6e-5, seed), 1)
    assert e <= 2e-5 and err < 3e-8


@pytest.mark.parametrize("seed", [0, 1])
def test_two_pieces_within_fp32_at_the_larger_threshold(seed):
    X1 = _block(3000, 96, 2.6e-3, seed)
    e, err2 = _last_pass(X1, 2)
    assert 1e-3 < e <= 3e-3 and err2 < 3e-8
    _, err1 = _last_pass(X1, 1)
    assert err1 > 3e-8          # one piece is not enough there
