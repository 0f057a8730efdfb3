"""The 2 x 2 identities the n = 2 (one dust species) kernels rely on, checked
with plain matrix arithmetic on the CPU (no GPU, no library).

For X = [[-x, x], [y, -y]] (a scaled velocity-form generator with zero row
sums), X^2 = tr(X) X with tr(X) = -(x + y), so every polynomial in X is
c_0 I + beta X:

* Taylor (the forward): T_m(X) = I + b X with b = sum_{k=1..m} b_k tr^(k-1),
  and a squaring maps W = P - I to 2 W + W^2 = (2 - p - q) W for
  W = [[-p, p], [q, -q]];
* Pade (the variant, Eq. PadeEqu): R_mm = D^-1 N = I + (b_N - b_D) /
  (c_0 + b_D tr) X with N = c_0 I + b_N X, D = N(-X) = c_0 I + b_D X;
* bound test: the 1-norm of c_0 I + beta X is max(|c_0 - beta x| + |beta y|,
  |beta x| + |c_0 - beta y|), and |X^q|_1 = |tr|^(q-1) (x + y).
"""
import math

import numpy as np
import pytest

import oracle


def gen(x, y):
    return np.array([[-x, x], [y, -y]])


CASES = [(1e-3, 2e-3), (0.3, 0.05), (1.2, 1.9), (2.5e-9, 4e-12), (0.0, 0.7), (2.6, 2.7)]


@pytest.mark.parametrize("x,y", CASES)
def test_taylor_and_squaring_in_two_coefficients(x, y):
    X = gen(x, y)
    tr = -(x + y)
    assert np.allclose(X @ X, tr * X, rtol=1e-14, atol=1e-300)
    for m in (2, 4, 6, 9, 12, 16, 20, 25, 30):
        b = 0.0
        for k in range(m, 0, -1):
            b = b * tr + 1.0 / math.factorial(k)
        T = sum(np.linalg.matrix_power(X, k) / math.factorial(k) for k in range(m + 1))
        assert np.allclose(T, np.eye(2) + b * X, rtol=1e-14, atol=1e-15)
    p, q = 0.3 * x, 0.3 * y
    W = gen(p, q)
    P = np.eye(2) + W
    assert np.allclose(P @ P - np.eye(2), (2.0 - p - q) * W, rtol=1e-14, atol=1e-16)


@pytest.mark.parametrize("x,y", CASES)
def test_pade_as_one_coefficient(x, y):
    X = gen(x, y)
    tr = -(x + y)
    for m in oracle.PADE_DEGREES:
        c = oracle.pade_coeffs(m)
        Nm = sum(c[j] * np.linalg.matrix_power(X, j) for j in range(m + 1))
        Dm = sum(c[j] * np.linalg.matrix_power(-X, j) for j in range(m + 1))
        R = np.linalg.solve(Dm, Nm)
        bn = sum(c[j] * tr ** (j - 1) for j in range(1, m + 1))
        bd = sum(c[j] * (-1) ** j * tr ** (j - 1) for j in range(1, m + 1))
        assert c[0] + bd * tr >= c[0] > 0.0          # D(tr) = N(-tr), positive coefficients, tr <= 0
        assert np.allclose(R, np.eye(2) + (bn - bd) / (c[0] + bd * tr) * X, rtol=1e-13, atol=1e-15)


@pytest.mark.parametrize("x,y", CASES)
def test_block_norms(x, y):
    X = gen(x, y)
    tr = -(x + y)
    rng = np.random.default_rng(7)
    for _ in range(20):
        c0, beta = rng.normal(), rng.normal() * 3.0
        B = c0 * np.eye(2) + beta * X
        want = max(abs(c0 - beta * x) + abs(beta * y), abs(beta * x) + abs(c0 - beta * y))
        assert np.isclose(np.linalg.norm(B, 1), want, rtol=1e-15, atol=0)
    for q in range(1, 6):
        assert np.isclose(np.linalg.norm(np.linalg.matrix_power(X, q), 1), abs(tr) ** (q - 1) * (x + y),
                          rtol=1e-13, atol=1e-300)
