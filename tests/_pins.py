"""Independent arithmetic used to pin the oracle.

GF(p^k) multiplication here goes through the companion matrix of the
defining polynomial (multiplication by X as a linear map on the basis
1, X, ..., X^{k-1}), a different algorithm from the oracle's schoolbook
product followed by long division.  Pure numpy, small sizes only.
"""
import itertools

import numpy as np


def companion(p, poly):
    """k x k matrix of 'multiply by X' on Z_p[X]/(P), P monic (k+1 coeffs)."""
    k = len(poly) - 1
    C = np.zeros((k, k), dtype=np.int64)
    for i in range(k - 1):
        C[i + 1, i] = 1
    for i in range(k):
        C[i, k - 1] = (-poly[i]) % p
    return C


def mult_matrix(p, poly, a):
    """Matrix of 'multiply by a' = sum_i a_i C^i (mod p)."""
    k = len(poly) - 1
    C = companion(p, poly)
    M = np.zeros((k, k), dtype=np.int64)
    Ci = np.eye(k, dtype=np.int64)
    for i in range(k):
        M = (M + int(a[i]) * Ci) % p
        Ci = (Ci @ C) % p
    return M


def mul(p, poly, a, b):
    return [int(x) for x in (mult_matrix(p, poly, a) @ np.asarray(b, dtype=np.int64)) % p]


def gemm(p, poly, A, B):
    """A: (m, K, k), B: (K, n, k) integer coefficients.  Block-matrix product
    sum_l M(A_il) b_lj over Z_p."""
    A = np.asarray(A, dtype=np.int64) % p
    B = np.asarray(B, dtype=np.int64) % p
    m, K, k = A.shape
    _, n, _ = B.shape
    MA = np.zeros((m * k, K * k), dtype=np.int64)
    for i in range(m):
        for l in range(K):
            MA[i * k:(i + 1) * k, l * k:(l + 1) * k] = mult_matrix(p, poly, A[i, l])
    Bst = np.transpose(B, (0, 2, 1)).reshape(K * k, n)   # rows: (l, coeff)
    C = (MA @ Bst) % p                                     # rows: (i, coeff)
    return np.transpose(C.reshape(m, k, n), (0, 2, 1))


def rank_mod_p(M, p):
    """Rank of an integer matrix over Z_p by Gaussian elimination."""
    M = [[int(x) % p for x in row] for row in M]
    rows, cols = len(M), len(M[0])
    r = 0
    for c in range(cols):
        piv = next((i for i in range(r, rows) if M[i][c]), None)
        if piv is None:
            continue
        M[r], M[piv] = M[piv], M[r]
        inv = pow(M[r][c], p - 2, p)
        M[r] = [(x * inv) % p for x in M[r]]
        for i in range(rows):
            if i != r and M[i][c]:
                f = M[i][c]
                M[i] = [(x - f * y) % p for x, y in zip(M[i], M[r])]
        r += 1
    return r


def is_field(p, poly):
    """Z_p[X]/(P) is a field iff every non-zero element's multiplication
    matrix is invertible (no zero divisors)."""
    k = len(poly) - 1
    for digits in itertools.product(range(p), repeat=k):
        if any(digits) and rank_mod_p(mult_matrix(p, poly, digits), p) < k:
            return False
    return True


def mat_pow(M, e, p):
    k = M.shape[0]
    R = np.eye(k, dtype=np.int64)
    B = M.copy()
    while e:
        if e & 1:
            R = (R @ B) % p
        B = (B @ B) % p
        e >>= 1
    return R


def prime_factors(n):
    f, d = set(), 2
    while d * d <= n:
        while n % d == 0:
            f.add(d)
            n //= d
        d += 1
    if n > 1:
        f.add(n)
    return sorted(f)


def is_primitive(p, poly, a):
    """a generates the multiplicative group iff a^(N/r) != 1 for every prime
    r | N, N = p^k - 1 (Lagrange), evaluated with matrix powers."""
    k = len(poly) - 1
    N = p ** k - 1
    M = mult_matrix(p, poly, a)
    eye = np.eye(k, dtype=np.int64)
    if not np.array_equal(mat_pow(M, N, p), eye):
        return False
    return all(not np.array_equal(mat_pow(M, N // r, p), eye) for r in prime_factors(N))


def value(digits, p):
    return sum(int(c) * p ** i for i, c in enumerate(digits))


def digits(v, p, k):
    return [(v // p ** i) % p for i in range(k)]
