"""Cost model of Sec. 4 (Table 1, eqs. (4.4)-(4.5)) and the storage count of the KP sum,
plus the flop ratio of this implementation's CGLS step (sparse differences, Kronecker
GEMMs), which the direct-versus-KP benchmark reports beside the paper's prediction.

Notation as in the paper: A is M x N with M = m1 m2 and N = n1 n2 (n1 = n for a square n x n
image), R(A) is M-bar x N-bar, k terms, k_p = k + p Krylov or sampled vectors, P rows of each
regularisation block, T = M + 2P rows of the augmented matrix, iota_total CGLS iterations
over the whole split Bregman solve; rho = 1 for EGKB and 2 for RSVD.
"""
from __future__ import annotations

EGKB, RSVD = 1, 2  # the rho of eq. (4.5) / Table 1, column 2


def tsvd_flops(n_bar: int, k_p: int, rho: int = EGKB) -> float:
    """Table 1, column 2: TSVD of R(A), 4 N-bar^2 k_p (EGKB) or 8 N-bar^2 k_p (RSVD)."""
    return 4.0 * rho * n_bar * n_bar * k_p


def cgls_flops_direct(T: int, N: int, iota_total: int) -> float:
    """Table 1, row (i), column 4: all CGLS iterations with the dense augmented matrix."""
    return 4.0 * T * N * iota_total


def cgls_flops_kp(m2: int, N: int, M: int, n1: int, k: int, iota_total: int) -> float:
    """Table 1, rows (ii)-(iii), column 4: all CGLS iterations with the k-term KP sum."""
    return 4.0 * (m2 * N + M * n1) * k * iota_total


def sb_speedup(N: int, P: int, k: int, n1: int) -> float:
    """Eq. (4.4): predicted speed-up of split Bregman with the KP sum over the dense A
    (square A; ratio of the two column-4 entries of Table 1)."""
    return (N + 2.0 * P) / (2.0 * k * n1)


def alg_speedup(N: int, P: int, iota_total: int, k_p: int, rho: int = EGKB) -> float:
    """Eq. (4.5): cost of the CGLS iterations with the dense A over the cost of the TSVD that
    builds the KP sum (Table 1, column 4 over column 2)."""
    return 4.0 * (N + 2.0 * P) * N * iota_total / (4.0 * rho * N * N * k_p)


def kp_storage(k: int, m1: int, n1: int, m2: int, n2: int) -> int:
    """Sec. 4.3: entries of a k-term KP sum, k (m1 n1 + m2 n2) (A itself has m1 m2 n1 n2)."""
    return k * (m1 * n1 + m2 * n2)


def sb_speedup_this_implementation(n: int, k: int) -> float:
    """Flop ratio of one CGLS step here for an n x n image: the dense A costs 4 N^2 (A and
    A^T products, N = n^2; the differences are applied sparsely), the KP sum 8 k n^3 (four
    n x n x n products per term, forward and transpose)."""
    N = n * n
    return 4.0 * N * N / (8.0 * k * n ** 3)
