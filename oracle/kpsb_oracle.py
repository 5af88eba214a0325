"""Plain FP64 CPU oracle for KP-sum approximation + split Bregman TV deblurring.

TEST INFRASTRUCTURE ONLY.  This module is the slow, obviously-correct statement of what
the CUDA path computes.  Only the tests, ``__graft_entry__.smoke()`` and the CPU-baseline
leg of ``bench.py`` may import it.  It shares no code with the CUDA library and imports
nothing from it; the seeded input generators are the only common ground.

Everything follows Alsubhi & Renaut, "Split Bregman isotropic and anisotropic image
deblurring with Kronecker product sum approximations using single precision enlarged-GKB
or RSVD algorithms to provide low rank truncated SVDs" (arXiv 2410.00233).  Section,
algorithm and equation numbers below refer to that paper.  Library primitives used as
steps: numpy matmul / norm / SVD (LAPACK gesdd), numpy QR (LAPACK Householder geqrf),
scipy.sparse products.

Notation: an image X is n x n, x = vec(X) column-major (Sec. 1).  A PSF P is s0 x s1
(rows x columns) with centre (s0 // 2, s1 // 2) (0-based).  m1 = m2 = n1 = n2 = n
(Sec. 5.1), so M = N = n^2 and R(A) is n^2 x n^2.

Readings of points where the paper is silent or ambiguous (each one is listed, with its
reason, in the design notes of the repository):
  * blur = convolution, reflexive boundary = half-sample mirror (x[-1] = x[0]);
  * L = 1/2 forward difference, square n x n with a zero last row (Sec. 5.3);
  * shrinkage threshold = beta / (2 lambda^2), the exact minimiser of the d-subproblem
    (Sec. 3.2, 3.3); ``threshold_rule="paper"`` gives the printed 1/gamma = beta/lambda^2;
  * nu_j = sqrt(zeta_j zeta_{j-1}) for j >= 3 (text of Sec. 2.2), auto-k stops at the first
    i >= max(3, k_min) with nu_{i+1} > nu_i or nu_i < tau * nu_3 (relative tolerance);
  * GKB breakdown (t_j or alpha_j below 100 eps ||B||) ends the recurrence early;
  * RC_CGLS divides by the norm of the updated iterate (x^(0) = 0 in Alg. 5).

Parity status: every function below is pinned by a test in tests/test_oracle_*.py
against an independent fact (explicit matrices, scipy's 2-D convolution, LAPACK SVD of the
full R(A), closed-form singular values, Van Loan-Pitsianis identity, Kronecker identity,
brute-force convex solves, a Chambolle-Pock solve of the TV problem, dense normal
equations, the Krylov-space minimiser of CGLS, Rayleigh-Ritz values of the RSVD range, GKB
coefficients of a hand-built bidiagonal).  tests/oracle_mutations.py plants 86 plausible
mistakes in a copy of this file one at a time; the pins catch every one.  None is marked
"parity unpinned".
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np
import scipy.sparse as sp

BC_ZERO = 0
BC_REFLEXIVE = 1

# --------------------------------------------------------------------------------------
# Blur operator A and its rearrangement R(A)  (Sec. 2.1)
# --------------------------------------------------------------------------------------


def ext(q: int, n: int, bc: int):
    """Boundary extension of a 0-based index q of a length-n signal.

    Zero boundary: indices outside [0, n) carry no value (None).  Reflexive boundary:
    half-sample mirror, -1 -> 0, -2 -> 1, n -> n-1 (one reflection, |overhang| <= n).
    """
    if 0 <= q < n:
        return q
    if bc == BC_ZERO:
        return None
    if q < 0:
        if q < -n:
            raise ValueError("PSF overhang larger than the image")
        return -1 - q
    if q > 2 * n - 1:
        raise ValueError("PSF overhang larger than the image")
    return 2 * n - 1 - q


def vec(X: np.ndarray) -> np.ndarray:
    """Column-major vectorisation (Sec. 1)."""
    return np.asarray(X).reshape(-1, order="F")


def array(x: np.ndarray, m: int, n: int) -> np.ndarray:
    """Inverse of vec (Sec. 1, Theorem 2.1's array(u, m, n))."""
    return np.asarray(x).reshape(m, n, order="F")


def blur_matrix(psf: np.ndarray, n: int, bc: int) -> np.ndarray:
    """Explicit N x N blur matrix A (N = n^2) of a spatially invariant PSF (Sec. 1, 5.2).

    (A vec(X))(r, c') = sum_{a,b} P[a, b] X[ext(r - a + c), ext(c' - b + c)].
    """
    s0, s1 = psf.shape
    ca, cb = s0 // 2, s1 // 2
    N = n * n
    A = np.zeros((N, N))
    for cc in range(n):
        for r in range(n):
            row = r + cc * n
            for a in range(s0):
                i = ext(r - a + ca, n, bc)
                if i is None:
                    continue
                for b in range(s1):
                    j = ext(cc - b + cb, n, bc)
                    if j is None:
                        continue
                    A[row, i + j * n] += psf[a, b]
    return A


def blur(psf: np.ndarray, X: np.ndarray, bc: int) -> np.ndarray:
    """A vec(X) as an image, by the same sum over PSF taps (vectorised over pixels)."""
    n = X.shape[0]
    s0, s1 = psf.shape
    ca, cb = s0 // 2, s1 // 2
    idx = np.arange(n)
    out = np.zeros((n, n))
    for a in range(s0):
        rows = [ext(r - a + ca, n, bc) for r in idx]
        rmask = np.array([q is not None for q in rows])
        rsrc = np.array([q if q is not None else 0 for q in rows])
        for b in range(s1):
            cols = [ext(c - b + cb, n, bc) for c in idx]
            cmask = np.array([q is not None for q in cols])
            csrc = np.array([q if q is not None else 0 for q in cols])
            tap = X[np.ix_(rsrc, csrc)] * np.outer(rmask, cmask)
            out += psf[a, b] * tap
    return out


def rearrange(A: np.ndarray, m1: int, n1: int, m2: int, n2: int) -> np.ndarray:
    """R(A) of eq. (2.2): block A_{i,j} (m2 x n2) becomes row i + j*m1 (0-based), holding
    vec(A_{i,j})^T."""
    R = np.empty((m1 * n1, m2 * n2))
    for j in range(n1):
        for i in range(m1):
            blk = A[i * m2:(i + 1) * m2, j * n2:(j + 1) * n2]
            R[i + j * m1, :] = vec(blk)
    return R


def shift_matrix(t: int, n: int, c: int, bc: int) -> np.ndarray:
    """M_t with (M_t x)_r = x_{ext(r - t + c)}: the 1-D action of PSF tap t."""
    M = np.zeros((n, n))
    for r in range(n):
        q = ext(r - t + c, n, bc)
        if q is not None:
            M[r, q] += 1.0
    return M


@dataclass
class RFactors:
    """R(A) = Kx P^T Ky^T, with Kx[:, b] = vec(M_b) (columns, x-direction) and
    Ky[:, a] = vec(M_a) (rows, y-direction).

    Derivation: A = sum_{a,b} P[a,b] (M_b (x) M_a) because
    (M_b (x) M_a) vec(X) = vec(M_a X M_b^T), and R(B (x) C) = vec(B) vec(C)^T
    (Theorem 2.1 applied term by term).
    """

    Kx: sp.csc_matrix
    Ky: sp.csc_matrix
    P: np.ndarray
    n: int


def r_factors(psf: np.ndarray, n: int, bc: int) -> RFactors:
    s0, s1 = psf.shape

    def kmat(s, c):
        rows, cols, vals = [], [], []
        for t in range(s):
            M = shift_matrix(t, n, c, bc)
            nz = np.nonzero(vec(M))[0]
            rows.extend(nz.tolist())
            cols.extend([t] * len(nz))
            vals.extend(vec(M)[nz].tolist())
        return sp.csc_matrix((vals, (rows, cols)), shape=(n * n, s))

    return RFactors(Kx=kmat(s1, s1 // 2), Ky=kmat(s0, s0 // 2), P=np.array(psf, dtype=np.float64), n=n)


def r_apply(F: RFactors, V: np.ndarray) -> np.ndarray:
    """R(A) V = Kx (P^T (Ky^T V)) for a vector or a block of columns."""
    return F.Kx @ (F.P.T @ (F.Ky.T @ V))


def r_apply_t(F: RFactors, U: np.ndarray) -> np.ndarray:
    """R(A)^T U = Ky (P (Kx^T U))."""
    return F.Ky @ (F.P @ (F.Kx.T @ U))


def r_index_maps(psf_shape, n: int, bc: int):
    """Integer structure of R(A): for each row (i, j) of R(A) (row index i + j*n) the PSF
    columns b with M_b[i, j] != 0 (with multiplicity), and for each column (r, r') of R(A)
    the PSF rows a with M_a[r, r'] != 0.  R(A)[(i,j), (r,r')] = sum over those (a, b) of
    P[a, b].  Returned as two lists of sorted tuples, derived from the shift matrices."""
    s0, s1 = psf_shape
    Mx = [shift_matrix(b, n, s1 // 2, bc) for b in range(s1)]
    My = [shift_matrix(a, n, s0 // 2, bc) for a in range(s0)]
    row_map = []
    for j in range(n):
        for i in range(n):
            lst = []
            for b in range(s1):
                lst.extend([b] * int(round(Mx[b][i, j])))
            row_map.append(tuple(lst))
    col_map = []
    for rp in range(n):
        for r in range(n):
            lst = []
            for a in range(s0):
                lst.extend([a] * int(round(My[a][r, rp])))
            col_map.append(tuple(lst))
    return row_map, col_map


def r_sigma_closed_form(F: RFactors) -> np.ndarray:
    """All singular values of R(A) = Kx P^T Ky^T from s x s matrices only.

    With Gx = Kx^T Kx and Gy = Ky^T Ky, sigma(R(A)) = sigma(Gx^{1/2} P^T Gy^{1/2}), since
    Kx = Wx Gx^{1/2} and Ky = Wy Gy^{1/2} with Wx, Wy having orthonormal columns on the
    ranges of Kx, Ky (polar decomposition).  Valid at any n; the rest are zero.
    """

    def psd_sqrt(G):
        w, Q = np.linalg.eigh(G)
        w = np.clip(w, 0.0, None)
        return (Q * np.sqrt(w)) @ Q.T

    Gx = (F.Kx.T @ F.Kx).toarray()
    Gy = (F.Ky.T @ F.Ky).toarray()
    return np.linalg.svd(psd_sqrt(Gx) @ F.P.T @ psd_sqrt(Gy), compute_uv=False)


def r_tsvd_closed_form(F: RFactors, k: int):
    """Leading k singular triplets of R(A) from the s x s problem (requires Gx, Gy
    invertible): u_i = Kx Gx^{-1/2} a_i, v_i = Ky Gy^{-1/2} b_i where
    Gx^{1/2} P^T Gy^{1/2} = sum sigma_i a_i b_i^T."""

    def psd_pow(G, e):
        w, Q = np.linalg.eigh(G)
        return (Q * w**e) @ Q.T

    Gx = (F.Kx.T @ F.Kx).toarray()
    Gy = (F.Ky.T @ F.Ky).toarray()
    a, sig, bt = np.linalg.svd(psd_pow(Gx, 0.5) @ F.P.T @ psd_pow(Gy, 0.5))
    U = F.Kx @ (psd_pow(Gx, -0.5) @ a[:, :k])
    V = F.Ky @ (psd_pow(Gy, -0.5) @ bt[:k, :].T)
    return U, sig[:k], V


# --------------------------------------------------------------------------------------
# EGKB (Alg. 1) and RSVD (Alg. 2)
# --------------------------------------------------------------------------------------


@dataclass
class TSVD:
    U: np.ndarray  # Mbar x k, left singular vectors (x-direction factors)
    sigma: np.ndarray  # k
    V: np.ndarray  # Nbar x k, right singular vectors (y-direction factors)
    k: int
    kp: int
    info: dict = field(default_factory=dict)


def _mgs(v: np.ndarray, basis: list) -> np.ndarray:
    """Modified Gram-Schmidt of v against the orthonormal columns in ``basis`` (Alg. 1
    step 6, Sec. 5.1)."""
    for b in basis:
        v = v - np.dot(v, b) * b
    return v


def egkb(B, BT, y: np.ndarray, k: int, p: int, tau: float = 0.0, k_min: int = 3,
         full_reorth: bool = True, eps: float = np.finfo(np.float64).eps) -> TSVD:
    """Enlarged Golub-Kahan bidiagonalisation, Alg. 1 (Sec. 2.2).

    B, BT: callables v -> B v and u -> B^T u.  y: start vector (length Mbar).
    Fixed-rank mode (tau == 0): k terms from k_p = k + p steps.  Automatic mode (tau > 0):
    k is chosen by the nu_j rule (2.6) with relative tolerance tau * nu_3, capped at the
    given k, and the recurrence continues to k_p = k + p steps.  full_reorth also
    reorthogonalises the s_j (the single-precision variant of Sec. 4.4); the q_j are always
    reorthogonalised (one-sided, step 6).
    """
    auto = tau > 0.0
    k_cap = k
    kp = None if auto else k + p
    S, Q, alpha, t = [], [], [], []
    t1 = np.linalg.norm(y)
    S.append(y / t1)
    q = BT(S[0])
    a1 = np.linalg.norm(q)
    Q.append(q / a1)
    alpha.append(a1)
    t.append(t1)  # t_1 is not part of C
    zeta = {}
    nu = {}
    bnorm = a1
    k_sel = None if auto else k
    breakdown = None
    j = 2
    while True:
        # step 3-4: s_j = B q_{j-1} - alpha_{j-1} s_{j-1}; t_j = ||s_j||
        s = B(Q[-1]) - alpha[-1] * S[-1]
        if full_reorth:
            s = _mgs(s, S)
        tj = np.linalg.norm(s)
        bnorm = max(bnorm, tj)
        if tj <= 100.0 * eps * bnorm:
            breakdown = ("t", j)
            t.append(0.0)
            S.append(np.zeros_like(S[0]))
            break
        S.append(s / tj)
        t.append(tj)
        if kp is not None and len(Q) == kp:
            break  # s_{kp+1}, t_{kp+1} complete C
        # step 5-7: q_j = B^T s_j - t_j q_{j-1}; reorthogonalise; alpha_j = ||q_j||
        q = BT(S[-1]) - tj * Q[-1]
        q = _mgs(q, Q)
        aj = np.linalg.norm(q)
        bnorm = max(bnorm, aj)
        if aj <= 100.0 * eps * bnorm:
            breakdown = ("alpha", j)
            break
        Q.append(q / aj)
        alpha.append(aj)
        # step 8: zeta_j = alpha_j t_j, nu_j = sqrt(zeta_j zeta_{j-1}) for j >= 3
        zeta[j] = aj * tj
        if j >= 3:
            nu[j] = math.sqrt(zeta[j] * zeta[j - 1])
        # step 9: automatic choice of k, tested for index i = j - 1 once nu_{i+1} is known
        if auto and k_sel is None and j >= 4:
            i = j - 1
            if i >= max(3, k_min) and (nu[j] > nu[i] or nu[i] < tau * nu[3]):
                k_sel = i
            elif i >= k_cap:
                k_sel = k_cap
            if k_sel is not None:
                kp = k_sel + p
                if len(Q) >= kp:
                    kp = len(Q)
        j += 1
    kp_eff = len(Q)
    if k_sel is None:  # breakdown before the rule fired
        k_sel = min(k_cap, kp_eff)
    k_eff = min(k_sel, kp_eff)
    # Lower bidiagonal C ((kp+1) x kp): diag alpha_1..alpha_kp, subdiag t_2..t_{kp+1}
    C = np.zeros((kp_eff + 1, kp_eff))
    for i in range(kp_eff):
        C[i, i] = alpha[i]
        C[i + 1, i] = t[i + 1]
    Smat = np.stack(S[:kp_eff + 1], axis=1)
    Qmat = np.stack(Q[:kp_eff], axis=1)
    Uc, sc, Vct = np.linalg.svd(C, full_matrices=False)  # step 15
    U = Smat @ Uc[:, :k_eff]  # steps 16-17
    V = Qmat @ Vct[:k_eff, :].T
    return TSVD(U=U, sigma=sc[:k_eff], V=V, k=k_eff, kp=kp_eff,
                info=dict(C=C, S=Smat, Q=Qmat, alpha=np.array(alpha[:kp_eff]),
                          t=np.array(t[:kp_eff + 1]), nu=nu, zeta=zeta,
                          breakdown=breakdown, sigma_all=sc))


def rsvd(B, BT, F: np.ndarray, k: int, q: int = 1) -> TSVD:
    """Randomised SVD, Alg. 2 (Sec. 2.3), with an orthonormalisation (Householder QR)
    after every application of B or B^T (step 2), then H = Q^T B (step 4), the SVD of H
    (step 5), U = Q U_H (step 6) and truncation to k terms (step 7)."""
    kp = F.shape[1]
    Qb, _ = np.linalg.qr(B(F))
    for _ in range(q):
        Z, _ = np.linalg.qr(BT(Qb))
        Qb, _ = np.linalg.qr(B(Z))
    H = BT(Qb).T  # kp x Nbar
    Uh, sh, Vht = np.linalg.svd(H, full_matrices=False)
    U = Qb @ Uh[:, :k]
    return TSVD(U=U, sigma=sh[:k], V=Vht[:k, :].T, k=k, kp=kp, info=dict(sigma_all=sh, Q=Qb))


# --------------------------------------------------------------------------------------
# Kronecker-product-sum operator (Theorem 2.1, Sec. 4.1.3, Sec. 4.2)
# --------------------------------------------------------------------------------------


@dataclass
class KPSum:
    """A ~ sum_i sigma_i Ax_i (x) Ay_i with unit-Frobenius Ax_i = array(u_i, n, n) and
    Ay_i = array(v_i, n, n) (Theorem 2.1; the paper folds sigma_i into Ax_i)."""

    Ax: np.ndarray  # k x n x n
    Ay: np.ndarray  # k x n x n
    sigma: np.ndarray  # k

    @property
    def k(self):
        return len(self.sigma)

    @property
    def n(self):
        return self.Ax.shape[1]


def kp_terms(ts: TSVD, n: int, sign_fix: bool = True) -> KPSum:
    """Terms(A_k): Ax_i = array(u_i, n, n), Ay_i = array(v_i, n, n), sigma_i kept apart.

    Sign convention (the SVD fixes each pair only up to a common sign): the entry of
    largest magnitude of Ay_i is made positive, flipping u_i with it."""
    k = ts.k
    Ax = np.empty((k, n, n))
    Ay = np.empty((k, n, n))
    for i in range(k):
        u = ts.U[:, i].copy()
        v = ts.V[:, i].copy()
        if sign_fix and v[np.argmax(np.abs(v))] < 0:
            u, v = -u, -v
        Ax[i] = array(u, n, n)
        Ay[i] = array(v, n, n)
    return KPSum(Ax=Ax, Ay=Ay, sigma=np.array(ts.sigma[:k], dtype=np.float64))


def kp_apply(K: KPSum, X: np.ndarray) -> np.ndarray:
    """array(A_k x) = sum_i sigma_i Ay_i X Ax_i^T (Sec. 4.2)."""
    Y = np.zeros_like(X, dtype=np.float64)
    for i in range(K.k):
        Y += K.sigma[i] * (K.Ay[i] @ X @ K.Ax[i].T)
    return Y


def kp_apply_t(K: KPSum, Y: np.ndarray) -> np.ndarray:
    """array(A_k^T y) = sum_i sigma_i Ay_i^T Y Ax_i."""
    X = np.zeros_like(Y, dtype=np.float64)
    for i in range(K.k):
        X += K.sigma[i] * (K.Ay[i].T @ Y @ K.Ax[i])
    return X


def kp_matrix(K: KPSum) -> np.ndarray:
    """Explicit sum_i sigma_i Ax_i (x) Ay_i (small n only)."""
    return sum(K.sigma[i] * np.kron(K.Ax[i], K.Ay[i]) for i in range(K.k))


# --------------------------------------------------------------------------------------
# Regularisation operator, shrinkage, CGLS, split Bregman (Sec. 3, Sec. 5.3)
# --------------------------------------------------------------------------------------


def L_matrix(n: int) -> np.ndarray:
    """L = 1/2 [1 -1 ...] (Sec. 5.3), square n x n, last row zero."""
    L = np.zeros((n, n))
    for i in range(n - 1):
        L[i, i] = 0.5
        L[i, i + 1] = -0.5
    return L


def Dx(X):
    """(L_x (x) I) vec(X) = vec(X L^T): horizontal difference."""
    return X @ L_matrix(X.shape[1]).T


def Dy(X):
    """(I (x) L_y) vec(X) = vec(L X): vertical difference."""
    return L_matrix(X.shape[0]) @ X


def Dx_t(Y):
    return Y @ L_matrix(Y.shape[1])


def Dy_t(Y):
    return L_matrix(Y.shape[0]).T @ Y


def shrink(w, v):
    """shrink(w, v) = sign(w) max(|w| - v, 0) (Sec. 3.2)."""
    return np.sign(w) * np.maximum(np.abs(w) - v, 0.0)


def shrink_iso(cx, cy, v):
    """Isotropic shrinkage (Sec. 3.3): d = (c / s) max(s - v, 0), s = sqrt(cx^2 + cy^2),
    and d = 0 where s = 0."""
    s = np.sqrt(cx * cx + cy * cy)
    scale = np.where(s > 0, np.maximum(s - v, 0.0) / np.where(s > 0, s, 1.0), 0.0)
    return cx * scale, cy * scale


@dataclass
class CGLSResult:
    x: np.ndarray
    iters: int
    rc: float


def cgls(Ahat, AhatT, bhat, x_shape, i_max: int = 100, tau: float = 1e-4,
         fixed: bool = False) -> CGLSResult:
    """CGLS, Alg. 5 (Sec. 3.4): min ||Ahat x - bhat||, x^(0) = 0.

    Ahat maps an image to a tuple of blocks, AhatT maps such a tuple back.  Stops when
    RC_CGLS = ||mu w|| / ||x|| < tau (5.1) unless ``fixed`` (then exactly i_max steps)."""

    def dot(a, b):
        return sum(float(np.sum(ai * bi)) for ai, bi in zip(a, b))

    x = np.zeros(x_shape)
    r = tuple(np.array(bi, dtype=np.float64) for bi in bhat)
    f = AhatT(r)
    w = f.copy()
    tau_k = float(np.sum(f * f))
    it = 0
    rc = math.inf
    while it < i_max:
        if tau_k == 0.0:
            break
        z = Ahat(w)  # step 3
        zz = dot(z, z)
        if zz == 0.0:
            break
        mu = tau_k / zz  # step 4
        x = x + mu * w  # step 5
        xn = np.linalg.norm(x)
        rc = mu * np.linalg.norm(w) / xn if xn > 0 else math.inf
        r = tuple(ri - mu * zi for ri, zi in zip(r, z))  # step 6
        f = AhatT(r)  # step 7
        tau_new = float(np.sum(f * f))  # step 8
        delta = tau_new / tau_k  # step 9
        w = f + delta * w  # step 10
        tau_k = tau_new
        it += 1
        if not fixed and rc < tau:
            break
    return CGLSResult(x=x, iters=it, rc=rc)


@dataclass
class SBResult:
    x: np.ndarray
    l_end: int
    iota_total: int
    rc_sb: float
    history: list = field(default_factory=list)


def sb_threshold(lam: float, beta: float, rule: str = "exact") -> float:
    """Shrinkage threshold of the d-subproblem argmin lambda^2||d - c||^2 + beta||d||_1.
    exact: beta / (2 lambda^2); paper: the printed 1/gamma = beta / lambda^2."""
    if rule == "exact":
        return beta / (2.0 * lam * lam)
    if rule == "paper":
        return beta / (lam * lam)
    raise ValueError(rule)


def split_bregman(A, AT, b: np.ndarray, mu: float, lam: float, beta: float, iso: bool,
                  iters: int, tau_sb: float = 0.0, tau_cgls: float = 1e-4, i_max: int = 100,
                  fixed_inner: bool = False, threshold_rule: str = "exact",
                  x_true: np.ndarray | None = None) -> SBResult:
    """Split Bregman TV deblurring, Alg. 3 (anisotropic) / Alg. 4 (isotropic).

    Objective: mu ||A x - b||^2 + beta TV(x) with the splitting penalty
    lambda^2 ||D x - d + g||^2 (Sec. 3.2-3.3, lambda_x = lambda_y, beta_x = beta_y).
    A, AT: callables on n x n images (A_k or the explicit blur).  Each outer step solves
    the x-subproblem (3.7) by CGLS (Alg. 5) on Ahat = [sqrt(mu) A; lambda Dx; lambda Dy],
    bhat = [sqrt(mu) b; lambda (dx - gx); lambda (dy - gy)] from x = 0, then the
    shrinkage (3.10) / (3.13) and the Bregman updates (3.8)-(3.9)."""
    sm = math.sqrt(mu)
    thr = sb_threshold(lam, beta, threshold_rule)

    def Ahat(X):
        return (sm * A(X), lam * Dx(X), lam * Dy(X))

    def AhatT(r):
        return sm * AT(r[0]) + lam * Dx_t(r[1]) + lam * Dy_t(r[2])

    x = np.array(b, dtype=np.float64)  # Alg. 3/4: x^(0) = b
    dx = np.zeros_like(x)
    dy = np.zeros_like(x)
    gx = np.zeros_like(x)
    gy = np.zeros_like(x)
    iota_total = 0
    rc_sb = math.inf
    hist = []
    ell = 0
    while ell < iters:
        bhat = (sm * b, lam * (dx - gx), lam * (dy - gy))
        res = cgls(Ahat, AhatT, bhat, x.shape, i_max=i_max, tau=tau_cgls, fixed=fixed_inner)
        iota_total += res.iters
        x_new = res.x
        cx = Dx(x_new) + gx
        cy = Dy(x_new) + gy
        if iso:
            dx, dy = shrink_iso(cx, cy, thr)
        else:
            dx, dy = shrink(cx, thr), shrink(cy, thr)
        gx = cx - dx
        gy = cy - dy
        nx = np.linalg.norm(x)
        rc_sb = np.linalg.norm(x_new - x) / nx if nx > 0 else math.inf
        x = x_new
        ell += 1
        rec = dict(ell=ell, iters=res.iters, rc_sb=rc_sb)
        if x_true is not None:
            rec["re"] = rel_error(x, x_true)
        hist.append(rec)
        if rc_sb < tau_sb:
            break
    return SBResult(x=x, l_end=ell, iota_total=iota_total, rc_sb=rc_sb, history=hist)


# --------------------------------------------------------------------------------------
# Metrics (Sec. 5.3.2) and convenience pipeline
# --------------------------------------------------------------------------------------


def rel_error(x, x_true):
    """RE (5.5)."""
    return float(np.linalg.norm(x - x_true) / np.linalg.norm(x_true))


def isnr(x, b, x_true):
    """ISNR (5.6) in dB."""
    return float(20.0 * math.log10(np.linalg.norm(b - x_true) / np.linalg.norm(x - x_true)))


def snr(b_true, b):
    """SNR (5.4) in dB."""
    return float(10.0 * math.log10(np.sum(b_true**2) / np.sum((b_true - b) ** 2)))


def kp_build(psf: np.ndarray, n: int, bc: int, k: int, p: int, method: str = "egkb",
             tau: float = 0.0, start: np.ndarray | None = None, F: np.ndarray | None = None,
             full_reorth: bool = True, q: int = 1) -> tuple[KPSum, TSVD]:
    """TSVD of R(A) (EGKB or RSVD) followed by Terms(A_k)."""
    Rf = r_factors(psf, n, bc)
    B = lambda v: r_apply(Rf, v)  # noqa: E731
    BT = lambda u: r_apply_t(Rf, u)  # noqa: E731
    if method == "egkb":
        ts = egkb(B, BT, np.asarray(start, dtype=np.float64), k, p, tau=tau, full_reorth=full_reorth)
    elif method == "rsvd":
        ts = rsvd(B, BT, np.asarray(F, dtype=np.float64), k, q=q)
    else:
        raise ValueError(method)
    return kp_terms(ts, n), ts
