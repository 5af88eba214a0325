"""Planted-mistake check of the oracle's pins (CPU only; not collected by pytest).

Each entry below is one plausible mistake in ``oracle/kpsb_oracle.py`` -- a dropped term, a
flipped sign, a wrong index or a transposed operand -- together with the part of the paper
it would break.  For every entry the oracle is copied to a temporary directory, the
mistake is written into the copy, and the oracle's pins (``tests/test_oracle_*.py``) are
run against the copy.  A pin suite that lets a mistake through has a gap; the run exits
with status 1 and names it.  The committed oracle file is never modified.

    python tests/oracle_mutations.py            # every entry, 4 at a time
    python tests/oracle_mutations.py -j 8 -k cgls   # entries whose name contains "cgls"

Mistakes that change nothing (equivalent mutants, e.g. ``+=`` into a shift matrix that has
one entry per row) are not listed.
"""
import argparse
import os
import shutil
import subprocess
import sys
import tempfile
from concurrent.futures import ThreadPoolExecutor

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
ORACLE = os.path.join(ROOT, "oracle", "kpsb_oracle.py")
PINS = ["test_oracle_golden.py", "test_oracle_operator.py", "test_oracle_sb.py",
        "test_oracle_tsvd.py", "test_oracle_properties.py"]

# (name, what it breaks, text in the oracle, replacement)
MUTATIONS = [
    # boundary extension and the blur (Sec. 1, Sec. 5.2)
    ("ext-reflect-low", "half-sample mirror", "        return -1 - q", "        return -q"),
    ("ext-reflect-high", "half-sample mirror", "    return 2 * n - 1 - q", "    return 2 * n - 2 - q"),
    ("ext-overhang", "one reflection per side", "if q < -n:", "if q < -n - 1:"),
    ("blur-matrix-row-flip", "convolution, not correlation", "i = ext(r - a + ca, n, bc)",
     "i = ext(r + a - ca, n, bc)"),
    ("blur-row-flip", "convolution, not correlation", "rows = [ext(r - a + ca, n, bc)",
     "rows = [ext(r + a - ca, n, bc)"),
    ("blur-col-flip", "convolution, not correlation", "cols = [ext(c - b + cb, n, bc)",
     "cols = [ext(c + b - cb, n, bc)"),
    ("blur-matrix-overwrite", "reflected taps add up", "A[row, i + j * n] += psf[a, b]",
     "A[row, i + j * n] = psf[a, b]"),
    # R(A) and its factors (eq. (2.2), Theorem 2.1)
    ("rearrange-index", "row i + j m1 of R(A)", "R[i + j * m1, :] = vec(blk)",
     "R[j + i * n1, :] = vec(blk)"),
    ("shift-flip", "tap t of M_t", "q = ext(r - t + c, n, bc)", "q = ext(r + t - c, n, bc)"),
    ("factors-swapped", "x factor from PSF columns, y from rows",
     "Kx=kmat(s1, s1 // 2), Ky=kmat(s0, s0 // 2)", "Kx=kmat(s0, s0 // 2), Ky=kmat(s1, s1 // 2)"),
    ("r-apply-P", "R(A) = Kx P^T Ky^T", "return F.Kx @ (F.P.T @ (F.Ky.T @ V))",
     "return F.Kx @ (F.P @ (F.Ky.T @ V))"),
    ("r-apply-t-P", "R(A)^T = Ky P Kx^T", "return F.Ky @ (F.P @ (F.Kx.T @ U))",
     "return F.Ky @ (F.P.T @ (F.Kx.T @ U))"),
    ("index-map-transposed", "row map of R(A)", "lst.extend([b] * int(round(Mx[b][i, j])))",
     "lst.extend([b] * int(round(Mx[b][j, i])))"),
    ("closed-form-sqrt", "sigma(Gx^1/2 P^T Gy^1/2)", "psd_sqrt(Gx) @ F.P.T @ psd_sqrt(Gy)",
     "psd_sqrt(Gx) @ F.P.T @ Gy"),
    ("closed-form-V-transposed", "right vectors of the s x s SVD",
     "V = F.Ky @ (psd_pow(Gy, -0.5) @ bt[:k, :].T)", "V = F.Ky @ (psd_pow(Gy, -0.5) @ bt[:, :k])"),
    # EGKB (Alg. 1, Sec. 2.2)
    ("egkb-s-sign", "s_j = B q_{j-1} - alpha_{j-1} s_{j-1}", "s = B(Q[-1]) - alpha[-1] * S[-1]",
     "s = B(Q[-1]) + alpha[-1] * S[-1]"),
    ("egkb-q-term-dropped", "q_j = B^T s_j - t_j q_{j-1}", "q = BT(S[-1]) - tj * Q[-1]",
     "q = BT(S[-1])"),
    ("egkb-no-q-reorth", "reorthogonalised q_j", "        q = _mgs(q, Q)", "        q = q"),
    ("egkb-no-s-reorth", "reorthogonalised s_j (single precision variant)",
     "        if full_reorth:\n            s = _mgs(s, S)", "        if False:\n            s = _mgs(s, S)"),
    ("mgs-half", "Gram-Schmidt projection", "v = v - np.dot(v, b) * b",
     "v = v - 0.5 * np.dot(v, b) * b"),
    ("nu-not-geometric-mean", "nu_j = sqrt(zeta_j zeta_{j-1})",
     "nu[j] = math.sqrt(zeta[j] * zeta[j - 1])", "nu[j] = zeta[j]"),
    ("nu-rule-direction", "stop when nu rises", "nu[j] > nu[i] or", "nu[j] < nu[i] or"),
    ("nu-rule-reference", "tolerance relative to nu_3", "nu[i] < tau * nu[3]",
     "nu[i] < tau * nu[4]"),
    ("egkb-kp-stop", "k_p = k + p steps", "if kp is not None and len(Q) == kp:",
     "if kp is not None and len(Q) == kp - 1:"),
    ("bidiag-subdiag", "C holds t_2..t_{kp+1} below the diagonal", "C[i + 1, i] = t[i + 1]",
     "C[i + 1, i] = t[i]"),
    ("egkb-U-last-row", "U = S_{kp+1} U_C", "U = Smat @ Uc[:, :k_eff]",
     "U = Smat[:, :kp_eff] @ Uc[:kp_eff, :k_eff]"),
    ("egkb-V-transposed", "V = Q_kp V_C", "V = Qmat @ Vct[:k_eff, :].T", "V = Qmat @ Vct[:, :k_eff]"),
    # RSVD (Alg. 2, Sec. 2.3)
    ("rsvd-no-power-step", "q power steps", "    for _ in range(q):\n        Z, _",
     "    for _ in range(0):\n        Z, _"),
    ("rsvd-U-transposed", "U = Q U_H", "U = Qb @ Uh[:, :k]", "U = Qb @ Uh[:k, :].T"),
    # Terms(A_k) and the KP apply (Theorem 2.1, Sec. 4.2)
    ("terms-sign-rule", "largest entry of Ay_i positive",
     "if sign_fix and v[np.argmax(np.abs(v))] < 0:", "if sign_fix and v[np.argmax(np.abs(v))] > 0:"),
    ("terms-flip-one-side", "a pair flips together", "            u, v = -u, -v",
     "            u, v = u, -v"),
    ("terms-swapped", "Ax from u, Ay from v", "Ax[i] = array(u, n, n)\n        Ay[i] = array(v, n, n)",
     "Ax[i] = array(v, n, n)\n        Ay[i] = array(u, n, n)"),
    ("apply-swapped", "array(A_k x) = sum sigma Ay X Ax^T",
     "Y += K.sigma[i] * (K.Ay[i] @ X @ K.Ax[i].T)", "Y += K.sigma[i] * (K.Ax[i] @ X @ K.Ay[i].T)"),
    ("apply-t-not-adjoint", "array(A_k^T y) = sum sigma Ay^T Y Ax",
     "X += K.sigma[i] * (K.Ay[i].T @ Y @ K.Ax[i])", "X += K.sigma[i] * (K.Ay[i] @ Y @ K.Ax[i].T)"),
    ("kron-order", "Ax (x) Ay", "np.kron(K.Ax[i], K.Ay[i])", "np.kron(K.Ay[i], K.Ax[i])"),
    # regularisation operator and shrinkage (Sec. 3.2, 3.3, 5.3)
    ("L-sign", "L = 1/2 [1 -1]", "L[i, i + 1] = -0.5", "L[i, i + 1] = 0.5"),
    ("L-scale", "L = 1/2 [1 -1]", "L[i, i] = 0.5", "L[i, i] = 1.0"),
    ("Dx-as-Dy", "Dx = L (x) I", "return X @ L_matrix(X.shape[1]).T", "return L_matrix(X.shape[0]) @ X"),
    ("Dy-transposed", "Dy = I (x) L", "return L_matrix(X.shape[0]) @ X", "return L_matrix(X.shape[0]).T @ X"),
    ("Dx-t-not-adjoint", "Dx^T", "return Y @ L_matrix(Y.shape[1])", "return Y @ L_matrix(Y.shape[1]).T"),
    ("Dy-t-not-adjoint", "Dy^T", "return L_matrix(Y.shape[0]).T @ Y", "return L_matrix(Y.shape[0]) @ Y"),
    ("shrink-threshold", "shrink(w, v)", "np.maximum(np.abs(w) - v, 0.0)",
     "np.maximum(np.abs(w) - 2 * v, 0.0)"),
    ("shrink-iso-threshold", "isotropic shrink", "np.maximum(s - v, 0.0)", "np.maximum(s - 2 * v, 0.0)"),
    ("shrink-iso-l1", "isotropic magnitude", "s = np.sqrt(cx * cx + cy * cy)",
     "s = np.abs(cx) + np.abs(cy)"),
    ("threshold-exact", "argmin of the d-subproblem", "return beta / (2.0 * lam * lam)",
     "return beta / (lam * lam)"),
    # CGLS (Alg. 5, eq. (5.1))
    ("cgls-delta", "delta = tau_new / tau", "delta = tau_new / tau_k", "delta = tau_k / tau_new"),
    ("cgls-direction", "w = f + delta w", "w = f + delta * w", "w = f + delta * f"),
    ("cgls-x-step", "x = x + mu w", "x = x + mu * w  # step 5", "x = x + mu * f  # step 5"),
    ("cgls-residual-sign", "r = r - mu z", "r = tuple(ri - mu * zi", "r = tuple(ri + mu * zi"),
    ("cgls-rc", "RC_CGLS = ||mu w|| / ||x||", "rc = mu * np.linalg.norm(w) / xn",
     "rc = np.linalg.norm(w) / xn"),
    # split Bregman (Alg. 3, 4; eq. (5.2))
    ("sb-x0", "x^(0) = b", "x = np.array(b, dtype=np.float64)  # Alg. 3/4",
     "x = np.zeros_like(b, dtype=np.float64)  # Alg. 3/4"),
    ("sb-data-sqrt-mu", "bhat = [sqrt(mu) b; ...]", "bhat = (sm * b, lam * (dx - gx)",
     "bhat = (b, lam * (dx - gx)"),
    ("sb-bhat-lambda", "bhat = [...; lambda (d - g)]", "bhat = (sm * b, lam * (dx - gx)",
     "bhat = (sm * b, (dx - gx)"),
    ("sb-bhat-dy", "y block uses d_y - g_y", "lam * (dy - gy))\n        res",
     "lam * (dx - gy))\n        res"),
    ("sb-Ahat-lambda", "Ahat = [sqrt(mu) A; lambda Dx; lambda Dy]",
     "return (sm * A(X), lam * Dx(X), lam * Dy(X))", "return (sm * A(X), Dx(X), lam * Dy(X))"),
    ("sb-c-sign", "c = D x + g", "cx = Dx(x_new) + gx", "cx = Dx(x_new) - gx"),
    ("sb-bregman-sign", "g = c - d", "gx = cx - dx", "gx = dx - cx"),
    ("sb-bregman-gy", "g_y = c_y - d_y", "gy = cy - dy", "gy = cy - dx"),
    ("sb-aniso-dy", "d_y = shrink(c_y)", "dx, dy = shrink(cx, thr), shrink(cy, thr)",
     "dx, dy = shrink(cx, thr), shrink(cx, thr)"),
    ("sb-iso-cy", "isotropic shrink of (c_x, c_y)", "dx, dy = shrink_iso(cx, cy, thr)",
     "dx, dy = shrink_iso(cx, cx, thr)"),
    ("sb-rc-denominator", "RC_SB over ||x^(l-1)||", "rc_sb = np.linalg.norm(x_new - x) / nx",
     "rc_sb = np.linalg.norm(x_new - x) / np.linalg.norm(x_new)"),
    ("sb-stop", "stop when RC_SB < tau_SB", "if rc_sb < tau_sb:", "if rc_sb <= tau_sb * 10:"),
    # more of the same families: centres, boundary rows, caps and thresholds, counters
    ("ext-zero-outside", "zero boundary reads nothing outside", "    if bc == BC_ZERO:\n        return None",
     "    if bc == BC_ZERO:\n        return 0"),
    ("blur-centre", "centre tap at s // 2", "    s0, s1 = psf.shape\n    ca, cb = s0 // 2, s1 // 2\n    N = n * n",
     "    s0, s1 = psf.shape\n    ca, cb = (s0 - 1) // 2, (s1 - 1) // 2\n    N = n * n"),
    ("factors-centre", "centre tap at s // 2", "return RFactors(Kx=kmat(s1, s1 // 2), Ky=kmat(s0, s0 // 2)",
     "return RFactors(Kx=kmat(s1, (s1 - 1) // 2), Ky=kmat(s0, (s0 - 1) // 2)"),
    ("index-map-col-transposed", "column map of R(A)", "lst.extend([a] * int(round(My[a][r, rp])))",
     "lst.extend([a] * int(round(My[a][rp, r])))"),
    ("closed-form-Gy", "Gy = Ky^T Ky", "    Gy = (F.Ky.T @ F.Ky).toarray()\n    return np.linalg.svd",
     "    Gy = (F.Kx.T @ F.Kx).toarray()\n    return np.linalg.svd"),
    ("L-last-row", "zero last row of L", "    for i in range(n - 1):\n        L[i, i] = 0.5",
     "    for i in range(n):\n        L[i, i] = 0.5"),
    ("auto-k-cap", "k capped as soon as i reaches the cap", "            elif i >= k_cap:\n                k_sel = k_cap",
     "            elif i > k_cap:\n                k_sel = k_cap"),
    ("auto-k-kp", "k_p = k + p once k is chosen", "                if len(Q) >= kp:\n                    kp = len(Q)",
     "                if len(Q) >= kp:\n                    kp = len(Q) + 1"),
    ("breakdown-t", "breakdown only at rounding level", "if tj <= 100.0 * eps * bnorm:", "if tj <= 1e-3 * bnorm:"),
    ("breakdown-alpha", "breakdown only at rounding level", "if aj <= 100.0 * eps * bnorm:", "if aj <= 1e-3 * bnorm:"),
    ("egkb-k-not-truncated", "truncate to k terms", "k_eff = min(k_sel, kp_eff)", "k_eff = kp_eff"),
    ("egkb-sigma-offset", "leading singular values of C", "sigma=sc[:k_eff]", "sigma=sc[1:k_eff + 1]"),
    ("rsvd-sigma-offset", "leading singular values of H", "sigma=sh[:k]", "sigma=sh[1:k + 1]"),
    ("rsvd-power-BT-dropped", "power step through B^T", "        Z, _ = np.linalg.qr(BT(Qb))",
     "        Z, _ = np.linalg.qr(BT(Qb) * 0 + Qb)"),
    ("terms-sigma-dropped", "sigma_i kept with the terms", "sigma=np.array(ts.sigma[:k], dtype=np.float64)",
     "sigma=np.ones(k)"),
    ("cgls-early-exit", "stop only when tau = 0", "        if tau_k == 0.0:\n            break",
     "        if tau_k < 1e-3:\n            break"),
    ("cgls-step-length", "mu = tau / ||z||^2", "mu = tau_k / zz  # step 4", "mu = tau_k / (zz + tau_k)  # step 4"),
    ("shrink-no-sign", "shrink keeps the sign", "return np.sign(w) * np.maximum", "return np.abs(w) * 0 + np.maximum"),
    ("sb-outer-count", "one outer step per loop", "        ell += 1\n        rec", "        ell += 2\n        rec"),
    ("sb-iota", "iota_total sums the CGLS counts", "iota_total += res.iters", "iota_total += res.iters + 1"),
    ("snr-noise", "noise = b - b_true", "np.sum((b_true - b) ** 2)", "np.sum((b_true + b) ** 2)"),
    # metrics (Sec. 5.3.2)
    ("rel-error-denominator", "RE over ||x_true||", "np.linalg.norm(x - x_true) / np.linalg.norm(x_true)",
     "np.linalg.norm(x - x_true) / np.linalg.norm(x)"),
    ("isnr-swapped", "ISNR", "np.linalg.norm(b - x_true) / np.linalg.norm(x - x_true)",
     "np.linalg.norm(x - x_true) / np.linalg.norm(b - x_true)"),
    ("snr-factor", "SNR in dB of a power ratio", "return float(10.0 * math.log10(np.sum(b_true**2)",
     "return float(20.0 * math.log10(np.sum(b_true**2)"),
]


def run_pins(oracle_text: str) -> bool:
    """True when the oracle pins pass with ``oracle_text`` as the oracle."""
    with tempfile.TemporaryDirectory() as tmp:
        os.mkdir(os.path.join(tmp, "oracle"))
        shutil.copy(os.path.join(ROOT, "oracle", "__init__.py"), os.path.join(tmp, "oracle"))
        with open(os.path.join(tmp, "oracle", "kpsb_oracle.py"), "w") as f:
            f.write(oracle_text)
        env = dict(os.environ, PYTHONPATH=os.pathsep.join([tmp, ROOT]))
        # cwd = tmp puts the copy first on sys.path (python -m adds the working directory)
        r = subprocess.run([sys.executable, "-m", "pytest", "-x", "-q", "-p", "no:cacheprovider",
                            "-m", "not gpu"] + [os.path.join(ROOT, "tests", p) for p in PINS],
                           cwd=tmp, env=env, capture_output=True, text=True, timeout=1800)
        return r.returncode == 0


def main() -> int:
    ap = argparse.ArgumentParser()
    ap.add_argument("-j", type=int, default=4, help="mutants run at once")
    ap.add_argument("-k", default="", help="only entries whose name contains this")
    a = ap.parse_args()
    with open(ORACLE) as f:
        orig = f.read()
    todo = [m for m in MUTATIONS if a.k in m[0]]
    for name, _, old, _ in todo:
        if orig.count(old) != 1:
            print(f"{name}: its text occurs {orig.count(old)} times in the oracle")
            return 2
    if not run_pins(orig):
        print("the pins fail on the unmodified oracle")
        return 2

    def one(m):
        name, what, old, new = m
        return name, what, run_pins(orig.replace(old, new))

    survived = []
    with ThreadPoolExecutor(max_workers=max(1, a.j)) as ex:
        for name, what, passed in ex.map(one, todo):
            print(f"{'SURVIVED' if passed else 'caught  '}  {name:26s} ({what})", flush=True)
            if passed:
                survived.append(name)
    print(f"{len(todo) - len(survived)} of {len(todo)} planted mistakes caught")
    return 1 if survived else 0


if __name__ == "__main__":
    sys.exit(main())
