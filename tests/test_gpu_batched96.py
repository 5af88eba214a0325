"""The 96-problem uneven batch (n in {64, 128, 256, 384}, 24 each; odd PSF sides 15..63,
Gaussian-mixture and turbulence PSFs, zero and reflexive boundaries, iso and aniso TV, k in
[5, 20]) built and solved in one batched call each, with two outer steps per problem (the full
100 are what the bench times).  Every problem must equal its build and its solve alone, bit for
bit, whatever kernels its size group ran on (tensor-core variants give identical bits, the
vector kernels reduce in a fixed order per problem)."""
import numpy as np
import pytest

from oracle import kpsb_oracle as O
from paper_2410_00233_gb300 import inputs as I
from tests.gpu_util import need_gpu

pytestmark = pytest.mark.gpu


def test_96_uneven_problems_equal_alone():
    need_gpu()
    from paper_2410_00233_gb300 import kpsb as K

    prs = [I.problem_batched(i) for i in range(96)]
    assert sorted({pr.n for pr in prs}) == [64, 128, 256, 384]
    assert {pr.bc for pr in prs} == {K.BC_ZERO, K.BC_REFLEXIVE} and {pr.iso for pr in prs} == {False, True}
    bs = []
    for pr in prs:
        bt = O.blur(pr.psf, pr.x_true, pr.bc)
        bs.append(bt + I.noise_vector(bt, pr.eta, pr.zeta))
    probs = [dict(psf=pr.psf, n=pr.n, bc=pr.bc, rank_or_tol=pr.k, method=K.EGKB, p=pr.p, seed=pr.seed)
             for pr in prs]
    kps = K.kp_build_batched(probs)
    jobs = [dict(kp=kp, b=b, mu=1.0, lam=0.1, tv=K.ISO if pr.iso else K.ANISO, iters=2)
            for kp, b, pr in zip(kps, bs, prs)]
    outs, stats = K.sb_solve_batched(jobs, prec=K.P_TF32X2)
    assert all(np.all(np.isfinite(x)) for x in outs)
    assert all(s.l_end == 2 and s.iota_total > 0 for s in stats)
    # one problem of every (size, boundary, TV type) combination present, alone
    seen = set()
    for i, pr in enumerate(prs):
        key = (pr.n, pr.bc, pr.iso)
        if key in seen:
            continue
        seen.add(key)
        kp_a = K.kp_build(pr.psf, pr.n, pr.bc, pr.k, K.EGKB, p=pr.p, seed=pr.seed)
        fa = K.kp_get_factors(kp_a)
        fb = K.kp_get_factors(kps[i])
        assert all(np.array_equal(a, b) for a, b in zip(fa, fb)), ("factors", i)
        x, st = K.sb_solve(kps[i], bs[i], 1.0, 0.1, K.ISO if pr.iso else K.ANISO, 2, prec=K.P_TF32X2)
        assert np.array_equal(x, outs[i]) and st.iota_total == stats[i].iota_total, ("solve", i, pr.n)
    assert len(seen) == 16  # 4 sizes x 2 boundaries x 2 TV types
