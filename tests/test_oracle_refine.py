"""Pins for the oracle's regression refinement (Section 4.2, 4.3): beta* as the library
least-squares solution, the quadratic-form losses against the direct residual, brute-force
codeword assignment, EM monotonicity, and the per-vector 'never worse than q(x)' bound."""
import numpy as np

from oracle import refine


def _toy(rng, n=300, d=12):
    G = rng.standard_normal((n, refine.KBETA + 1, d))
    true = np.array([0.7, 0.2, 0.1, 0.05, 0, 0, 0, 0, 0])
    x = np.einsum("j,njd->nd", true, G) + 0.05 * rng.standard_normal((n, d))
    return G, x


def test_beta_star_is_the_pseudoinverse_solution(rng):
    # Section 4.2: L(beta) = ||X - beta^T Y||^2 has the closed form beta* = Y^+ X
    G, x = _toy(rng)
    Y = np.concatenate([G[i].T for i in range(G.shape[0])], 0)       # [n*d][9]
    X = np.concatenate(list(x), 0)
    ref = np.linalg.pinv(Y) @ X
    lst = np.linalg.lstsq(Y, X, rcond=None)[0]
    got = refine.beta_star(G, x)
    assert np.allclose(got, ref, rtol=1e-9, atol=1e-10)
    assert np.allclose(got, lst, rtol=1e-9, atol=1e-10)


def test_single_cluster_update_equals_lstsq(rng):
    # Eq. for one cluster: the update is the same least squares restricted to its members
    G, x = _toy(rng, n=120)
    B = refine.train_codebook(G, x, n_beta=2, iters=1)
    a = refine.assign_codewords(G, x, B)
    m = a == 1
    assert m.any()
    Y = np.concatenate([G[i].T for i in np.flatnonzero(m)], 0)
    X = np.concatenate([x[i] for i in np.flatnonzero(m)], 0)
    assert np.allclose(B[1], np.linalg.lstsq(Y, X, rcond=None)[0], rtol=1e-8, atol=1e-9)
    assert np.array_equal(B[0], refine.e0())


def test_quadratic_losses_equal_direct_residuals(rng):
    G, x = _toy(rng, n=50)
    B = rng.standard_normal((17, 9))
    A, b = refine.normal_eq(G, x)
    q = refine.quad_losses(A, b, (x ** 2).sum(1), B)
    direct = np.array([[np.sum((x[i] - B[c] @ G[i]) ** 2) for c in range(17)] for i in range(50)])
    assert np.allclose(q, direct, rtol=1e-10, atol=1e-10)


def test_assignment_is_exhaustive_argmin(rng):
    G, x = _toy(rng, n=40)
    B = rng.standard_normal((256, 9)) * 0.3
    B[0] = refine.e0()
    a = refine.assign_codewords(G, x, B)
    for i in range(40):
        errs = [np.sum((x[i] - B[c] @ G[i]) ** 2) for c in range(256)]
        assert a[i] == int(np.argmin(errs))


def test_em_loss_non_increasing(rng):
    G, x = _toy(rng, n=600)
    hist = []
    refine.train_codebook(G, x, n_beta=16, iters=6, history=hist)
    assert len(hist) == 12
    for a, b in zip(hist, hist[1:]):
        assert b <= a * (1 + 1e-12)


def test_estimator_ordering(rng):
    # Section 3.2: per-vector regression <= shared weights beta* <= q(x) alone (= e0)
    G, x = _toy(rng)
    A, b = refine.normal_eq(G, x)
    per = refine.ridge_solve(A, b)
    e_per = np.array([np.sum((x[i] - per[i] @ G[i]) ** 2) for i in range(len(x))])
    bs = refine.beta_star(G, x)
    e_bs = refine.losses(G, x, bs[None])[:, 0]
    e_q = refine.losses(G, x, refine.e0()[None])[:, 0]
    assert np.all(e_per <= e_bs * (1 + 1e-9) + 1e-12)
    assert e_bs.sum() <= e_q.sum()


def test_refined_error_never_worse_than_qx(mix3k):
    # codeword 0 = e0 is always available, so the chosen beta is never worse than q(x)
    ix, xb, _ = mix3k
    xr = ix.extra["xr"]
    xh = ix.extra["xh"]
    G = refine.gmatrix(xh, ix.adj0, np.arange(ix.N))
    B = ix.B.astype(np.float64)
    ref = refine.losses_assigned(G, xr, B, ix.beta.astype(np.int64))
    base = ((xr - xh) ** 2).sum(1)
    assert np.all(ref <= base * (1 + 1e-9))
    assert ref.mean() < base.mean()          # and it helps on average (Section 4.3)
    # the shared weight on q(x) itself lies in the range the paper reports (0.5 - 0.9)
    bs = refine.beta_star(G, xr)
    assert 0.4 < bs[0] < 1.0


def test_gmatrix_rows_follow_adjacency(mix3k):
    ix, _, _ = mix3k
    xh = ix.extra["xh"]
    G = refine.gmatrix(xh, ix.adj0, np.arange(20))
    for i in range(20):
        assert np.array_equal(G[i, 0], xh[i])
        for j in range(refine.KBETA):
            v = ix.adj0[i, j]
            if v >= 0:
                assert np.array_equal(G[i, j + 1], xh[v])
            else:
                assert not G[i, j + 1].any()
