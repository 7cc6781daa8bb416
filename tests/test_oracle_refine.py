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


# ---- product regression codebook and 0-byte weights per block (Section 4.2, 4.3) ----

def _blocks(d, M):
    # contiguous blocks, the first d mod M one coordinate wider (written out independently)
    sizes = [d // M + (1 if j < d % M else 0) for j in range(M)]
    starts = np.cumsum([0] + sizes[:-1])
    return [np.arange(a, a + s) for a, s in zip(starts, sizes)]


def test_product_zero_byte_is_blockwise_pseudoinverse(rng):
    # one codeword per block: each block's weights solve the least squares restricted to
    # that block's coordinates (Section 4.2's closed form, per block)
    G, x = _toy(rng, n=200, d=13)
    B = refine.train_product(G, x, 4, 1)
    assert B.shape == (4, 1, 9)
    for m, cols in enumerate(_blocks(13, 4)):
        Y = np.concatenate([G[i][:, cols].T for i in range(len(x))], 0)
        X = np.concatenate([x[i][cols] for i in range(len(x))], 0)
        assert np.allclose(B[m, 0], np.linalg.lstsq(Y, X, rcond=None)[0], rtol=1e-8, atol=1e-9)
    assert not np.any(refine.assign_product(G, x, B))        # nothing stored per vector


def test_product_zero_byte_never_worse_than_shared(rng):
    # the shared beta* is one feasible choice in every block, so the blockwise optimum
    # cannot lose to it on the training set
    G, x = _toy(rng, n=300, d=12)
    bs = refine.beta_star(G, x)
    Bp = refine.train_product(G, x, 3, 1)
    whole = sum(np.sum((x[i] - bs @ G[i]) ** 2) for i in range(len(x)))
    prod = 0.0
    for m, cols in enumerate(_blocks(12, 3)):
        prod += sum(np.sum((x[i][cols] - Bp[m, 0] @ G[i][:, cols]) ** 2) for i in range(len(x)))
    assert prod <= whole * (1 + 1e-12)


def test_product_assignment_is_blockwise_exhaustive_argmin(rng):
    G, x = _toy(rng, n=30, d=13)
    B = rng.standard_normal((4, 32, 9)) * 0.3
    B[:, 0] = refine.e0()
    a = refine.assign_product(G, x, B)
    for m, cols in enumerate(_blocks(13, 4)):
        for i in range(30):
            errs = [np.sum((x[i][cols] - B[m, c] @ G[i][:, cols]) ** 2) for c in range(32)]
            assert a[i, m] == int(np.argmin(errs))


def test_product_codebook_e0_and_per_block_bound(rng):
    # codeword 0 of every block is e0, so every block's error is at most that of q(x)
    G, x = _toy(rng, n=400, d=16)
    hist = []
    B = refine.train_product(G, x, 4, 16, iters=4, history=hist)
    assert np.array_equal(B[:, 0], np.tile(refine.e0(), (4, 1)))
    a = refine.assign_product(G, x, B)
    for m, cols in enumerate(_blocks(16, 4)):
        got = np.array([np.sum((x[i][cols] - B[m, a[i, m]] @ G[i][:, cols]) ** 2) for i in range(len(x))])
        base = np.array([np.sum((x[i][cols] - G[i][0, cols]) ** 2) for i in range(len(x))])
        assert np.all(got <= base * (1 + 1e-12) + 1e-15)
    # EM per block: its loss never increases
    assert len(hist) == 4
    for h in hist:
        for u, v in zip(h, h[1:]):
            assert v <= u * (1 + 1e-12)


def test_reconstruct_blocks(rng):
    G, x = _toy(rng, n=20, d=10)
    B = rng.standard_normal((3, 5, 9))
    codes = rng.integers(0, 5, size=(20, 3))
    y = refine.reconstruct(G, B, codes)
    for m, cols in enumerate(_blocks(10, 3)):
        for i in range(20):
            ref = sum(B[m, codes[i, m], j] * G[i, j, cols] for j in range(9))
            assert np.allclose(y[i, cols], ref, rtol=1e-12, atol=1e-14)
