"""Pins for the oracle's codec (Section 3.3, 4.1, 5.1): split rule, brute-force PQ
assignment, k-means properties, OPQ orthogonality and gain, two-level vs one-level error."""
import numpy as np
import pytest

from oracle import codec


def test_splits_uneven_rule():
    # 96 dimensions in 31 blocks: 96 mod 31 = 3 blocks of 4, then 28 of 3
    offs, lens = codec.splits(96, 31)
    assert lens == [4, 4, 4] + [3] * 28
    assert offs[0] == 0 and offs[3] == 12 and offs[-1] + lens[-1] == 96
    assert all(offs[j] + lens[j] == offs[j + 1] for j in range(30))
    offs, lens = codec.splits(128, 63)
    assert lens == [3, 3] + [2] * 61 and sum(lens) == 128
    assert codec.splits(96, 32)[1] == [3] * 32


def test_pq_encode_is_bruteforce_argmin(rng):
    d, M = 10, 3
    X = rng.standard_normal((40, d))
    C = rng.standard_normal((256, d))
    codes = codec.pq_encode(X, C, M)
    offs, lens = codec.splits(d, M)
    for i in range(X.shape[0]):
        for j in range(M):
            best, bestd = -1, np.inf
            for c in range(256):
                dd = sum((X[i, t] - C[c, t]) ** 2 for t in range(offs[j], offs[j] + lens[j]))
                if dd < bestd:
                    best, bestd = c, dd
            assert codes[i, j] == best


def test_pq_roundtrip_of_centroid_vectors(rng):
    d, M = 12, 4
    C = rng.standard_normal((256, d))
    offs, lens = codec.splits(d, M)
    picks = rng.integers(0, 256, size=(25, M))
    X = np.zeros((25, d))
    for j in range(M):
        X[:, offs[j]:offs[j] + lens[j]] = C[picks[:, j], offs[j]:offs[j] + lens[j]]
    codes = codec.pq_encode(X, C, M)
    assert np.array_equal(codes, picks)
    assert np.allclose(codec.pq_decode(codes, C, M), X, atol=0)


def test_kmeans_recovers_separated_clusters(rng):
    true = np.array([[0.0, 0.0], [10.0, 0.0], [0.0, 10.0], [10.0, 10.0]])
    X = np.concatenate([t + 0.1 * rng.standard_normal((200, 2)) for t in true])
    C = codec.kmeans(X, 4, niter=20, seed=3)
    Cr = np.round(C)
    order = np.lexsort((Cr[:, 1], Cr[:, 0]))            # by x, then y
    assert np.allclose(C[order], true[[0, 2, 1, 3]], atol=0.05)


def test_kmeans_objective_never_increases(rng):
    X = rng.standard_normal((800, 3))
    C = codec.kmeans(X, 16, niter=0, seed=1)
    prev = np.inf
    for _ in range(8):
        C = codec.kmeans(X, 16, niter=1, init=C)
        obj = codec.assign(X, C)[1].sum()
        assert obj <= prev * (1 + 1e-12)
        prev = obj


def test_assign_distance_matches_difference_form(rng):
    X = rng.standard_normal((30, 5))
    C = rng.standard_normal((7, 5))
    a, dm = codec.assign(X, C)
    direct = ((X[:, None, :] - C[None]) ** 2).sum(-1)
    assert np.array_equal(a, direct.argmin(1))
    assert np.allclose(dm, direct.min(1), rtol=1e-12, atol=1e-12)


def test_opq_rotation_orthogonal_and_helps(rng):
    # anisotropic correlated data: a rotation that balances variance across sub-spaces helps PQ
    d, M = 8, 4
    A = np.diag([8.0, 6.0, 4.0, 3.0, 0.3, 0.2, 0.1, 0.05])
    Q, _ = np.linalg.qr(rng.standard_normal((d, d)))
    X = rng.standard_normal((3000, d)) @ A @ Q.T
    R, C = codec.opq_train(X, M, n_outer=8, niter_final=10, seed=0)
    assert np.allclose(R @ R.T, np.eye(d), atol=1e-12)
    Xr = X @ R.T
    err_opq = ((Xr - codec.pq_decode(codec.pq_encode(Xr, C, M), C, M)) ** 2).sum(1).mean()
    Cp = codec.pq_train(X, M, niter=10, seed=0)
    err_pq = ((X - codec.pq_decode(codec.pq_encode(X, Cp, M), Cp, M)) ** 2).sum(1).mean()
    assert err_opq < err_pq


def test_two_level_beats_one_level():
    # Section 3.3: the residual level lowers the reconstruction error
    from paper_1804_09996_gb300 import datagen as dg
    xt = dg.gaussian_mixture(4000, 96, 64, stream=dg.STREAM_TRAIN).astype(np.float64)
    xb = dg.gaussian_mixture(1000, 96, 64, stream=dg.STREAM_BASE).astype(np.float64)
    R, C1, C2 = codec.train_codec(xt, 16, 16, use_opq=False, niter=10)
    c1, c2, xr, xh = codec.encode(xb, R, C1, C2, 16, 16)
    e1 = ((xr - codec.pq_decode(c1, C1, 16)) ** 2).sum(1)
    e2 = ((xr - xh) ** 2).sum(1)
    assert e2.mean() < 0.8 * e1.mean()
    assert np.allclose(xr, xb)  # no rotation: R = I
