"""The oracle's own index build: codec training, encoding, graph, regression codebook and
codeword assignment, producing the arrays that both the oracle search and the GPU search
read.  Float64 arithmetic; stored codebooks are rounded to float32 (the precision of the
index arrays) before anything is computed from them.

Test infrastructure only (see the package docstring).
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

from . import codec, graph, refine


@dataclass
class OracleIndex:
    d: int
    M1: int
    M2: int
    R: np.ndarray          # float32 [d][d], y' = R y
    C1: np.ndarray         # float32 [256][d], full-width level-1 centroids
    C2: np.ndarray         # float32 [256][d], full-width level-2 (residual) centroids
    codes1: np.ndarray     # uint8 [N][M1]
    codes2: np.ndarray     # uint8 [N][M2]
    beta: np.ndarray       # uint8 [N] (one block) or [N][bM]: regression codeword(s) per vector
    B: np.ndarray          # float32 [bK][9] (one block) or [bM][bK][9]: regression codebook(s)
    adj0: np.ndarray       # int32 [N][32], level-0 rows sorted by distance to the owner
    upper_off: np.ndarray  # int32 [N], first upper row of a node (-1 if level 0)
    upper_adj: np.ndarray  # int32 [rows][32], upper rows holding global ids
    ep: int
    max_level: int
    levels: np.ndarray     # int32 [N]
    bM: int = 1            # regression blocks (product codebook, Section 4.3)
    bK: int = 256          # codewords per block; 1 = the 0-byte weights beta* (Section 4.2)
    extra: dict = field(default_factory=dict)

    @property
    def N(self) -> int:
        return self.codes1.shape[0]

    def decoded(self) -> np.ndarray:
        """q(x) for every indexed vector, float64, in the rotated space."""
        C1 = self.C1.astype(np.float64)
        C2 = self.C2.astype(np.float64)
        return codec.pq_decode(self.codes1, C1, self.M1) + codec.pq_decode(self.codes2, C2, self.M2)


def build_index(xt: np.ndarray, xb: np.ndarray, M1: int, M2: int, use_opq: bool,
                seed: int = 1804, efc: int = 40, deg: int = 32, batch_max: int = 1,
                batch_div: int = 16, beta_train_n: int = 250_000, beta_iters: int = 10,
                codec_niter: int = 25, opq_outer: int = 10, B: np.ndarray | None = None,
                beta_M: int = 1, beta_K: int = 256) -> OracleIndex:
    """Build an index over ``xb`` with codebooks trained on ``xt``.  ``B`` may supply a
    regression codebook instead of training one.  ``beta_M`` > 1 trains a product
    regression codebook over that many blocks; ``beta_K`` = 1 the 0-byte weights."""
    d = xb.shape[1]
    R, C1, C2 = codec.train_codec(xt, M1, M2, use_opq, seed=seed, niter=codec_niter,
                                  n_outer=opq_outer)
    R32, C1_32, C2_32 = (np.ascontiguousarray(a, np.float32) for a in (R, C1, C2))
    c1, c2, xr, xh = codec.encode(xb, R32.astype(np.float64), C1_32.astype(np.float64),
                                  C2_32.astype(np.float64), M1, M2)
    lev = graph.levels(xb.shape[0], seed)
    adj0, off, uadj, ep, ml = graph.build_graph(xr, xh, lev, deg=deg, deg_up=deg, efc=efc,
                                                batch_max=batch_max, batch_div=batch_div)
    n = xb.shape[0]
    B, beta, hist = _regression(xr, xh, adj0, beta_M, beta_K, seed, beta_train_n, beta_iters, B)
    return OracleIndex(d=d, M1=M1, M2=M2, R=R32, C1=C1_32, C2=C2_32, codes1=c1, codes2=c2,
                       beta=beta, B=B, adj0=adj0, upper_off=off, upper_adj=uadj, ep=ep,
                       max_level=ml, levels=lev, bM=beta_M, bK=beta_K,
                       extra=dict(em_history=hist, xr=xr, xh=xh))


def _regression(xr, xh, adj0, beta_M, beta_K, seed, beta_train_n, beta_iters, B=None):
    """Regression codebook(s) trained on a seeded subset of the indexed vectors, then every
    vector's codeword(s).  Returns (B float32, beta uint8, EM history) in the layouts of
    OracleIndex."""
    n = xr.shape[0]
    hist: list = []
    if B is None:
        g = np.random.Generator(np.random.Philox(np.random.SeedSequence([seed, 5])))
        sub = np.arange(n) if n <= beta_train_n else np.sort(g.choice(n, beta_train_n, replace=False))
        Gs = refine.gmatrix(xh, adj0, sub)
        if beta_M == 1 and beta_K == refine.NBETA:
            B = refine.train_codebook(Gs, xr[sub], iters=beta_iters, seed=seed, history=hist)
        else:
            B = refine.train_product(Gs, xr[sub], beta_M, beta_K, iters=beta_iters, seed=seed, history=hist)
    B32 = np.ascontiguousarray(np.reshape(B, (beta_M, beta_K, refine.KBETA + 1)), np.float32)
    beta = np.empty((n, beta_M), np.uint8)
    for a in range(0, n, 8192):
        idx = np.arange(a, min(n, a + 8192))
        beta[idx] = refine.assign_product(refine.gmatrix(xh, adj0, idx), xr[idx], B32.astype(np.float64))
    if beta_M == 1:
        return B32[0].copy(), beta[:, 0].copy(), hist
    return B32, beta, hist


def with_regression(ix: OracleIndex, beta_M: int, beta_K: int, seed: int = 1804,
                    beta_train_n: int = 250_000, beta_iters: int = 10) -> OracleIndex:
    """The same index (codes, graph) with another regression codebook: ``beta_M`` blocks of
    ``beta_K`` codewords (Section 4.3; ``beta_K`` = 1: the 0-byte weights of Section 4.2)."""
    import dataclasses
    xr, xh = ix.extra["xr"], ix.extra["xh"]
    B, beta, hist = _regression(xr, xh, ix.adj0, beta_M, beta_K, seed, beta_train_n, beta_iters)
    return dataclasses.replace(ix, B=B, beta=beta, bM=beta_M, bK=beta_K,
                               extra=dict(ix.extra, em_history=hist))
