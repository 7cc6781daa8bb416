import os
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (sm_103a); parity tests against the oracle")


_CACHE: dict = {}


def oracle_index(name: str):
    """Small indexes built by the oracle's own build, cached for the session.

    mix3k   3,000 x 96-d mixture, PQ16 + residual PQ16, no rotation
    mix10k  the 10k-vector workload (1,000 queries), PQ16 + residual PQ16
    opq3k   3,000 x 96-d mixture (256 centres), OPQ32 + residual PQ31 (64-byte shape)
    sift2k  2,000 x 128-d SIFT-like, OPQ64 + residual PQ63 (128-byte shape)
    odd2k   2,000 x 40-d mixture, PQ16 + residual PQ10 (uneven sub-space splits)
    """
    if name in _CACHE:
        return _CACHE[name]
    import oracle
    from paper_1804_09996_gb300 import datagen as dg
    spec = {
        "mix3k": dict(kind="mixture", n=3000, nt=5000, nq=300, d=96, c=64, M1=16, M2=16, opq=False),
        "mix10k": dict(kind="mixture", n=10000, nt=10000, nq=1000, d=96, c=64, M1=16, M2=16, opq=False),
        "opq3k": dict(kind="mixture", n=3000, nt=6000, nq=300, d=96, c=256, M1=32, M2=31, opq=True),
        "sift2k": dict(kind="sift", n=2000, nt=4000, nq=200, d=128, c=256, M1=64, M2=63, opq=True),
        "odd2k": dict(kind="mixture", n=2000, nt=3000, nq=200, d=40, c=32, M1=16, M2=10, opq=False),
    }[name]
    xt = dg.make(spec["kind"], spec["nt"], spec["d"], spec["c"], dg.STREAM_TRAIN)
    xb = dg.make(spec["kind"], spec["n"], spec["d"], spec["c"], dg.STREAM_BASE)
    xq = dg.make(spec["kind"], spec["nq"], spec["d"], spec["c"], dg.STREAM_QUERY)
    ix = oracle.build_index(xt, xb, spec["M1"], spec["M2"], spec["opq"],
                            opq_outer=4 if spec["opq"] else 10)
    _CACHE[name] = (ix, xb, xq)
    return _CACHE[name]


@pytest.fixture(scope="session")
def mix3k():
    return oracle_index("mix3k")


@pytest.fixture(scope="session")
def mix10k():
    return oracle_index("mix10k")


@pytest.fixture(scope="session")
def opq3k():
    return oracle_index("opq3k")


@pytest.fixture(scope="session")
def sift2k():
    return oracle_index("sift2k")


@pytest.fixture(scope="session")
def odd2k():
    return oracle_index("odd2k")


@pytest.fixture
def rng():
    return np.random.default_rng(12345)
