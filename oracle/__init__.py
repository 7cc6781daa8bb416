"""Plain CPU oracle for the Link-and-Code search path (Douze, Sablayrolles, Jegou,
"Link and code: Fast indexing with graphs and compact regression codes", CVPR 2018).

TEST INFRASTRUCTURE ONLY.  The oracle is what the GPU path is checked against.  Only the
tests, the package entry point's ``smoke()`` check and the benchmark's CPU-baseline and
reference legs may import it.  It shares no code with the product (the C-ABI library, its
CUDA kernels and its Python binding) and imports nothing from it; the product never
imports it.  All arithmetic is float64; stored index arrays are float32/uint8/int32.

Modules:
  codec   k-means, PQ, OPQ, two-level residual codec (Section 3.3, 4.1, 5.1)
  graph   HNSW level draws and insertion build (Section 2, 4.1, 5.1)
  refine  G(x), beta*, regression codebook EM and assignment (Section 4.2, 4.3)
  search  two-stage search: ADC walk, shortlist, refined re-rank (Section 2, 4.1, 4.3),
          and exhaustive exact k-NN
  index   the oracle's own index build, feeding both searches

Every function here is pinned by the CPU tests against closed forms, library routines,
brute force or invariants the paper states; see the tests named test_oracle_*.
"""
from . import codec, graph, refine  # noqa: F401
from ._clib import build  # noqa: F401
from .index import OracleIndex, build_index  # noqa: F401
from .search import dists, knn, merge_topk, search, trace  # noqa: F401
