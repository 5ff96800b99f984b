"""Seeded synthetic inputs shared by the oracle and the CUDA path.

Nothing here computes any step of the clustering method: it only writes the
document-term matrix (CSR, fp32 tf-idf, L2-normalised rows) and the seeded
initial centroid document ids.
"""
from .corpus import Corpus, generate, init_ids, build_library  # noqa: F401
from .configs import CONFIGS, small_config, batched_instances  # noqa: F401
