"""SIVF spherical k-means (Aoyama & Saito, arXiv 2103.16141) on GB300 (sm_103a).

The assignment step (Algorithm 4) and update step (Algorithm 5) run as
hand-written CUDA kernels in lib/libsivf.so behind the C ABI of
include/sivf.h; this package is the thin Python binding.
"""
from .sivf import SIVF, SIVFBatch, SivfError, load, library_path  # noqa: F401
