"""GB300 (sm_103a) frequency-domain CQM boundary elements for the acoustic
single layer, with H^2 far field and frequency ACA (Seibel, arXiv 2006.05186).

The compute path is the CUDA library libcqmbem.so behind the C ABI in
include/cqm_bem.h; this package is its binding (`CqmBem`), the in-tree build
(`build`), and seeded synthetic inputs (`synth`).
"""
from ._lib import CqmBem, CqmError, Server, default_params, estimate_bytes, load  # noqa: F401
from . import synth  # noqa: F401
