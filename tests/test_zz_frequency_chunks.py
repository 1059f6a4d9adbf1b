"""Frequency chunking of the inner far coupling.

The tensor-core coupling holds at most 160 frequency columns in one TMEM
accumulator pass; with more solved frequencies (N >= 320) every chunk of
columns gets its own pass through the same slab pipeline.  This checks, for
the tensor-core and the SIMT coupling, that the FP32 inner operator still
agrees with the FP64-accurate apply to FP32 accuracy at every frequency when
Ls spans two chunks.  (Collected after the other GPU tests.)
"""
import numpy as np
import pytest

from paper_2006_05186_gb300 import synth

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def lib():
    from paper_2006_05186_gb300 import build, _lib
    build.build()
    return _lib.load()


@pytest.mark.parametrize("tensor_cores", [1, 0])
def test_inner_operator_across_frequency_chunks(lib, tensor_cores):
    from paper_2006_05186_gb300 import CqmBem
    m = synth.icosphere(3)
    N, dt = 340, 0.1  # Ls = 171: two chunks of the tensor-core coupling
    op = CqmBem(m.xyz, m.tri, dt, N, 2, mode="h2maca", tensor_cores=tensor_cores)
    assert op.Ls > 160 and op.info()["n_far"] > 0
    rng = np.random.default_rng(13)
    x = rng.standard_normal((op.Ls, m.nt)) + 1j * rng.standard_normal((op.Ls, m.nt))
    y = op.apply(x)
    yi = op.apply_inner(x)
    op.close()
    err = np.linalg.norm(yi - y, axis=1) / np.linalg.norm(y, axis=1)
    assert np.max(err) < 1e-5, (int(np.argmax(err)), float(np.max(err)))
