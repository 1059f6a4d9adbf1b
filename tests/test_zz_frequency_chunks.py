"""Frequency chunking of the inner far coupling.

The bf16 tensor-core coupling puts 128 frequencies on the MMA rows per pass
(the TF32 one at most 160 frequency columns); with more solved frequencies
every chunk gets its own pass through the same pipeline, and a remainder of 1
to 4 frequencies is applied from an expanded FP32 table instead.  This
checks, for the tensor-core and the SIMT couplings, that the inner operator
still agrees with the FP64-accurate apply to 1e-5 at every frequency.
(Collected after the other GPU tests.)
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


@pytest.mark.parametrize("tensor_cores,N", [(1, 340), (1, 256), (1, 262), (2, 340), (0, 340)])
def test_inner_operator_across_frequency_chunks(lib, tensor_cores, N):
    """N = 340 (Ls = 171): two chunks of 128 frequencies, the second padded;
    N = 256, 262 (Ls = 129, 132): one chunk and 1 or 4 tail frequencies applied
    from the expanded FP32 table."""
    from paper_2006_05186_gb300 import CqmBem
    m = synth.icosphere(3)
    dt = 0.1
    op = CqmBem(m.xyz, m.tri, dt, N, 2, mode="h2maca", tensor_cores=tensor_cores)
    assert op.Ls > 128 and op.info()["n_far"] > 0
    rng = np.random.default_rng(13)
    x = rng.standard_normal((op.Ls, m.nt)) + 1j * rng.standard_normal((op.Ls, m.nt))
    y = op.apply(x)
    yi = op.apply_inner(x)
    op.close()
    err = np.linalg.norm(yi - y, axis=1) / np.linalg.norm(y, axis=1)
    assert np.max(err) < 1e-5, (int(np.argmax(err)), float(np.max(err)))
