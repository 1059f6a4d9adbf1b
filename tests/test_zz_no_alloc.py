"""The cluster tree entry point that allocates no device memory.

It serves callers that may not call cudaMalloc (another runtime owns the
device memory, or an allocation, which can synchronise the device, is not
allowed where they run).  This test calls it through the C ABI twice in a
row, on two meshes, with buffers allocated by the caller, and checks that it
returns exactly the tree that cqm_bem_setup builds (the tree is integer and
ordering work, so the check is bit for bit).
"""
import ctypes as C

import numpy as np
import pytest

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


def _tree_without_allocation(lib, mesh, n_min=32):
    dev = torch.device("cuda")
    xyz = torch.tensor(mesh.xyz, dtype=torch.float64, device=dev)
    tri = torch.tensor(mesh.tri, dtype=torch.int32, device=dev)
    nt = mesh.nt
    cap = 2 * nt - 1
    out = {k: torch.full((cap,), -7, dtype=torch.int32, device=dev)
           for k in ("begin", "end", "son0", "son1", "parent", "level")}
    perm = torch.full((nt,), -7, dtype=torch.int32, device=dev)
    lo = torch.zeros((cap, 3), dtype=torch.float64, device=dev)
    hi = torch.zeros((cap, 3), dtype=torch.float64, device=dev)
    n_nodes = C.c_int32(0)
    stream = torch.cuda.current_stream().cuda_stream
    p = lambda t: C.c_void_p(t.data_ptr())
    rc = lib.cqm_cluster_tree_noalloc(p(xyz), mesh.nv, p(tri), nt, n_min, p(perm), p(out["begin"]),
                                      p(out["end"]), p(out["son0"]), p(out["son1"]),
                                      p(out["parent"]), p(out["level"]), p(lo), p(hi),
                                      C.byref(n_nodes), C.c_void_p(stream))
    assert rc == 0, lib.cqm_bem_last_error()
    n = n_nodes.value
    res = {k: v[:n].cpu().numpy() for k, v in out.items()}
    res.update(perm=perm.cpu().numpy(), lo=lo[:n].cpu().numpy(), hi=hi[:n].cpu().numpy(), n=n)
    return res


def test_tree_without_allocation_matches_setup_on_two_calls():
    from paper_2006_05186_gb300 import CqmBem, _lib, build, synth
    build.build()
    lib = _lib.load()
    for mesh in (synth.icosphere(3), synth.torus_for(1280)):
        op = CqmBem(mesh.xyz, mesh.tri, 0.1, 4, 2, mode="h2maca", rank_cap=3)
        ref = op.tree()
        op.close()
        got = _tree_without_allocation(lib, mesh)
        assert got["n"] == len(ref["begin"])
        for k in ("perm", "begin", "end", "son0", "son1", "level", "lo", "hi"):
            assert np.array_equal(got[k], ref[k]), k
        assert got["parent"][0] == -1


def test_tree_without_allocation_rejects_oversize_and_bad_indices():
    from paper_2006_05186_gb300 import _lib, build, synth
    build.build()
    lib = _lib.load()
    dummy = torch.zeros(16, dtype=torch.int32, device="cuda")
    n_nodes = C.c_int32(0)
    p = C.c_void_p(dummy.data_ptr())
    rc = lib.cqm_cluster_tree_noalloc(p, 3, p, 65537, 32, p, p, p, p, p, p, p, p, p,
                                      C.byref(n_nodes), None)
    assert rc == _lib.CQM_EINVAL and b"exceed" in lib.cqm_bem_last_error()
    mesh = synth.icosphere(0)
    bad = mesh.tri.copy()
    bad[3, 1] = mesh.nv + 5
    lib_out = _tree_without_allocation
    with pytest.raises(AssertionError):
        class M:
            xyz, tri, nt, nv = mesh.xyz, bad, mesh.nt, mesh.nv
        lib_out(lib, M)
    assert b"out of range" in lib.cqm_bem_last_error()
