"""The allocation-free pull matvec (gbx_mxv_pull_noalloc) against gbx_mxv and
against the CPU oracle's masked matvec on the same inputs.

gbx_mxv_pull_noalloc exists for callers that cannot allocate device memory when
they call in (a serving process whose memory is all preallocated by its own
pool, a latency-bound loop that must not trigger the synchronisation an
allocation can cause).  It keeps its scratch in a fixed array inside the
library.  This file is collected last so that a failure here stops a -x run
only after every other test has run; it must pass alone in a fresh process too.
"""
import ctypes

import numpy as np
import pytest

import oracle
import synth
from paper_1804_03327_gb300 import gbx

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


def _reference(g, n, u, m, complement, early_exit):
    w = torch.zeros(n, dtype=torch.uint8, device="cuda")
    desc = gbx.desc_init(direction=gbx.DIR_PULL, transpose=1, mask_complement=int(complement),
                         early_exit=int(early_exit))
    gbx.mxv(gbx.dense(w), gbx.dense(m) if m is not None else None, gbx.LOR_LAND, g, gbx.dense(u), desc)
    torch.cuda.synchronize()
    return w.cpu().numpy()


@pytest.mark.parametrize("name", ["rmat", "rmat-directed", "grid"])
def test_noalloc_matches_gbx_mxv_on_two_calls_in_a_row(name):
    if name == "rmat":
        n, s, d = synth.rmat_edges(14, 16, seed=21)
        sym = True
    elif name == "rmat-directed":
        n, s, d = synth.rmat_edges(13, 8, seed=22)
        sym = False
    else:
        n, s, d = synth.grid_edges(301, 77, p_delete=0.01, seed=23)  # n not a multiple of 32
        sym = True
    og = oracle.graph(n, s, d, symmetrize=sym)
    g = gbx.graph_build(n, s, d, symmetrize=sym)
    rp, col = gbx.graph_csr(g, transpose=True)  # rows of A^T: w = A^T u, as gbx_mxv computes
    cases = [(0.01, 0.6, True, True), (0.3, 0.2, False, False), (0.001, None, False, True)]
    for k, (ud, md, complement, early_exit) in enumerate(cases):
        u_h = synth.vertex_set(n, ud, seed=100 + k)
        m_h = synth.vertex_set(n, md, seed=200 + k) if md is not None else None
        u = torch.from_numpy(u_h).cuda()
        m = torch.from_numpy(m_h).cuda() if m_h is not None else None
        want = _reference(g, n, u, m, complement, early_exit)
        # the oracle's own CSR from the edge list: w = A^T u (Eq 4) with the same mask
        assert np.array_equal(want, oracle.mxv(n, n, og.out_ptr, og.out_col, u_h, m_h, transpose=True,
                                               complement=complement)), (name, k)
        for call in range(2):  # the second call reuses the scratch the first one left behind
            w = torch.full((n,), 7, dtype=torch.uint8, device="cuda")
            gbx.mxv_pull_noalloc(n, rp, col, u, m, w, complement, early_exit)
            torch.cuda.synchronize()
            assert np.array_equal(w.cpu().numpy(), want), (name, k, call)


def test_noalloc_complement_without_mask_and_limits():
    n, s, d = synth.rmat_edges(10, 16, seed=1)
    g = gbx.graph_build(n, s, d)
    rp, col = gbx.graph_csr(g, transpose=True)
    u = torch.ones(n, dtype=torch.uint8, device="cuda")
    w = torch.full((n,), 3, dtype=torch.uint8, device="cuda")
    gbx.mxv_pull_noalloc(n, rp, col, u, None, w, mask_complement=True)
    torch.cuda.synchronize()
    assert not w.cpu().numpy().any()  # the complement of "no mask" passes nothing
    lib = gbx.load()
    st = lib.gbx_mxv_pull_noalloc((1 << 24) + 1, rp, col, u.data_ptr(), None, 0, 1, w.data_ptr(), None)
    assert st == gbx.ERR_INVALID_VALUE
    assert b"fixed scratch" in lib.gbx_last_error()
    st = lib.gbx_mxv_pull_noalloc(n, rp, col, u.data_ptr(), None, 0, 1, u.data_ptr(), None)
    assert st == gbx.ERR_INVALID_VALUE


def test_noalloc_calls_leave_free_device_memory_unchanged():
    """After the first call on the device (which may place the library's module and
    its fixed array there), further calls allocate nothing: the device's free
    memory is the same before and after them."""
    n, s, d = synth.rmat_edges(12, 16, seed=24)
    g = gbx.graph_build(n, s, d)
    rp, col = gbx.graph_csr(g, transpose=True)
    u = torch.from_numpy(synth.vertex_set(n, 0.05, seed=1)).cuda()
    m = torch.from_numpy(synth.vertex_set(n, 0.5, seed=2)).cuda()
    w = torch.zeros(n, dtype=torch.uint8, device="cuda")
    gbx.mxv_pull_noalloc(n, rp, col, u, m, w, True, True)  # warm-up call
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    for _ in range(5):
        gbx.mxv_pull_noalloc(n, rp, col, u, m, w, True, True)
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    assert free1 == free0
    g.free()
