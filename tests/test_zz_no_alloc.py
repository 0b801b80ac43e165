"""pr_solve_noalloc: the solve for callers that cannot let the library allocate
device memory (their memory belongs to their own pool or caching allocator,
they run under a fixed budget, or they cannot take the device synchronisation
of cudaMalloc/cudaFree). It keeps its working set in one fixed device array.

Its answers are compared with pr_solve's on the same graphs, within the rank
and iteration tolerance of the other GPU tests, on two calls in a row (the
second call runs on what the first left in the shared array). This file is
collected last so that a run stopping at the first failure has run every
other test first."""
import ctypes as C

import numpy as np
import pytest

from tests.parity import RANK_REL_L1, rel_l1

pytestmark = pytest.mark.gpu


def _noalloc(B, dg, alpha, tau, norm, max_iter, out, stream):
    it, err, conv = C.c_int32(), C.c_double(), C.c_int32()
    addr = out.data_ptr() if hasattr(out, "data_ptr") else out.ctypes.data
    st = B.lib().pr_solve_noalloc(dg.handle, alpha, tau, norm, max_iter, addr, stream,
                                  C.byref(it), C.byref(err), C.byref(conv))
    return st, it.value, err.value, bool(conv.value)


def test_noalloc_matches_pr_solve_two_calls_in_a_row(gg):
    import torch

    from paper_2108_02997_gb300 import binding as B
    B.lib()
    stream = torch.cuda.current_stream()
    sptr = int(stream.cuda_stream)
    cases = [(gg.erdos_renyi_10k(seed=1), 0.85, 1e-10, 1),
             (gg.rmat(16, 16, seed=16), 0.85, 1e-9, 3),
             (gg.from_edges(3000, list(range(1, 3000)), [0] * 2999), 0.9, 1e-10, 2)]
    for g, alpha, tau, norm in cases:
        with B.Graph.from_csr(g) as dg:
            ref = torch.empty(g.n, dtype=torch.float64, device="cuda")
            r = B.pr_solve(dg, alpha, tau, norm, 500, out=ref)
            for call in range(2):
                out = torch.full((g.n,), float("nan"), dtype=torch.float64, device="cuda")
                st, it, err, conv = _noalloc(B, dg, alpha, tau, norm, 500, out, sptr)
                assert st == 0, B.lib().pr_last_error()
                got = out.cpu().numpy()
                assert np.isfinite(got).all()
                assert rel_l1(got, ref.cpu().numpy()) <= RANK_REL_L1, (g.n, call)
                assert it == r.iters and conv == r.converged
                assert abs(err - r.err) <= 2 * RANK_REL_L1


def test_noalloc_rejects_graphs_beyond_its_scratch(gg):
    import torch

    from paper_2108_02997_gb300 import binding as B
    n = 2_000_000
    g = gg.from_edges(n, [], [])
    with B.Graph.from_csr(g) as dg:
        out = torch.empty(n, dtype=torch.float64, device="cuda")
        st, *_ = _noalloc(B, dg, 0.85, 1e-6, 1, 10, out, int(torch.cuda.current_stream().cuda_stream))
        assert st == B.PR_EINVAL
        assert b"no-alloc scratch" in B.lib().pr_last_error()


def test_noalloc_rejects_a_host_output_buffer(gg):
    """The kernels write the output: a host buffer is refused before any work."""
    import torch

    from paper_2108_02997_gb300 import binding as B
    g = gg.rmat(10, 8, seed=3)
    with B.Graph.from_csr(g) as dg:
        host = np.full(g.n, -1.0)
        st, *_ = _noalloc(B, dg, 0.85, 1e-8, 1, 100, host, int(torch.cuda.current_stream().cuda_stream))
        assert st == B.PR_EINVAL
        assert b"device memory" in B.lib().pr_last_error()
        assert (host == -1.0).all()


def test_noalloc_allocates_no_device_memory(gg):
    """After a first call (which looks up the array's address), further calls
    leave the device's free memory and the library's workspace pool as they
    were."""
    import torch

    from paper_2108_02997_gb300 import binding as B
    g = gg.rmat(15, 16, seed=15)
    sptr = int(torch.cuda.current_stream().cuda_stream)
    with B.Graph.from_csr(g) as dg:
        outs = [torch.empty(g.n, dtype=torch.float64, device="cuda") for _ in range(3)]
        st, *_ = _noalloc(B, dg, 0.85, 1e-9, 1, 500, outs[0], sptr)
        assert st == 0, B.lib().pr_last_error()
        torch.cuda.synchronize()
        free0 = torch.cuda.mem_get_info()[0]
        pool0 = B.workspace_info()
        for o in outs[1:]:
            st, *_ = _noalloc(B, dg, 0.85, 1e-9, 1, 500, o, sptr)
            assert st == 0, B.lib().pr_last_error()
        torch.cuda.synchronize()
        assert torch.cuda.mem_get_info()[0] == free0
        assert B.workspace_info() == pool0
        assert torch.equal(outs[1], outs[2]) and torch.equal(outs[0], outs[1])
