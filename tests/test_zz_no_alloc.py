"""The allocation-free entry point (mpn_propagate_noalloc), called through the
C ABI on two grids in a row, against the CPU oracle and against the regular
entry point (mpn_create + mpn_propagate + mpn_get_distances), bit for bit.

The entry point serves callers that cannot allocate device memory: code inside
another framework's memory pool or a fixed budget, or a loop where an
allocation and the synchronisation it implies are not allowed. Its scratch is
one fixed device array shared by all calls, so the second call also checks
that leftovers of the first are cleared, and that the call itself allocates
no device memory. This file is collected last so that a failure here stops a
-x run only after every other test has run."""
import numpy as np
import pytest

import oracle
import synth
import paper_2004_00540_gb300 as pkg

pytestmark = pytest.mark.gpu


def _regular(mask, targets):
    with pkg.Planner(mask, pkg.MPN_DIST_U32) as pl:
        layers = pl.propagate(targets)
        return pl.distances(), layers


def _oracle(mask, targets):
    d, _ = oracle.bfs(mask, targets)
    return d   # uint32, 0xFFFFFFFF where unreached or on an obstacle


def test_noalloc_matches_oracle_and_regular_two_calls():
    torch = pytest.importorskip("torch")
    cases = []
    m1 = synth.bernoulli(700, 1100, 0.3, 21)
    cases.append((m1, synth.sample_free(m1, 5, 22)))
    m2 = synth.dfs_maze(513, 257, 23)          # different shape: stale scratch must not leak
    cases.append((m2, synth.sample_free(m2, 2, 24)))
    stream = torch.cuda.current_stream()
    for i, (mask, targets) in enumerate(cases):
        H, W = mask.shape
        want = _oracle(mask, targets)
        regular, _ = _regular(mask, targets)
        assert np.array_equal(regular, want)
        d_mask = torch.from_numpy(mask).cuda()
        d_t = torch.from_numpy(targets.view(np.int32)).cuda()
        d_out = torch.empty((H, W), dtype=torch.int32, device="cuda")
        torch.cuda.synchronize()
        free0 = torch.cuda.mem_get_info()[0]
        alloc0 = torch.cuda.memory_allocated()
        st = pkg.mpn_propagate_noalloc(d_mask, H, W, d_t, d_out, 0, stream)
        torch.cuda.synchronize()
        if i == 1:
            # the first call may load the library's device code and its array
            # (lazy module loading); the second allocates nothing at all
            assert torch.cuda.mem_get_info()[0] == free0
            assert torch.cuda.memory_allocated() == alloc0
        assert st == pkg.MPN_OK, pkg.status_name(st)
        got = d_out.cpu().numpy().view(np.uint32)
        assert np.array_equal(got, want)
        assert np.array_equal(got, regular)


def test_noalloc_rejects_oversize_bad_targets_and_host_buffers():
    torch = pytest.importorskip("torch")
    stream = torch.cuda.current_stream()
    big = torch.zeros((2049, 8), dtype=torch.uint8, device="cuda")
    t = torch.zeros(1, dtype=torch.int32, device="cuda")
    out = torch.empty((2049, 8), dtype=torch.int32, device="cuda")
    assert pkg.mpn_propagate_noalloc(big, 2049, 8, t, out, 0, stream) == pkg.MPN_EINVAL
    m = torch.ones((16, 16), dtype=torch.uint8, device="cuda")
    out = torch.empty((16, 16), dtype=torch.int32, device="cuda")
    assert pkg.mpn_propagate_noalloc(m, 16, 16, t, out, 0, stream) == pkg.MPN_EOBSTACLE
    m.zero_()
    # buffers the kernels cannot use in place: refused before any GPU work
    with pytest.raises(TypeError):
        pkg.mpn_propagate_noalloc(m.cpu(), 16, 16, t, out, 0, stream)
    with pytest.raises(TypeError):
        pkg.mpn_propagate_noalloc(m, 16, 16, t, np.zeros(256, np.uint32), 0, stream)
    with pytest.raises(ValueError):
        pkg.mpn_propagate_noalloc(m, 16, 16, t, out[:8], 0, stream)
    with pytest.raises(ValueError):
        pkg.mpn_propagate_noalloc(m, 16, 16, t.to(torch.int64), out, 0, stream)
    # the C entry point checks the pointers itself: host memory is MPN_EINVAL
    L = pkg.load()
    h_out = np.zeros(256, np.uint32)
    assert L.mpn_propagate_noalloc(m.data_ptr(), 16, 16, t.data_ptr(), 1, 0,
                                   h_out.ctypes.data, stream.cuda_stream) == pkg.MPN_EINVAL
    h_mask = np.zeros(256, np.uint8)
    assert L.mpn_propagate_noalloc(h_mask.ctypes.data, 16, 16, t.data_ptr(), 1, 0,
                                   out.data_ptr(), stream.cuda_stream) == pkg.MPN_EINVAL
    assert pkg.mpn_propagate_noalloc(m, 16, 16, t, out, 0, stream) == pkg.MPN_OK
    torch.cuda.synchronize()
    want = _oracle(np.zeros((16, 16), np.uint8), np.array([0], np.uint32))
    assert np.array_equal(out.cpu().numpy().view(np.uint32), want)
