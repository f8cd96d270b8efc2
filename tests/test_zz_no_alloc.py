"""The allocation-free entry point (mpn_propagate_noalloc) against the
regular one (mpn_create + mpn_propagate), bit for bit, on two calls in a row.

It serves callers that cannot allocate device memory (inside another
framework's pool or a fixed budget, or where an allocation is not allowed at
run time); its scratch is one fixed device array shared by all calls, so the
second call also checks that leftovers of the first are cleared. This file is
collected last so that a failure here stops a -x run only after every other
test has run."""
import numpy as np
import pytest

import synth
import paper_2004_00540_gb300 as pkg

pytestmark = pytest.mark.gpu


def _regular(mask, targets):
    with pkg.Planner(mask, pkg.MPN_DIST_U32) as pl:
        layers = pl.propagate(targets)
        return pl.distances(), layers


def test_noalloc_matches_regular_two_calls():
    torch = pytest.importorskip("torch")
    cases = []
    m1 = synth.bernoulli(700, 1100, 0.3, 21)
    cases.append((m1, synth.sample_free(m1, 5, 22)))
    m2 = synth.dfs_maze(513, 257, 23)          # different shape: stale scratch must not leak
    cases.append((m2, synth.sample_free(m2, 2, 24)))
    stream = torch.cuda.current_stream()
    for mask, targets in cases:
        H, W = mask.shape
        want, _ = _regular(mask, targets)
        d_mask = torch.from_numpy(mask).cuda()
        d_t = torch.from_numpy(targets.view(np.int32)).cuda()
        d_out = torch.empty((H, W), dtype=torch.int32, device="cuda")
        st = pkg.mpn_propagate_noalloc(d_mask, H, W, d_t, d_out, 0, stream)
        assert st == pkg.MPN_OK, pkg.status_name(st)
        torch.cuda.synchronize()
        got = d_out.cpu().numpy().view(np.uint32)
        assert np.array_equal(got, want)


def test_noalloc_rejects_oversize_and_bad_targets():
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
    assert pkg.mpn_propagate_noalloc(m, 16, 16, t, out, 0, stream) == pkg.MPN_OK
    torch.cuda.synchronize()
    assert int(out.max().item()) == 15 and int(out[0, 0].item()) == 0
