"""Failure detection on the device, made to happen without a GPU fault.

Every wait or walk in the library's kernels is bounded.  The tile merge,
which unites the parts of a segment that crosses detection-tile edges,
follows union-find chains in device memory; a chain longer than the
context's walk limit makes the walk give up and record GP_ERR_TIMEOUT in the
context's device status word.  The test lowers the limit to one step on a
spiral segment that crosses hundreds of tile edges, checks that gp_ctx_sync
reports GP_ERR_TIMEOUT (the kernels returned; nothing hung), then restores
the default and checks that the same context and stream still give the
oracle's labels.
"""
import numpy as np
import pytest

import oracle

torch = pytest.importorskip("torch")
gp = pytest.importorskip("paper_2609_32375_gb300")

pytestmark = pytest.mark.gpu


def spiral(n=600):
    s = np.zeros((n, n), np.uint8)
    for k in range(0, n // 2, 2):
        s[k, k:n - k] = 1
        s[k:n - k, n - k - 1] = 1
        s[n - k - 1, k + 2:n - k] = 1
        if k + 2 < n - k:
            s[k + 2:n - k, k + 2] = 1
    return s


def test_walk_limit_reports_timeout_and_the_context_recovers():
    mask = spiral()
    ref, nref = oracle.label(mask, 1)
    assert nref <= 2                                   # one long segment (plus possibly a centre dot)
    ctx = gp.Context(0, workspace_bytes=256 << 20)
    try:
        t = torch.from_numpy(mask).cuda()
        ctx.set_walk_limit(1)
        ctx.gp_label_mask(t, 1)
        with pytest.raises(gp.GpError) as e:
            ctx.sync()
        assert e.value.status == gp.GP_ERR_TIMEOUT
        # the default bound again: the same context labels the mask exactly
        ctx.set_walk_limit(0)
        seg, n = ctx.gp_label_mask(t, 1)
        ctx.sync()
        assert np.array_equal(seg.cpu().numpy().view(np.uint32), ref)
        assert int(n.item()) == nref
        # a negative limit is an argument error, detected on the host
        with pytest.raises(gp.GpError) as e:
            ctx.set_walk_limit(-1)
        assert e.value.status == gp.GP_ERR_INVALID_ARG
    finally:
        ctx.close()
