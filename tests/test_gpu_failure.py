"""Failure detection on the GPU, without a GPU fault.

Every wait in the library's kernels is bounded.  The failure is made on the
host: spider_batch_drop_item leaves one work item of the persistent batch
queue out, so the items of the next pass that need that tile wait for a pass
counter that never advances.  With a short wait limit the kernel records a
timeout and finishes; spider_batch must report SPIDER_ERR_TIMEOUT, and the
device, the plans and the library must stay usable: the next ordinary calls
give the oracle's results.
"""
import numpy as np
import pytest

import oracle
import stencil_inputs as si

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
spider = pytest.importorskip("paper_2506_22035_gb300")
from paper_2506_22035_gb300 import _native  # noqa: E402

SPIDER_ERR_TIMEOUT = 5
DEFAULT_LIMIT = 4_000_000_000


def test_dropped_queue_item_times_out_and_the_device_stays_usable():
    lib = _native.load()
    g = si.rng(70, 0)
    # 200 x 320 points (< 2^16): the persistent queue takes it, 4 x 3 tiles
    # of 62 x 120 per pass of two steps, items 0..11 are pass 0
    u0 = si.grid((200, 320), -1, 1, g)
    w = si.normalised_coeffs(2, 1, "box", si.rng(70, 1))
    steps = 6
    plan = spider.Plan(w, u0.shape, "box", "tf32")
    a = torch.from_numpy(u0).cuda()
    b = torch.full_like(a, float("nan"))
    try:
        _native.check(lib.spider_set_wait_limit(200_000), "spider_set_wait_limit")   # ~0.1 ms
        _native.check(lib.spider_batch_drop_item(5), "spider_batch_drop_item")        # pass 0, tile (2, 1)
        with pytest.raises(spider.SpiderError) as ei:
            spider.batch([plan], [a], [b], [steps])
        assert ei.value.status == SPIDER_ERR_TIMEOUT
    finally:
        _native.check(lib.spider_set_wait_limit(DEFAULT_LIMIT), "spider_set_wait_limit")
    torch.cuda.synchronize()                       # the context is still usable
    ref = oracle.stencil(u0, w, steps)
    # the hook applied to one call: the same batch now completes correctly
    b.fill_(float("nan"))
    spider.batch([plan], [a], [b], [steps])
    torch.cuda.synchronize()
    got = b.cpu().numpy().astype(np.float64)
    assert np.linalg.norm(got - ref) / np.linalg.norm(ref) <= 1e-3
    # and so does an ordinary run of the same plan, bit for bit the batch's
    c = torch.full_like(a, float("nan"))
    plan.run(a, c, steps)
    plan.sync()
    assert torch.equal(b, c)
    plan.close()
