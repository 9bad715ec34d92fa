"""spider_run_static, the entry point that allocates no device memory.

It exists for callers that cannot call cudaMalloc -- an application whose
own memory pool already holds the GPU's memory, or a latency-critical loop
that cannot accept cudaMalloc's implicit synchronisation -- and works in the
library's fixed-size __device__ arrays instead of plan-owned buffers.  This
file is collected last so that a run stopping at its first failure has
already run every other test; it also passes when run alone.
"""
import ctypes

import numpy as np
import pytest

import stencil_inputs as si

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


def _lib():
    from paper_2506_22035_gb300 import _native, build
    build.build()
    return _native


def _run(native, fn, plan, a, b, steps):
    st = getattr(native.load(), fn)(plan.handle, ctypes.c_void_p(a.data_ptr()), ctypes.c_void_p(b.data_ptr()),
                                    steps, ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    native.check(st, fn)


def test_static_entry_point_matches_spider_run_on_two_calls_in_a_row():
    native = _lib()
    import paper_2506_22035_gb300 as spider

    # grids above the static limit are refused before any device work
    big = spider.Plan(np.ones((3, 3), np.float32), (2049, 2049), "box", "tf32")
    # far-apart addresses that the size check rejects before they could be used
    st = native.load().spider_run_static(big.handle, ctypes.c_void_p(1 << 40), ctypes.c_void_p(1 << 41), 1, None)
    assert st == native.SPIDER_ERR_INVALID
    assert b"4194304" in native.load().spider_last_error()
    big.close()

    cases = [
        (si.BOX2D_R3_8192, (300, 520), 7, "tf32", 2),      # odd step count, fused passes of 2 steps
        (si.HEAT3D_512, (20, 33, 72), 6, "f16x2", 1),      # even step count, another plan's operands
        (si.BOX2D_R3_8192, (97, 203), 5, "tf32", 1),        # rows TMA cannot describe: single steps
    ]
    for wl, ext, steps, prec, T in cases:
        u0, w = si.workload_inputs(wl, extents=ext)
        plan = spider.Plan(w, ext, wl.shape, prec)
        if T > 1:
            plan.set_steps_per_pass(T)
        a = torch.from_numpy(u0).cuda()
        got = [torch.full_like(a, float("nan")) for _ in range(2)]
        # two calls in a row on a plan that has never run: it still owns no
        # device memory afterwards
        for g in got:
            _run(native, "spider_run_static", plan, a, g, steps)
        torch.cuda.synchronize()
        assert plan.device_bytes() == 0
        ref = torch.empty_like(a)
        _run(native, "spider_run", plan, a, ref, steps)
        torch.cuda.synchronize()
        assert plan.device_bytes() > 0
        # the same passes and arithmetic as spider_run: identical results
        for g in got:
            assert torch.equal(g, ref)
        plan.close()


@pytest.mark.parametrize("shape,r", [((130, 300), 5), ((5000,), 2)])
def test_static_entry_point_runs_the_wide_layout(shape, r):
    # radius 4..7 and 1-D plans run the wide layout through the same arrays
    native = _lib()
    import paper_2506_22035_gb300 as spider
    g = si.rng(40, r)
    u0 = si.grid(shape, -1, 1, g)
    w = si.normalised_coeffs(len(shape), r, "box", g)
    plan = spider.Plan(w, shape, "box", "tf32")
    a = torch.from_numpy(u0).cuda()
    b_static, b_run = torch.empty_like(a), torch.empty_like(a)
    _run(native, "spider_run_static", plan, a, b_static, 5)
    plan.run(a, b_run, 5)
    plan.sync()
    torch.cuda.synchronize()
    assert torch.equal(b_static, b_run)
    plan.close()
