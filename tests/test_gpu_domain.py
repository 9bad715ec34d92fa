"""GPU: a grid cut into slabs with ghost planes (spider_domain_*) gives the
undivided run's result bit for bit, and matches the FP64 oracle.

Each slab runs E steps on its owned planes plus g >= E r ghost planes per
interior side; the ghost planes go wrong from the outside in at r planes per
step, so the owned planes stay exact, and the exchange refreshes the ghosts.
Every owned point is computed with the same products in the same order as
in the undivided grid, hence the bit-for-bit comparison."""
import numpy as np
import pytest

import oracle
import stencil_inputs as si

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
spider = pytest.importorskip("paper_2506_22035_gb300")


def _run_both(u0, w, steps, shape, prec, engine, T, parts, E):
    plan = spider.Plan(w, u0.shape, shape, prec, engine)
    plan.set_steps_per_pass(T)
    a = torch.from_numpy(np.ascontiguousarray(u0, np.float32)).cuda()
    whole = torch.full_like(a, float("nan"))
    plan.run(a, whole, steps)
    plan.sync()
    dom = spider.Domain(plan, parts, E)
    split = torch.full_like(a, float("nan"))
    dom.run(a, split, steps)
    dom.sync()
    torch.cuda.synchronize()
    assert np.array_equal(a.cpu().numpy(), u0)  # input preserved
    layout = [dom.slab(i) for i in range(parts)]
    dom.close()
    plan.close()
    return whole.cpu().numpy(), split.cpu().numpy(), layout


@pytest.mark.parametrize("shape,r,prec,engine,T,parts,E,steps", [
    ((300, 520), 3, "tf32", "sparse_tc", 2, 3, 2, 9),       # fused passes, one pass per period
    ((300, 520), 3, "tf32", "sparse_tc", 2, 2, 4, 9),       # two fused passes per period
    ((301, 517), 2, "tf32", "sparse_tc", 1, 4, 3, 10),      # unaligned rows (no TMA)
    ((256, 384), 1, "f16x2", "sparse_tc", 1, 2, 3, 7),      # odd ghost depth rounded to a row pair
    ((256, 384), 3, "bf16x3", "sparse_tc", 2, 3, 2, 6),
    ((200, 264), 2, "tf32", "dense_tc", 2, 2, 2, 5),
    ((200, 264), 1, "tf32", "cuda_core", 1, 3, 2, 5),
    ((4000,), 2, "tf32", "sparse_tc", 1, 3, 3, 8),          # 1-D, x slabs on 8-point segments
    ((4000,), 6, "tf32", "sparse_tc", 1, 3, 2, 5),          # 1-D radius 6: 16-point segments
    ((300, 264), 5, "tf32", "sparse_tc", 1, 2, 2, 5),       # 2-D radius 5
    ((24, 40, 72), 1, "tf32", "sparse_tc", 1, 2, 2, 5),     # 3-D z slabs, z-streaming kernel
    ((40, 24, 72), 1, "tf32", "sparse_tc", 2, 2, 2, 7),     # 3-D fused passes
    ((20, 33, 70), 2, "f16x2", "sparse_tc", 1, 2, 1, 3),    # 3-D, unaligned rows
])
def test_domain_run_equals_undivided_run(shape, r, prec, engine, T, parts, E, steps):
    g = si.rng(13, r + 10 * len(shape))
    u0 = si.grid(shape, -1, 1, g)
    w = si.normalised_coeffs(len(shape), r, "box", g)
    whole, split, layout = _run_both(u0, w, steps, "box", prec, engine, T, parts, E)
    assert np.all(np.isfinite(split))
    assert np.array_equal(split, whole), (shape, prec, engine, layout)
    # several exchanges happened and the slabs really overlap
    assert steps > E and all(lo + hi > 0 for _, _, lo, hi in layout)
    ref = oracle.stencil(u0, w, steps)
    rel = np.linalg.norm(split - ref) / np.linalg.norm(ref)
    tol = 2e-6 if engine == "cuda_core" else {"tf32": 3e-3, "f16x2": 2e-5, "bf16x3": 2e-4}[prec]
    assert rel <= tol, rel


def test_domain_zero_steps_and_star_stencil():
    g = si.rng(13, 99)
    u0 = si.grid((128, 256), 0, 1, g)
    w = si.normalised_coeffs(2, 1, "star", g)
    whole, split, _ = _run_both(u0, w, 0, "star", "tf32", "sparse_tc", 1, 2, 1)
    assert np.array_equal(split, u0) and np.array_equal(whole, u0)
    whole, split, _ = _run_both(u0, w, 11, "star", "tf32", "sparse_tc", 4, 3, 4)
    assert np.array_equal(split, whole)
