"""GPU accuracy over long runs against the FP64 oracle.

Two things are checked for every arithmetic the library runs (sparse TF32, the
FP16 hi/lo and BF16 hi/mid/lo splits, dense TF32, FP32 on CUDA cores):

* the measured relative L2 error never exceeds the library's own a priori
  bound (spider_plan_error_bound), which the serving loop relies on to pick
  an arithmetic for a job's error target;
* the split precisions meet 1e-5 after 100 steps, the accuracy the
  benchmark's split-precision configurations call for.

The fields are uniform on [0, 1) (one sign: the constant mode dominates, the
worst case for any error in the sum of the weights) and on [-1, 1).  The
benchmark workload itself (Box-2D r = 3, 8192^2, 100 steps) is checked on the
full grid, in the configuration the autotuner picks.
"""
import numpy as np
import pytest

import oracle
import stencil_inputs as si

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
spider = pytest.importorskip("paper_2506_22035_gb300")

ARITHMETIC = [("tf32", "sparse_tc"), ("f16x2", "sparse_tc"), ("bf16x3", "sparse_tc"), ("tf32", "dense_tc"),
              ("tf32", "cuda_core")]
STEPS = (100, 500)

# name -> (extents, radius, shape, field low, field high, seed)
CASES = {
    "2d-star-r1+": ((192, 256), 1, "star", 0.0, 1.0, 60),
    "2d-box-r1+": ((192, 256), 1, "box", 0.0, 1.0, 61),
    "2d-star-r2+": ((192, 256), 2, "star", 0.0, 1.0, 62),
    "2d-box-r2+": ((192, 256), 2, "box", 0.0, 1.0, 63),
    "2d-star-r3+": ((192, 256), 3, "star", 0.0, 1.0, 64),
    "2d-box-r3+": ((192, 256), 3, "box", 0.0, 1.0, 65),
    "2d-box-r3+-": ((192, 256), 3, "box", -1.0, 1.0, 66),
    "3d-star-r1+": ((40, 48, 64), 1, "star", 0.0, 1.0, 67),
    "3d-box-r1+": ((40, 48, 64), 1, "box", 0.0, 1.0, 68),
}


def case_inputs(name):
    ext, r, shape, lo, hi, seed = CASES[name]
    g = si.rng(seed, 0)
    u0 = si.grid(ext, lo, hi, g)
    w = si.normalised_coeffs(len(ext), r, shape, si.rng(seed, 1))
    return u0, w, shape


@pytest.fixture(scope="module")
def references():
    refs = {}
    for name in CASES:
        u0, w, _ = case_inputs(name)
        cur, done = u0, 0
        for n in STEPS:
            cur = oracle.stencil(cur, w, n - done)
            done = n
            refs[(name, n)] = cur
    return refs


def run(u0, w, shape, prec, engine, steps):
    plan = spider.Plan(w, u0.shape, shape, prec, engine)
    a = torch.from_numpy(u0).cuda()
    b = torch.empty_like(a)
    plan.run(a, b, steps)
    plan.sync()
    out = b.cpu().numpy().astype(np.float64)
    return out, plan


@pytest.mark.parametrize("prec,engine", ARITHMETIC)
@pytest.mark.parametrize("name", list(CASES))
def test_error_stays_within_the_a_priori_bound(references, name, prec, engine):
    u0, w, shape = case_inputs(name)
    for n in STEPS:
        got, plan = run(u0, w, shape, prec, engine, n)
        ref = references[(name, n)]
        rel = np.linalg.norm(got - ref) / np.linalg.norm(ref)
        bound = plan.error_bound(n)
        plan.close()
        assert rel <= bound, (name, prec, engine, n, rel, bound)


@pytest.mark.parametrize("prec", ["f16x2", "bf16x3"])
@pytest.mark.parametrize("name", list(CASES))
def test_split_precisions_meet_1e5_after_100_steps(references, name, prec):
    u0, w, shape = case_inputs(name)
    got, plan = run(u0, w, shape, prec, "sparse_tc", 100)
    plan.close()
    ref = references[(name, 100)]
    assert np.linalg.norm(got - ref) / np.linalg.norm(ref) <= 1e-5, (name, prec)


def test_weight_sum_error_is_what_grows():
    # On a field of one sign the error of T steps grows about linearly, by
    # about the weight-sum error per step: sparse TF32 (weights rounded to 11
    # bits, their sum kept as close as the TF32 grid allows) against FP32 on
    # CUDA cores (exact weights), same stencil, 100 and 500 steps.
    u0, w, shape = case_inputs("2d-box-r1+")
    refs = {n: oracle.stencil(u0, w, n) for n in (100, 500)}
    err = {}
    for prec, engine in (("tf32", "sparse_tc"), ("tf32", "cuda_core")):
        for n in (100, 500):
            got, plan = run(u0, w, shape, prec, engine, n)
            plan.close()
            err[(engine, n)] = np.linalg.norm(got - refs[n]) / np.linalg.norm(refs[n])
    assert err[("sparse_tc", 500)] > 2.5 * err[("sparse_tc", 100)]        # grows with the step count
    assert err[("cuda_core", 500)] < 2.0 * err[("cuda_core", 100)] + 1e-8  # exact weights: flat
    assert err[("cuda_core", 500)] < 1e-6


@pytest.fixture(scope="module")
def box2d_reference():
    wl = si.BOX2D_R3_8192
    u0, w = si.workload_inputs(wl)
    ref = oracle.stencil(u0, w, wl.steps)
    return u0, w, torch.from_numpy(ref).cuda()


# full-grid errors measured on GB300 (TF32 3.0e-4, FP16 hi/lo 4.1e-6, BF16
# hi/mid/lo 4.2e-7) and the tolerances, about three times measured
BOX2D_FULL_TOL = {"tf32": 9e-4, "f16x2": 1.2e-5, "bf16x3": 1.3e-6}


@pytest.mark.parametrize("prec", ["tf32", "f16x2", "bf16x3"])
def test_box2d_r3_8192_full_grid_error(box2d_reference, prec):
    # the benchmark workload at full size and step count, autotuned as
    # bench.py runs it; relative L2 error of the whole grid in FP64 on the GPU
    u0, w, ref = box2d_reference
    wl = si.BOX2D_R3_8192
    plan = spider.Plan(w, u0.shape, "box", prec)
    a = torch.from_numpy(u0).cuda()
    b = torch.empty_like(a)
    plan.autotune(a, b, wl.steps)
    plan.run(a, b, wl.steps)
    plan.sync()
    rel = spider.relative_l2_error(b, ref)
    assert rel <= BOX2D_FULL_TOL[prec], (prec, rel)
    assert rel <= plan.error_bound(wl.steps)
    plan.close()


# full-grid errors measured on GB300 (Heat-3D 4.0e-4, Box-3D 1.3e-4 after 50
# steps in TF32) and the tolerances, about three times measured
BOX3D_FULL_TOL = {"heat3d": 1.2e-3, "box3d": 4e-4}


@pytest.mark.parametrize("name", ["heat3d", "box3d"])
def test_3d_512_full_grid_error(name):
    # the 3-D benchmark workloads at full size and step count, autotuned as
    # bench.py runs them; relative L2 error of the whole grid in FP64 on the GPU
    wl = si.HEAT3D_512 if name == "heat3d" else si.BOX3D_512
    u0, w = si.workload_inputs(wl)
    ref = torch.from_numpy(oracle.stencil(u0, w, wl.steps)).cuda()
    plan = spider.Plan(w, u0.shape, wl.shape, "tf32")
    a = torch.from_numpy(u0).cuda()
    b = torch.empty_like(a)
    plan.autotune(a, b, wl.steps)
    plan.run(a, b, wl.steps)
    plan.sync()
    rel = spider.relative_l2_error(b, ref)
    assert rel <= BOX3D_FULL_TOL[name], (name, rel)
    assert rel <= plan.error_bound(wl.steps)
    plan.close()


@pytest.mark.parametrize("target", [1e-2, 1e-5, 1e-6])
def test_autotune_arithmetic_meets_the_error_target(target):
    # the split-depth autotuner: the fastest arithmetic whose a priori bound
    # meets the target; running in it meets the target against the oracle
    g = si.rng(71, 0)
    u0 = si.grid((512, 512), -1, 1, g)
    w = si.normalised_coeffs(2, 2, "box", si.rng(71, 1))
    steps = 50
    plan = spider.Plan(w, u0.shape, "box", "tf32")
    a = torch.from_numpy(u0).cuda()
    b = torch.empty_like(a)
    prec, engine, rate = plan.autotune_arithmetic(a, b, steps, target)
    assert rate > 0
    assert plan.error_bound(steps, prec, engine) <= target
    if target >= 1e-2:
        assert (prec, engine) == ("tf32", "sparse_tc")   # the fastest, and its bound meets 1e-2
    got, chosen = run(u0, w, "box", prec, engine, steps)
    chosen.close()
    ref = oracle.stencil(u0, w, steps)
    assert np.linalg.norm(got - ref) / np.linalg.norm(ref) <= target, (prec, engine)
    with pytest.raises(spider.SpiderError) as e:
        plan.autotune_arithmetic(a, b, steps, 1e-12)         # no arithmetic's bound is that small
    assert e.value.status == 2
    plan.close()


def test_autotune_arithmetic_keeps_large_values_out_of_fp16():
    # values of 2e4 do not fit the FP16 split: a 1e-5 target goes elsewhere
    g = si.rng(72, 0)
    u0 = (si.grid((256, 256), -1, 1, g) * 2e4).astype(np.float32)
    w = si.normalised_coeffs(2, 1, "box", si.rng(72, 1))
    plan = spider.Plan(w, u0.shape, "box", "tf32")
    a = torch.from_numpy(u0).cuda()
    b = torch.empty_like(a)
    prec, engine, _ = plan.autotune_arithmetic(a, b, 20, 1e-5)
    assert prec != "f16x2"
    plan.close()
