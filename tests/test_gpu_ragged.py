"""Runs whose grids TMA cannot read in the caller's layout: rows of
nx % 4 != 0 floats, or buffers that do not start on a 16-byte boundary.
Such runs step through the plan's row-padded grids (every pass after the
first reads through TMA and may fuse time steps); the results must be the
stencil's, bit for bit equal across fusion depths, tile variants and buffer
alignments, and exact against the FP64 oracle on integer inputs."""
import numpy as np
import pytest

import oracle
import stencil_inputs as si

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
spider = pytest.importorskip("paper_2506_22035_gb300")

TF32_TOL = (3e-3, 1e-2)


def offset_copy(a, off):
    """A device copy of `a` starting `off` floats into its allocation."""
    t = torch.from_numpy(np.ascontiguousarray(a, np.float32)).cuda()
    buf = torch.empty(t.numel() + off, dtype=torch.float32, device="cuda")
    v = buf[off:].view(t.shape)
    v.copy_(t)
    return v


def run(u0, w, steps, shape="box", prec="tf32", engine="sparse_tc", T=1, variant=0, off_in=0, off_out=0):
    plan = spider.Plan(w, u0.shape, shape, prec, engine)
    if T > 1:
        plan.set_steps_per_pass(T)
    plan.set_tile_variant(variant)
    a = offset_copy(u0, off_in)
    b = offset_copy(np.full(u0.shape, np.nan, np.float32), off_out)
    plan.run(a, b, steps)
    plan.sync()
    torch.cuda.synchronize()
    out = b.cpu().numpy()
    assert np.array_equal(a.cpu().numpy(), u0)
    plan.close()
    return out


def close(got, ref):
    assert np.all(np.isfinite(got))
    rel = np.linalg.norm(got - ref) / np.linalg.norm(ref)
    mx = np.max(np.abs(got - ref)) / np.max(np.abs(ref))
    assert rel <= TF32_TOL[0] and mx <= TF32_TOL[1], (rel, mx)


@pytest.mark.parametrize("shape,r,steps,T", [((70, 131), 2, 6, 2), ((37, 75), 1, 6, 4), ((64, 130), 3, 5, 3),
                                             ((129, 257), 3, 6, 2), ((9, 10, 71), 1, 5, 2)])
def test_integer_inputs_exact_with_fusion(shape, r, steps, T):
    # three taps of +-1 on values in {-1, 0, 1}: every intermediate is an
    # integer of magnitude <= 3^6 < 2^11, exact in TF32, so every pass, padded
    # or not, fused or not, must reproduce the oracle exactly
    g = np.random.default_rng(sum(shape) + r)
    u = g.integers(-1, 2, size=shape).astype(np.float32)
    w = np.zeros((2 * r + 1,) * len(shape), np.float32)
    taps = g.choice(w.size, size=3, replace=False)
    w.flat[taps] = g.choice([-1.0, 1.0], size=3)
    ref = oracle.stencil(u, w, steps)
    assert np.max(np.abs(ref)) < 2048
    got = run(u, w, steps, T=T)
    assert np.array_equal(got.astype(np.float64), ref)


@pytest.mark.parametrize("shape", [(200, 333), (130, 1001), (96, 258)])
@pytest.mark.parametrize("kind,r", [("box", 3), ("star", 2), ("box", 1)])
def test_ragged_rows_fused_equal_single_step(shape, kind, r):
    g = si.rng(41, r + len(kind))
    u0 = si.grid(shape, -1, 1, g)
    w = si.normalised_coeffs(2, r, kind, g)
    single = run(u0, w, 9, kind, T=1)
    close(single, oracle.stencil(u0, w, 9))
    for T in (2, 3, 4):
        for v in (0, 1, 4):
            assert np.array_equal(run(u0, w, 9, kind, T=T, variant=v), single), (T, v)


@pytest.mark.parametrize("off_in,off_out", [(1, 0), (0, 1), (2, 3), (4, 4)])
def test_unaligned_buffers_equal_aligned(off_in, off_out):
    g = si.rng(42, off_in * 5 + off_out)
    u0 = si.grid((150, 256), -1, 1, g)
    w = si.normalised_coeffs(2, 3, "box", g)
    ref = run(u0, w, 8, T=2)
    got = run(u0, w, 8, T=2, off_in=off_in, off_out=off_out)
    assert np.array_equal(got, ref)
    close(got, oracle.stencil(u0, w, 8))


@pytest.mark.parametrize("key", [("sparse_tc", "f16x2"), ("sparse_tc", "bf16x3"), ("dense_tc", "tf32"),
                                 ("cuda_core", "tf32")])
def test_ragged_rows_other_engines_match_aligned_layout(key):
    # the same grid embedded in a wider, packed one is a different problem;
    # instead: every engine's padded run equals its unfused, unaligned-input
    # run (first pass through the cooperative loader, later passes through
    # TMA), and stays within that engine's error against the oracle
    engine, prec = key
    g = si.rng(43, len(prec))
    u0 = si.grid((90, 203), -1, 1, g)
    w = si.normalised_coeffs(2, 2, "box", g)
    a = run(u0, w, 6, "box", prec, engine, T=2)
    b = run(u0, w, 6, "box", prec, engine, T=1, off_in=1, off_out=1)
    assert np.array_equal(a, b)
    ref = oracle.stencil(u0, w, 6)
    assert np.linalg.norm(a - ref) / np.linalg.norm(ref) < 3e-3


def test_3d_ragged_rows_fused_and_wide_radius():
    g = si.rng(44, 0)
    u0 = si.grid((20, 33, 71), -1, 1, g)
    w = si.normalised_coeffs(3, 1, "star", g)
    single = run(u0, w, 6, "star", T=1)
    close(single, oracle.stencil(u0, w, 6))
    assert np.array_equal(run(u0, w, 6, "star", T=2), single)
    # radius 5 (wide layout, one step per pass) on ragged rows
    u1 = si.grid((80, 203), -1, 1, g)
    w1 = si.normalised_coeffs(2, 5, "box", g)
    close(run(u1, w1, 5), oracle.stencil(u1, w1, 5))


def test_ragged_rows_graph_replay_and_batch_share_padded_grids():
    # repeated runs replay a captured graph that holds the padded grids; a
    # batch call on the same plan uses the same grids in between
    g = si.rng(45, 0)
    u0 = si.grid((100, 199), -1, 1, g)
    w = si.normalised_coeffs(2, 2, "star", g)
    ref = run(u0, w, 7, "star", T=2)
    plan = spider.Plan(w, u0.shape, "star", "tf32")
    plan.set_steps_per_pass(2)
    a = torch.from_numpy(u0).cuda()
    b = torch.empty_like(a)
    for k in range(4):
        b.fill_(float("nan"))
        plan.run(a, b, 7)
        torch.cuda.synchronize()
        assert np.array_equal(b.cpu().numpy(), ref), k
        if k == 1:
            spider.batch([plan], [a], [b], [7])
            torch.cuda.synchronize()
    plan.close()


@pytest.mark.parametrize("n", [3001, 4099, 10245, 130, 7])
@pytest.mark.parametrize("r", [1, 3, 7])
def test_1d_lengths_not_multiple_of_8(n, r):
    # 1-D arrays are read through TMA as rows of 8 floats; other lengths run
    # in the plan's padded arrays (zero tail) after the first pass.  Nine
    # one-step calls never use the padded arrays (a single step reads the
    # caller's array and writes the caller's array): the padded runs must
    # reproduce them bit for bit.
    g = si.rng(46, n % 97 + r)
    u0 = si.grid((n,), -1, 1, g)
    w = si.normalised_coeffs(1, r, "box", g)
    plan = spider.Plan(w, (n,), "box", "tf32")
    a = torch.from_numpy(u0).cuda()
    b = torch.empty_like(a)
    for _ in range(9):
        plan.run(a, b, 1)
        a, b = b, a
    torch.cuda.synchronize()
    chain = a.cpu().numpy()
    plan.close()
    for T in (1, 2, 4):
        assert np.array_equal(run(u0, w, 9, T=T), chain), T
    assert np.array_equal(run(u0, w, 9, T=3, off_in=1, off_out=2), chain)
    if n >= 64:  # a few points of mixed sign cancel: relative error is not TF32's there
        close(chain, oracle.stencil(u0, w, 9))


def test_1d_integer_exact_and_other_engines():
    g = np.random.default_rng(47)
    u = g.integers(-1, 2, size=(5003,)).astype(np.float32)
    w = np.zeros(7, np.float32)
    w[[0, 3, 5]] = [1.0, -1.0, 1.0]
    ref = oracle.stencil(u, w, 6)
    assert np.max(np.abs(ref)) < 2048
    for T in (1, 2, 4):
        assert np.array_equal(run(u, w, 6, T=T).astype(np.float64), ref), T
    for engine, prec in (("cuda_core", "tf32"), ("sparse_tc", "f16x2"), ("dense_tc", "tf32")):
        assert np.array_equal(run(u, w, 6, "box", prec, engine).astype(np.float64), ref), (engine, prec)
