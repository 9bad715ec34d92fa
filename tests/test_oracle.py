"""Pins for the FP64 oracle (CPU only).

Each test ties the oracle to something other than itself: closed forms,
special cases that reduce to a library routine (scipy.ndimage.correlate,
numpy.diff), invariants of the definition, the paper's worked examples and
Table 2, and brute force on tiny integer inputs.
"""
import os

import numpy as np
import pytest

import oracle
from oracle import cost_model, lowered

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _rand_coeffs(gen, ndim, r):
    return gen.standard_normal((2 * r + 1,) * ndim)


# ----------------------------------------------------------------- definition pins

@pytest.mark.parametrize("ndim,shape", [(1, (37,)), (2, (19, 23)), (3, (7, 9, 11))])
def test_identity_kernel_is_exact_copy(ndim, shape):
    gen = np.random.default_rng(1)
    u = gen.standard_normal(shape)
    for r in (1, 2):
        w = np.zeros((2 * r + 1,) * ndim)
        w[(r,) * ndim] = 1.0
        assert np.array_equal(oracle.stencil(u, w, 3), u)


def test_offcentre_one_is_shift_with_zero_fill():
    # correlation convention u_{t+1}[i] = sum_o w[o] u_t[i+o]: a single 1 at
    # offset (dy, dx) = (+1, -2) reads the point one row below and two left.
    gen = np.random.default_rng(2)
    u = gen.standard_normal((12, 15))
    w = np.zeros((5, 5))
    w[2 + 1, 2 - 2] = 1.0
    got = oracle.stencil(u, w, 1)
    want = np.zeros_like(u)
    want[:-1, 2:] = u[1:, :-2]
    assert np.array_equal(got, want)
    # two steps shift twice, zero-filled
    got2 = oracle.stencil(u, w, 2)
    want2 = np.zeros_like(u)
    want2[:-2, 4:] = u[2:, :-4]
    assert np.array_equal(got2, want2)


def test_1d_second_difference():
    gen = np.random.default_rng(3)
    u = gen.integers(-50, 50, size=64).astype(np.float64)
    got = oracle.stencil(u, np.array([1.0, -2.0, 1.0]), 1)
    want = np.diff(np.pad(u, 1), n=2)          # textbook second difference, zero outside
    assert np.array_equal(got, want)


@pytest.mark.parametrize("ndim,shape,r", [(1, (101,), 3), (2, (33, 29), 1), (2, (40, 37), 3),
                                          (3, (9, 10, 12), 1), (3, (8, 9, 10), 2)])
def test_matches_scipy_correlate(ndim, shape, r):
    scipy_ndimage = pytest.importorskip("scipy.ndimage")
    gen = np.random.default_rng(10 + r + ndim)
    u = gen.standard_normal(shape)
    w = _rand_coeffs(gen, ndim, r)                # non-symmetric: pins sign and axis order
    want = u.copy()
    for _ in range(3):
        want = scipy_ndimage.correlate(want, w, mode="constant", cval=0.0)
    got = oracle.stencil(u, w, 3)
    np.testing.assert_allclose(got, want, rtol=1e-12, atol=1e-12 * np.abs(want).max())


@pytest.mark.parametrize("ndim,shape,r", [(1, (64,), 2), (2, (32, 48), 1), (2, (24, 40), 3), (3, (16, 12, 20), 1)])
def test_fourier_mode_decays_by_symbol(ndim, shape, r):
    # periodic grid, u0 = cos(theta . i): u_t = Re(sigma(theta)^t exp(i theta . i)),
    # sigma(theta) = sum_o w[o] exp(i theta . o)
    gen = np.random.default_rng(20 + ndim + r)
    w = gen.uniform(0, 1, (2 * r + 1,) * ndim)
    w /= w.sum()
    ks = [int(gen.integers(1, 3)) for n in shape]
    theta = [2 * np.pi * k / n for k, n in zip(ks, shape)]
    idx = np.meshgrid(*[np.arange(n) for n in shape], indexing="ij")
    phase = sum(t * i for t, i in zip(theta, idx))
    u0 = np.cos(phase)
    offs = np.meshgrid(*[np.arange(-r, r + 1)] * ndim, indexing="ij")
    sigma = np.sum(w * np.exp(1j * sum(t * o for t, o in zip(theta, offs))))
    steps = 5
    want = np.real(sigma ** steps * np.exp(1j * phase))
    got = oracle.stencil(u0, w, steps, periodic=True)
    # rounding grows with the step count relative to the initial amplitude 1;
    # a dropped or mis-signed term would change sigma by percents
    assert abs(sigma) ** steps > 1e-3
    assert np.max(np.abs(got - want)) <= 1e-13 + 1e-12 * abs(sigma) ** steps


def test_constant_field_preserved_with_dyadic_weights():
    # weights are exact in binary and sum to 1: a constant field stays exactly
    # constant on a periodic grid, and on interior points of a zero-Dirichlet
    # grid farther than steps*r from the boundary.
    w = np.zeros((3, 3))
    w[1, 1] = 0.5
    w[0, 1] = w[2, 1] = w[1, 0] = w[1, 2] = 0.125
    u = np.full((20, 24), 0.75)
    assert np.array_equal(oracle.stencil(u, w, 5, periodic=True), u)
    d = oracle.stencil(u, w, 5)
    assert np.array_equal(d[6:-6, 6:-6], u[6:-6, 6:-6])
    assert d[0, 0] < 0.75                          # the zero halo leaks in at the corner
    w3 = np.zeros((3, 3, 3))
    w3[1, 1, 1] = 0.25
    w3[0, 1, 1] = w3[2, 1, 1] = w3[1, 0, 1] = w3[1, 2, 1] = w3[1, 1, 0] = w3[1, 1, 2] = 0.125
    u3 = np.full((10, 11, 12), -1.5)
    assert np.array_equal(oracle.stencil(u3, w3, 4, periodic=True), u3)


def test_linearity_and_shift_equivariance():
    gen = np.random.default_rng(4)
    w = _rand_coeffs(gen, 2, 2)
    a = gen.standard_normal((18, 21))
    b = gen.standard_normal((18, 21))
    lhs = oracle.stencil(2.0 * a - 3.0 * b, w, 3)
    rhs = 2.0 * oracle.stencil(a, w, 3) - 3.0 * oracle.stencil(b, w, 3)
    np.testing.assert_allclose(lhs, rhs, rtol=1e-12, atol=1e-11)
    shifted = oracle.stencil(np.roll(a, (3, -5), axis=(0, 1)), w, 4, periodic=True)
    assert np.array_equal(shifted, np.roll(oracle.stencil(a, w, 4, periodic=True), (3, -5), axis=(0, 1)))


def test_thread_count_does_not_change_result():
    gen = np.random.default_rng(5)
    u = gen.standard_normal((50, 61))
    w = _rand_coeffs(gen, 2, 3)
    assert np.array_equal(oracle.stencil(u, w, 4, threads=1), oracle.stencil(u, w, 4, threads=4))


@pytest.mark.parametrize("ndim,shape,r,steps", [(2, (90, 100), 3, 5), (3, (30, 31, 33), 1, 6), (1, (500,), 2, 9)])
def test_stencil_points_equal_full_sweep(ndim, shape, r, steps):
    gen = np.random.default_rng(6)
    u = gen.standard_normal(shape).astype(np.float32)
    w = _rand_coeffs(gen, ndim, r).astype(np.float32)
    full = oracle.stencil(u, w, steps)
    pts = [tuple(int(gen.integers(0, n)) for n in shape) for _ in range(12)]
    pts += [tuple(0 for _ in shape), tuple(n - 1 for n in shape)]
    got = oracle.stencil_points(u, w, steps, pts)
    assert np.array_equal(got, np.array([full[p] for p in pts]))


def test_float32_inputs_are_widened_exactly():
    u = np.array([[1.1, 2.2], [3.3, 4.4]], dtype=np.float32)
    w = np.zeros((3, 3), dtype=np.float32)
    w[1, 1] = np.float32(0.1)
    got = oracle.stencil(u, w, 1)
    assert np.array_equal(got, u.astype(np.float64) * np.float64(np.float32(0.1)))


# ------------------------------------------------------------- transform pins (Sec. 3.1)

def test_kernel_matrix_shape_and_padding_r3():
    K = lowered.kernel_matrix(np.arange(1, 8))
    assert K.shape == (8, 14)                      # Sec. 3.1.2: 8 x 14 for r = 3 ...
    assert lowered.pad_kernel_matrix(K).shape == (8, 16)   # ... padded to 8 x 16
    # the kernel row is repeated along the diagonal
    for m in range(8):
        assert list(K[m, m:m + 7]) == list(range(1, 8))
        assert np.count_nonzero(K[m]) == 7


def test_eq1_density_rule():
    for r in range(1, 8):
        for L in range(2, 4 * r + 6):
            assert (lowered.nonzero_fraction(r, L) <= 0.5) == (L >= 2 * r + 2)
        assert lowered.default_L(r) == 2 * r + 2
    assert abs(lowered.nonzero_fraction(3, 8) - 0.5) < 1e-15


@pytest.mark.parametrize("parity", ["even", "odd"])
def test_swap_makes_2_4_and_1_2_for_r_1_to_7(parity):
    for r in range(1, 8):
        K = lowered.pad_kernel_matrix(lowered.kernel_matrix(np.ones(2 * r + 1)))
        L = K.shape[0]
        pi = lowered.strided_swap_permutation(L, parity)
        assert np.array_equal(pi[pi], np.arange(2 * L))      # involution
        assert sorted(pi) == list(range(2 * L))              # permutation
        Ks = lowered.swap_columns(K, pi)
        assert lowered.is_2_4(Ks != 0) and lowered.is_1_2(Ks != 0)
        if r >= 1:
            assert not lowered.is_2_4(K != 0)                 # the banded form is not 2:4


def test_metadata_worked_examples_from_paper():
    rows = [l.split() for l in open(os.path.join(GOLDEN, "metadata_examples.txt"))
            if l.strip() and not l.startswith("#")]
    assert len(rows) == 2
    for group, values, m0, m1 in rows:
        # letters are non-zero placeholders; give each letter a distinct value
        code = {c: float(i + 1) for i, c in enumerate(sorted(set(group) - {"0"}))}
        seg = np.array([[code.get(c, 0.0) for c in group]])
        vals, idx = lowered.compress_2_4(seg)
        inv = {v: k for k, v in code.items()}
        assert "".join(inv.get(v, "0") for v in vals[0]) == values
        assert lowered.metadata_bits(idx[0]) == [f"{m0} {m1}"]


def test_metadata_word_lsb_first():
    idx = np.array([[0, 2], [1, 2], [0, 1], [2, 3]])
    # group g occupies bits 4g..4g+3 with its first index in the low bits
    assert lowered.metadata_word(idx) == (0b1000 | (0b1001 << 4) | (0b0100 << 8) | (0b1110 << 12))


def test_compress_roundtrip_random_2_4_and_1_2():
    gen = np.random.default_rng(7)
    for r in range(1, 8):
        w = gen.integers(-9, 10, size=2 * r + 1)
        w[w == 0] = 1
        Ks = lowered.swapped_kernel_matrix(w.astype(np.int64))
        v, i = lowered.compress_2_4(Ks)
        assert v.shape == (Ks.shape[0], Ks.shape[0])           # L x L value matrix
        assert np.array_equal(lowered.decompress_2_4(v, i), Ks)
        assert np.all(i[..., 0] < i[..., 1])                   # increasing indices
        v1, i1 = lowered.compress_1_2(Ks)
        assert np.array_equal(lowered.decompress_1_2(v1, i1), Ks)


@pytest.mark.parametrize("parity", ["even", "odd"])
@pytest.mark.parametrize("ndim,shape,r", [(1, (29,), 1), (1, (40,), 3), (2, (13, 17), 1),
                                          (2, (12, 21), 2), (2, (11, 19), 3), (3, (5, 6, 13), 1)])
def test_lowered_products_equal_direct_sweep_bit_exact(parity, ndim, shape, r):
    # small integers keep every intermediate exact: the dense banded product,
    # the swapped 2:4 product and the direct sweep must agree bit for bit,
    # which shows the swap is a pure permutation (Sec. 3.2).
    gen = np.random.default_rng(8 + r)
    u = gen.integers(-1, 2, size=shape).astype(np.int64)
    w = gen.integers(-1, 2, size=(2 * r + 1,) * ndim).astype(np.int64)
    steps = 3
    direct = oracle.stencil(u, w, steps)
    dense = lowered.lowered_stencil(u, w, steps, "dense")
    swapped = lowered.lowered_stencil(u, w, steps, "swapped", parity)
    assert np.array_equal(dense, swapped)
    assert np.array_equal(dense.astype(np.float64), direct)


# -------------------------------------------------------------------- cost model pins

def test_table2_costs():
    rows = {l.split()[0]: [float(x) for x in l.split()[1:]]
            for l in open(os.path.join(GOLDEN, "table2_box2d3r_c8.txt")) if l.strip() and not l.startswith("#")}
    lb = cost_model.lower_bound(3, 8)
    np.testing.assert_allclose(lb, rows["LowerBound"], atol=0.006)
    comp, inp, par = cost_model.spider_costs(3, 8, ceil_compute=False)
    assert (comp, inp, par) == tuple(rows["SPIDER"])
    assert comp == (2 * 3 + 1) * (2 * 3 + 2)                   # (2r+1)(2r+2) MACs per point
    assert cost_model.spider_costs(3, 8)[0] == 64              # with the ceiling kept
