"""CPU-only checks of the C-ABI library: it loads, exports every entry point
declared in include/spider.h, validates its arguments, and its host-side plan
(the offline transform of Sec. 3.1 and the fragment packing of Sec. 3.3.2)
packs operands that decode back to the stencil's banded kernel matrices.

No compute call is made here (plan creation touches no device)."""
import ctypes
import os
import re

import numpy as np
import pytest

import paper_2506_22035_gb300 as spider
from paper_2506_22035_gb300 import _native, build

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    build.build()
    return _native.load()


def declared_entry_points():
    names = set()
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if fn.endswith(".h"):
            src = open(os.path.join(ROOT, "include", fn)).read()
            src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
            names |= set(re.findall(r"\b(spider_[a-z0-9_]+)\s*\(", src))
    return names


def test_every_declared_symbol_is_exported(lib):
    names = declared_entry_points()
    assert {"spider_plan_create", "spider_run", "spider_batch", "spider_submit"} <= names
    for n in names:
        assert hasattr(lib, n), n
    # the binding declares exactly the header's entry points
    assert set(_native.SIGNATURES) == names


def _create(lib, ndim, ext, shape, r, coeffs, prec=0):
    h = ctypes.c_void_p()
    w = np.ascontiguousarray(coeffs, dtype=np.float32)
    st = lib.spider_plan_create(ndim, (ctypes.c_int64 * max(1, len(ext)))(*ext), shape, r,
                                w.ctypes.data_as(ctypes.POINTER(ctypes.c_float)), prec, ctypes.byref(h))
    if st == 0:
        lib.spider_plan_destroy(h)
    return st


def test_plan_argument_validation(lib):
    ok = np.ones((3, 3), np.float32)
    assert _create(lib, 2, (16, 16), 1, 1, ok) == _native.SPIDER_OK
    assert _create(lib, 4, (16, 16), 1, 1, ok) == _native.SPIDER_ERR_INVALID
    assert _create(lib, 2, (0, 16), 1, 1, ok) == _native.SPIDER_ERR_INVALID
    assert _create(lib, 2, (16, 16), 1, 0, ok) == _native.SPIDER_ERR_INVALID
    assert _create(lib, 2, (16, 16), 1, 4, np.ones((9, 9), np.float32)) == _native.SPIDER_OK  # wide layout
    assert _create(lib, 2, (16, 16), 1, 8, np.ones((17, 17), np.float32)) == _native.SPIDER_ERR_UNSUPPORTED
    bad = ok.copy()
    bad[0, 0] = np.nan
    assert _create(lib, 2, (16, 16), 1, 1, bad) == _native.SPIDER_ERR_INVALID
    # a star stencil may not carry off-axis coefficients
    assert _create(lib, 2, (16, 16), 0, 1, ok) == _native.SPIDER_ERR_INVALID
    star = np.zeros((3, 3), np.float32)
    star[1, :] = 1
    star[:, 1] = 1
    assert _create(lib, 2, (16, 16), 0, 1, star) == _native.SPIDER_OK
    assert lib.spider_plan_create(2, None, 1, 1, None, 0, None) == _native.SPIDER_ERR_INVALID
    assert b"NULL" in lib.spider_last_error()


def test_run_rejects_bad_arguments_without_touching_a_device(lib):
    p = spider.Plan(np.ones((3, 3), np.float32), (8, 8))
    assert lib.spider_run(p.handle, None, None, 1, None) == _native.SPIDER_ERR_INVALID
    assert lib.spider_run(p.handle, ctypes.c_void_p(4096), ctypes.c_void_p(4096 + 16), 1, None) == \
        _native.SPIDER_ERR_INVALID                                   # overlapping grids
    assert lib.spider_run(p.handle, ctypes.c_void_p(4096), ctypes.c_void_p(1 << 20), -1, None) == \
        _native.SPIDER_ERR_INVALID
    assert lib.spider_plan_set_steps_per_pass(p.handle, 0) == _native.SPIDER_ERR_INVALID
    assert lib.spider_plan_set_steps_per_pass(p.handle, 11) == _native.SPIDER_ERR_UNSUPPORTED
    assert lib.spider_plan_set_steps_per_pass(p.handle, 10) == _native.SPIDER_OK   # radius 1: deep tiles
    assert lib.spider_plan_set_steps_per_pass(p.handle, 3) == _native.SPIDER_OK
    assert lib.spider_plan_set_tile_variant(p.handle, 6) == _native.SPIDER_ERR_INVALID
    assert lib.spider_plan_set_tile_variant(p.handle, 5) == _native.SPIDER_OK
    assert lib.spider_plan_set_tile_variant(p.handle, 4) == _native.SPIDER_OK
    assert lib.spider_plan_set_tile_variant(p.handle, 1) == _native.SPIDER_OK
    assert lib.spider_plan_autotune(p.handle, None, None, 1, None, None, None) == _native.SPIDER_ERR_INVALID
    p.close()
    p3 = spider.Plan(np.ones((5, 5, 5), np.float32), (8, 8, 8))  # 3-D fusion is built for r = 1 only
    assert lib.spider_plan_set_steps_per_pass(p3.handle, 2) == _native.SPIDER_ERR_UNSUPPORTED
    p3.close()


def test_failure_hooks_validate_their_arguments(lib):
    assert lib.spider_set_wait_limit(999) == _native.SPIDER_ERR_INVALID
    assert lib.spider_batch_drop_item(-2) == _native.SPIDER_ERR_INVALID
    assert lib.spider_batch_drop_item(-1) == 0


def test_error_bound_model(lib):
    # bound = steps * (weight-sum error + drift) + floor, per arithmetic;
    # radius 4..7 has no split or comparator kernel
    w = si_coeffs(2, 2)
    p = spider.Plan(w, (64, 64), "box", "tf32")
    b = {k: [p.error_bound(n, *k) for n in (0, 100, 200)] for k in
         (("tf32", "sparse_tc"), ("f16x2", "sparse_tc"), ("bf16x3", "sparse_tc"), ("tf32", "cuda_core"))}
    for v in b.values():
        assert 0 < v[0] < v[1] < v[2]
        assert abs((v[2] - v[1]) - (v[1] - v[0])) <= 1e-12 * v[2]     # linear in the step count
    assert b[("tf32", "cuda_core")][2] < b[("f16x2", "sparse_tc")][2] < b[("tf32", "sparse_tc")][2]
    with pytest.raises(spider.SpiderError):
        p.error_bound(-1)
    p.close()
    wide = spider.Plan(si_coeffs(2, 6), (64, 64), "box", "tf32")
    assert wide.error_bound(10) > 0
    for k in (("f16x2", "sparse_tc"), ("tf32", "cuda_core"), ("tf32", "dense_tc")):
        with pytest.raises(spider.SpiderError) as ei:
            wide.error_bound(10, *k)
        assert ei.value.status == 2
    wide.close()


def si_coeffs(ndim, r):
    import stencil_inputs as si
    return si.normalised_coeffs(ndim, r, "box", si.rng(80, r))


def test_plan_owns_no_device_memory_before_its_first_run(lib):
    p = spider.Plan(si_coeffs(2, 1), (64, 64), "box", "tf32")
    assert p.device_bytes() == 0
    p.close()


def test_batch_rejects_bad_arguments_without_touching_a_device(lib):
    # every case fails in the argument checks, before any device call
    a = spider.Plan(np.ones((3, 3), np.float32), (8, 8))
    b = spider.Plan(np.ones((3, 3), np.float32), (8, 8))
    P = lambda *h: (ctypes.c_void_p * len(h))(*h)
    S = lambda *n: (ctypes.c_int64 * len(n))(*n)
    ok_in, ok_out = P(4096, 1 << 20), P(1 << 21, 1 << 22)
    assert lib.spider_batch(-1, P(a.handle), P(4096), P(1 << 20), S(1), None) == _native.SPIDER_ERR_INVALID
    assert lib.spider_batch(5000, P(a.handle), P(4096), P(1 << 20), S(1), None) == _native.SPIDER_ERR_INVALID
    assert lib.spider_batch(0, None, None, None, None, None) == _native.SPIDER_OK      # nothing to do
    assert lib.spider_batch(1, None, P(4096), P(1 << 20), S(1), None) == _native.SPIDER_ERR_INVALID
    assert lib.spider_batch(1, P(a.handle), P(4096), P(1 << 20), S(-1), None) == _native.SPIDER_ERR_INVALID
    assert lib.spider_batch(1, P(a.handle), P(4096), P(4096 + 16), S(1), None) == _native.SPIDER_ERR_INVALID
    assert lib.spider_batch(1, P(None), P(4096), P(1 << 20), S(1), None) == _native.SPIDER_ERR_INVALID
    # a plan owns its scratch grids: it may appear once per batch
    assert lib.spider_batch(2, P(a.handle, a.handle), ok_in, ok_out, S(1, 1), None) == _native.SPIDER_ERR_INVALID
    assert "once" in lib.spider_last_error().decode()
    a.close()
    b.close()


# ------------------------------------------------------------------ operand decoding
# Decoding uses the fragment maps of the sparse TF32 m16n8k16 MMA (measured on
# the device): A compressed 16 x 8 with a0 (g, q), a1 (g+8, q), a2 (g, q+4),
# a3 (g+8, q+4); metadata in lanes q in {0,1}: nibble i of the low half is row
# g, pair 4q+i, of the high half row g+8; 0x4 keeps the first element of the
# pair, 0xE the second.  MMA K-index k sits at window position
# 4*sigma(k % 4) + k // 4 with sigma = (0, 2, 1, 3).

SIGMA = (0, 2, 1, 3)


def phi(k):
    return 4 * SIGMA[k % 4] + k // 4


def decode_tf32(words, meta):
    """16 x 16 window matrix from one A operand (words: 32 x 4, meta: 32)."""
    comp = np.zeros((16, 8), np.float32)
    idx = np.full((16, 8), -1)
    for lane in range(32):
        g, q = divmod(lane, 4)
        vals = words[lane].view(np.float32)
        comp[g, q], comp[g + 8, q], comp[g, q + 4], comp[g + 8, q + 4] = vals
        if q < 2:
            for i in range(4):
                for half, row in ((0, g), (16, g + 8)):
                    nib = (int(meta[lane]) >> (half + 4 * i)) & 0xF
                    assert nib in (0x4, 0xE)
                    idx[row, 4 * q + i] = 0 if nib == 0x4 else 1
    assert (idx >= 0).all()
    A = np.zeros((16, 16), np.float32)
    for m in range(16):
        for c in range(8):
            A[m, phi(2 * c + idx[m, c])] += comp[m, c]
    return A


def expected_window(w, a, ry, rx, dz_index=0):
    """Row m = (s, xo): output row y+s, x offset xo; column p: input x0-4+p;
    input row j = y + a - ry.  Entry w[dz][j - (y+s)][p - 4 - xo]."""
    A = np.zeros((16, 16), np.float64)
    for m in range(16):
        s, xo = divmod(m, 8)
        dy = a - ry - s
        for p in range(16):
            dx = p - 4 - xo
            if abs(dy) <= ry and abs(dx) <= rx:
                A[m, p] = w[dz_index][dy + ry][dx + rx]
    return A


def tf32(x):
    b = np.asarray(x, np.float32).view(np.uint32).astype(np.uint64)
    b = ((b + 0x1000) & 0xFFFFE000).astype(np.uint32)
    return b.view(np.float32)


@pytest.mark.parametrize("ndim,r", [(2, 1), (2, 2), (2, 3), (3, 1), (3, 2)])
def test_tf32_operands_decode_to_banded_kernel_rows(ndim, r):
    gen = np.random.default_rng(100 + r)
    w = gen.standard_normal((2 * r + 1,) * ndim).astype(np.float32)
    p = spider.Plan(w, (8,) * ndim, "box", "tf32")
    words, meta = p.operands()
    ry = r if ndim >= 2 else 0
    rz = r if ndim == 3 else 0
    w3 = w.reshape((2 * rz + 1, 2 * ry + 1, 2 * r + 1))
    na = 2 * ry + 2
    assert words.size == (2 * rz + 1) * na * 128 and meta.size == (2 * rz + 1) * na * 32
    words = words.reshape(-1, 32, 4)
    meta = meta.reshape(-1, 32)
    # the TF32 weights the plan used: read back from the top half of each A
    # (row m = 0: output x0, window position 4 + dx holds w[dz][a - ry][dx])
    used = np.zeros_like(w3)
    for dzi in range(2 * rz + 1):
        for a in range(2 * ry + 1):
            used[dzi, a] = decode_tf32(words[dzi * na + a], meta[dzi * na + a])[0, 4 - r:5 + r]
    # every window matrix is the banded kernel of those weights
    for dzi in range(2 * rz + 1):
        for a in range(na):
            got = decode_tf32(words[dzi * na + a], meta[dzi * na + a])
            assert np.array_equal(got, expected_window(used, a, ry, r, dzi).astype(np.float32)), (dzi, a)
    # each weight is one of its two TF32 neighbours, and the rounded weights
    # sum at least as close to the FP32 sum as round-to-nearest does
    bits = w3.view(np.uint32) & np.uint32(0xFFFFE000)
    lo = bits.view(np.float32)
    hi = (bits + np.uint32(0x2000)).view(np.float32)
    assert np.all((used == lo) | (used == hi))
    true_sum = w3.astype(np.float64).sum()
    assert abs(used.astype(np.float64).sum() - true_sum) <= abs(tf32(w3).astype(np.float64).sum() - true_sum)
    p.close()


def test_tf32_sum_preserving_rounding_keeps_exact_weights():
    w = np.zeros((3, 3), np.float32)
    w[1, 1], w[0, 1], w[2, 1], w[1, 0], w[1, 2] = 0.5, 0.125, 0.125, 0.125, 0.125
    p = spider.Plan(w, (16, 16), "star", "tf32")
    words, meta = p.operands()
    top = decode_tf32(words.reshape(-1, 32, 4)[1], meta.reshape(-1, 32)[1])
    assert np.array_equal(top[0, 3:6], w[1])
    p.close()


def test_window_matrices_are_the_papers_banded_K():
    # The 8 x 16 half of a window matrix for one kernel row is the paper's
    # banded K (Sec. 3.1.1) for L = 8 outputs shifted into the 16-wide window:
    # K[m][n] = w[n - m] for 0 <= n - m <= 2r, placed at window column n + 4 - r.
    from oracle import lowered
    for r in (1, 2, 3):
        w_row = np.arange(1, 2 * r + 2, dtype=np.float64)
        K = lowered.kernel_matrix(w_row, L=8)              # 8 x (2r + 8)
        win = expected_window(w_row.reshape(1, 1, -1), 0, 0, r)[:8]
        assert np.array_equal(win[:, 4 - r:4 - r + K.shape[1]], K)
        assert np.count_nonzero(win) == np.count_nonzero(K)


def test_fragment_permutation_is_a_strided_swap_giving_1_2_and_2_4():
    # the permutation places the members of every 1:2 pair 8 window positions
    # apart; with a band of 2r+1 <= 7 positions the permuted K is 1:2 and 2:4
    from oracle import lowered
    perm = np.array([phi(k) for k in range(16)])
    assert sorted(perm) == list(range(16))
    for c in range(8):
        assert abs(perm[2 * c] - perm[2 * c + 1]) == 8
    for r in (1, 2, 3):
        band = expected_window(np.ones((1, 1, 2 * r + 1)), 0, 0, r)[:8] != 0
        permuted = band[:, perm]
        assert lowered.is_1_2(permuted) and lowered.is_2_4(permuted)
        assert not lowered.is_2_4(band)


@pytest.mark.parametrize("prec", ["f16x2", "bf16x3"])
def test_split_operands_have_expected_layout(prec):
    w = np.random.default_rng(3).uniform(0, 1, (7, 7)).astype(np.float32)
    w /= w.sum()
    p = spider.Plan(w, (16, 16), "box", prec)
    words, meta = p.operands()
    passes = 2 if prec == "bf16x3" else 1
    combos = passes * ((3 + 1) + 8)         # per pass: (ry+1) two-row combos + (2ry+2) one-row combos
    assert words.size == combos * 128 and meta.size == combos * 32
    # metadata nibbles: two increasing 2-bit indices per group, lanes q >= 2 unused
    m = meta.reshape(combos, 32)
    for c in range(combos):
        for lane in range(32):
            if lane % 4 >= 2:
                assert m[c, lane] == 0
                continue
            for k in range(8):
                nib = (int(m[c, lane]) >> (4 * k)) & 0xF
                assert (nib & 3) < (nib >> 2)
    p.close()


def b_fragment_rows():
    """Sec. 3.2's row-offset equation for a 16-bit B fragment (golden fixture):
    rows[q][i] = K row of element i held by lanes with lane mod 4 = q."""
    path = os.path.join(ROOT, "tests", "golden", "b_fragment_rows_m16n8k16.txt")
    rows = {}
    for line in open(path):
        if line.strip() and not line.startswith("#"):
            f = [int(x) for x in line.split()]
            rows[f[0]] = f[1:]
    return rows


def bits16_to_f32(u, bf16):
    u = np.asarray(u, np.uint16)
    if bf16:
        return (u.astype(np.uint32) << 16).view(np.float32)
    return u.view(np.float16).astype(np.float32)


def rn16(x, bf16):
    """Round float32 to FP16 / BF16 (nearest, ties to even), as float32."""
    x = np.asarray(x, np.float32)
    if not bf16:
        return x.astype(np.float16).astype(np.float32)
    b = x.view(np.uint32).astype(np.uint64)
    b = (b + 0x7FFF + ((b >> 16) & 1)) & 0xFFFF0000
    return b.astype(np.uint32).view(np.float32)


def decode_16bit_k32(words, meta, bf16):
    """One packed m16n8k32 A operand -> the two 16 x 16 window matrices it
    multiplies (K half 0, K half 1).  Values and metadata decode to a 16 x 32
    matrix in MMA K order (group c of 4 K indices, nibble = idx0 | idx1 << 2);
    K row -> window position follows the kernel's loads: lane q loads window
    positions 4 sigma(q) + i (i = 0..3) and hands element i to the K row the
    paper's B-fragment equation gives (plus 16 for the second half)."""
    comp = np.zeros((16, 16), np.float32)
    for lane in range(32):
        g, q = divmod(lane, 4)
        wv = words[lane]
        for reg, (row, col) in enumerate(((g, 2 * q), (g + 8, 2 * q), (g, 2 * q + 8), (g + 8, 2 * q + 8))):
            comp[row, col] = bits16_to_f32(int(wv[reg]) & 0xFFFF, bf16)
            comp[row, col + 1] = bits16_to_f32(int(wv[reg]) >> 16, bf16)
    K = np.zeros((16, 32), np.float32)
    for lane in range(32):
        g, q = divmod(lane, 4)
        if q >= 2:
            continue
        for i in range(4):
            grp = 4 * q + i
            for half, row in ((0, g), (16, g + 8)):
                nib = (int(meta[lane]) >> (half + 4 * i)) & 0xF
                idx = (nib & 3, nib >> 2)
                for s in range(2):
                    K[row, 4 * grp + idx[s]] += comp[row, 2 * grp + s]
    rows = b_fragment_rows()
    H = np.zeros((2, 16, 16), np.float32)
    for h in range(2):
        for q in range(4):
            for i in range(4):
                H[h][:, 4 * SIGMA[q] + i] = K[:, 16 * h + rows[q][i]]
    return H


@pytest.mark.parametrize("prec", ["f16x2", "bf16x3"])
@pytest.mark.parametrize("ndim,r", [(2, 1), (2, 3), (3, 1)])
def test_split_operands_decode_to_sum_preserving_split_weights(prec, ndim, r):
    bf16 = prec == "bf16x3"
    gen = np.random.default_rng(200 + 10 * ndim + r)
    w = gen.uniform(0, 1, (2 * r + 1,) * ndim)
    w = (w / w.sum()).astype(np.float32)
    p = spider.Plan(w, (8,) * ndim, "box", prec)
    words, meta = p.operands()
    ry = r if ndim >= 2 else 0
    rz = r if ndim == 3 else 0
    na = 2 * ry + 2
    per_pass = (ry + 1) + na
    passes = 2 if bf16 else 1
    cpp = passes * per_pass
    planes = 2 * rz + 1
    assert words.size == planes * cpp * 128 and meta.size == planes * cpp * 32
    words = words.reshape(-1, 32, 4)
    meta = meta.reshape(-1, 32)
    w3 = w.reshape((planes, 2 * ry + 1, 2 * r + 1))
    dec = lambda c: decode_16bit_k32(words[c], meta[c], bf16)  # noqa: E731
    # split terms read back from the top row of the one-row combos
    # [K_hi(a) | K_y(a)] of each pass (a = 0 .. 2ry): y = lo (FP16), mid then lo (BF16)
    hi = np.zeros_like(w3)
    ys = [np.zeros_like(w3) for _ in range(passes)]
    for dzi in range(planes):
        for pz in range(passes):
            for a in range(2 * ry + 1):
                Hh = dec(dzi * cpp + pz * per_pass + (ry + 1) + a)
                hi[dzi, a] = Hh[0][0, 4 - r:5 + r]
                ys[pz][dzi, a] = Hh[1][0, 4 - r:5 + r]
    two_row_terms = [hi] + ([ys[0]] if bf16 else [])  # pass 0: hi, BF16 pass 1: mid
    for dzi in range(planes):
        for pz in range(passes):
            for c in range(ry + 1):
                Hh = dec(dzi * cpp + pz * per_pass + c)
                for h in range(2):
                    exp = expected_window(two_row_terms[pz], 2 * c + h, ry, r, dzi).astype(np.float32)
                    assert np.array_equal(Hh[h], exp), (dzi, pz, c, h)
            for a in range(na):
                Hh = dec(dzi * cpp + pz * per_pass + (ry + 1) + a)
                assert np.array_equal(Hh[0], expected_window(hi, a, ry, r, dzi).astype(np.float32))
                assert np.array_equal(Hh[1], expected_window(ys[pz], a, ry, r, dzi).astype(np.float32))
    # hi (and BF16 mid) round to nearest; the last term is one of the two
    # 16-bit neighbours of what is left, chosen so the split weights sum at
    # least as close to the FP32 sum as rounding every term to nearest
    assert np.array_equal(hi, rn16(w3, bf16))
    if bf16:
        mid, lo, scale = ys[0], ys[1], 1.0
        assert np.array_equal(mid, rn16(w3 - hi, bf16))
        rest = w3 - hi - mid
    else:
        mid, lo, scale = np.zeros_like(hi), ys[0], 1.0 / 2048
        rest = (w3 - hi) * np.float32(2048)
    rn = rn16(rest, bf16)
    ulp_rn = np.abs(rn16(rn * np.float32(1 + 2 ** -6), bf16) - rn)   # spacing near each residual
    assert np.all(np.abs(lo.astype(np.float64) - rest) <= np.maximum(ulp_rn, 2.0 ** -133) * 1.0001)
    true_sum = w3.astype(np.float64).sum()
    split = lambda last: (hi.astype(np.float64) + mid + scale * last.astype(np.float64)).sum()  # noqa: E731
    assert abs(split(lo) - true_sum) <= abs(split(rn) - true_sum)
    assert abs(split(lo) - true_sum) <= scale * float(ulp_rn.max())
    p.close()


def _slabs(dom):
    return [dom.slab(i) for i in range(dom.parts)]


@pytest.mark.parametrize("extents,r,E,parts,align", [((300, 520), 3, 2, 3, 2), ((301, 64), 1, 3, 4, 2),
                                                      ((1000,), 2, 1, 3, 16), ((20, 33, 70), 1, 3, 2, 1),
                                                      ((64, 64), 2, 4, 1, 2)])
def test_domain_layout(lib, extents, r, E, parts, align):
    # host logic of the slab decomposition: owned ranges tile the slowest
    # axis, ghost depth >= E * r rounded up to the tile alignment, boundaries
    # on that alignment, and each ghost region lies inside the neighbour
    nd = len(extents)
    plan = spider.Plan(np.full((2 * r + 1,) * nd, 1.0 / (2 * r + 1) ** nd, np.float32), extents, "box")
    plan.set_steps_per_pass(1)
    dom = spider.Domain(plan, parts, E)
    slabs = _slabs(dom)
    g = 0 if parts == 1 else -(-E * r // align) * align
    nxt = 0
    for i, (first, owned, glo, ghi) in enumerate(slabs):
        assert first == nxt and owned >= max(1, g)
        assert first % align == 0
        assert glo == (g if i > 0 else 0) and ghi == (g if i + 1 < parts else 0)
        nxt = first + owned
    assert nxt == extents[0]
    dom.close()
    plan.close()


def test_domain_argument_validation(lib):
    w = np.full((7, 7), 1 / 49, np.float32)
    plan = spider.Plan(w, (10, 64), "box")
    with pytest.raises(spider.SpiderError) as e:
        spider.Domain(plan, 2, 4)            # ghost depth 12 > 5 owned planes
    assert e.value.status == _native.SPIDER_ERR_INVALID
    for parts, E in ((0, 1), (11, 1), (2, -1)):
        with pytest.raises(spider.SpiderError):
            spider.Domain(plan, parts, E)
    h = ctypes.c_void_p()
    assert lib.spider_domain_create(None, 2, 1, ctypes.byref(h)) == _native.SPIDER_ERR_INVALID
    dom = spider.Domain(plan, 1, 4)          # one slab: no ghost planes needed
    assert dom.slab(0) == (0, 10, 0, 0)
    with pytest.raises(spider.SpiderError):
        dom.slab(1)
    dom.close()
    plan.close()


def test_steps_per_pass_where_fusion_is_built(lib):
    # fused passes exist for 2-D stencils of radius 1..3, and for 3-D radius-1
    # and 1-D sparse TF32 plans
    def plan(nd, r, prec="tf32"):
        return spider.Plan(np.full((2 * r + 1,) * nd, 0.1, np.float32), (16,) * nd, "box", prec)
    for nd, r, prec, ok in ((2, 3, "tf32", True), (2, 1, "f16x2", True), (3, 1, "tf32", True),
                            (3, 2, "tf32", False), (3, 1, "f16x2", False), (1, 1, "tf32", True),
                            (1, 7, "tf32", True), (1, 2, "f16x2", False), (2, 5, "tf32", False)):
        p = plan(nd, r, prec)
        for T in (2, 4):
            if ok:
                p.set_steps_per_pass(T)
            else:
                with pytest.raises(spider.SpiderError) as e:
                    p.set_steps_per_pass(T)
                assert e.value.status == _native.SPIDER_ERR_UNSUPPORTED
        with pytest.raises(spider.SpiderError):
            p.set_steps_per_pass(5)  # deep tiles (5..10) are built for radius 1
        p.close()
    p = plan(3, 1)
    p.set_engine("dense_tc")
    with pytest.raises(spider.SpiderError):
        p.set_steps_per_pass(2)
    p.close()


def phi_wide(h, k):
    """Wide layout (radius 4..7): window position of K index k in K half h;
    the 1:2 pair (2c, 2c+1) lands on positions p and p + 16."""
    return 8 * h + 4 * ((k % 4) >> 1) + 16 * ((k % 4) & 1) + k // 4


def decode_k_order(words, meta):
    """16 x 16 matrix in MMA K order from one sparse TF32 A operand."""
    comp = np.zeros((16, 8), np.float32)
    idx = np.full((16, 8), -1)
    for lane in range(32):
        g, q = divmod(lane, 4)
        comp[g, q], comp[g + 8, q], comp[g, q + 4], comp[g + 8, q + 4] = words[lane].view(np.float32)
        if q < 2:
            for i in range(4):
                for half, row in ((0, g), (16, g + 8)):
                    nib = (int(meta[lane]) >> (half + 4 * i)) & 0xF
                    assert nib in (0x4, 0xE)
                    idx[row, 4 * q + i] = 0 if nib == 0x4 else 1
    K = np.zeros((16, 16), np.float32)
    for m in range(16):
        for c in range(8):
            K[m, 2 * c + idx[m, c]] += comp[m, c]
    return K


def test_wide_layout_pairs_are_16_apart_and_lane_loads_contiguous():
    for h in (0, 1):
        pos = [phi_wide(h, k) for k in range(16)]
        assert sorted(pos) == sorted(set(pos))
        for c in range(8):
            assert pos[2 * c + 1] - pos[2 * c] == 16
        for q in range(4):
            assert [pos[q + 4 * i] for i in range(4)] == list(range(pos[q], pos[q] + 4))
    assert sorted(phi_wide(h, k) for h in (0, 1) for k in range(16)) == list(range(32))
    # no band of 2r + 1 <= 15 positions holds both members of a pair
    for r in range(4, 8):
        for start in range(0, 32 - 2 * r):
            band = set(range(start, start + 2 * r + 1))
            for h in (0, 1):
                for c in range(8):
                    assert not ({phi_wide(h, 2 * c), phi_wide(h, 2 * c + 1)} <= band)


@pytest.mark.parametrize("ndim,r", [(2, 4), (2, 5), (2, 7), (1, 1), (1, 3), (1, 6), (1, 7)])
def test_wide_operands_decode_to_banded_kernel_rows(ndim, r):
    # radius 4..7, and every 1-D radius, use the wide layout
    gen = np.random.default_rng(200 + r)
    w = gen.standard_normal((2 * r + 1,) * ndim).astype(np.float32)
    p = spider.Plan(w, (16,) * ndim, "box", "tf32")
    words, meta = p.operands()
    nkr = 2 * r + 1 if ndim == 2 else 1
    w2 = w.reshape((nkr, 2 * r + 1))
    assert words.size == nkr * 2 * 128 and meta.size == nkr * 2 * 32
    words = words.reshape(nkr, 2, 32, 4)
    meta = meta.reshape(nkr, 2, 32)
    used = np.zeros_like(w2)
    for kr in range(nkr):
        win = np.zeros((16, 32), np.float32)  # row m: output m of the segment; column: window position
        for h in (0, 1):
            K = decode_k_order(words[kr, h], meta[kr, h])
            for k in range(16):
                win[:, phi_wide(h, k)] += K[:, k]
        used[kr] = win[0, 8 - r:9 + r]
        exp = np.zeros((16, 32), np.float32)
        for m in range(16):
            for pos in range(32):
                dx = pos - 8 - m
                if abs(dx) <= r:
                    exp[m, pos] = used[kr, dx + r]
        assert np.array_equal(win, exp), kr
    bits = w2.view(np.uint32) & np.uint32(0xFFFFE000)
    assert np.all((used == bits.view(np.float32)) | (used == (bits + np.uint32(0x2000)).view(np.float32)))
    p.close()


def test_wide_radius_limits(lib):
    def create(nd, r, prec="tf32"):
        return spider.Plan(np.full((2 * r + 1,) * nd, 0.01, np.float32), (32,) * nd, "box", prec)
    for nd, r in ((1, 4), (2, 7)):
        p = create(nd, r)
        with pytest.raises(spider.SpiderError) as e:
            p.set_engine("dense_tc")
        assert e.value.status == _native.SPIDER_ERR_UNSUPPORTED
        if nd == 1:
            p.set_steps_per_pass(4)  # 1-D wide plans have fused passes
        else:
            with pytest.raises(spider.SpiderError):
                p.set_steps_per_pass(2)
        p.close()
    for nd, r, prec in ((3, 4, "tf32"), (2, 8, "tf32"), (2, 5, "f16x2"), (1, 4, "bf16x3")):
        with pytest.raises(spider.SpiderError) as e:
            create(nd, r, prec)
        assert e.value.status == _native.SPIDER_ERR_UNSUPPORTED


def test_batched_workload_generators_match_their_descriptions():
    # the small-grid batch must stay under the queue's 2^16-point routing
    # threshold; the mix spans it (sides 256..4096); both are reproducible
    import stencil_inputs as si
    small, mix = si.batched_small_jobs(), si.batched_jobs()
    assert len(small) == 256 and len(mix) == 64
    assert all(32 <= s <= 255 for j in small for s in j.extents)
    assert max(int(np.prod(j.extents)) for j in small) < 2 ** 16
    assert all(256 <= s <= 4096 for j in mix for s in j.extents)
    assert all(10 <= j.steps <= 200 and 1 <= j.r <= 3 for j in small + mix)
    assert si.batched_small_jobs() == small and si.batched_jobs() == mix


@pytest.mark.parametrize("engine", ["sparse_tc_copy", "sparse_tc_no_co"])
def test_one_step_comparator_engines_are_2d_tf32_only(lib, engine):
    # host-side checks (no device work): the explicit-copy and no-CO
    # comparators exist for 2-D TF32 plans of radius 1..3, one step per pass
    import stencil_inputs as si
    w2 = si.normalised_coeffs(2, 2, "box", si.rng(31, 0))
    p = spider.Plan(w2, (40, 72), "box", "tf32", engine)
    with pytest.raises(spider.SpiderError) as e:
        p.set_steps_per_pass(2)
    assert e.value.status == _native.SPIDER_ERR_UNSUPPORTED
    assert p.error_bound(100, "tf32", engine) == pytest.approx(p.error_bound(100, "tf32", "dense_tc"))
    p.close()
    for ext, prec in (((40, 72), "f16x2"), ((40, 72), "bf16x3"), ((8, 16, 72), "tf32")):
        p = spider.Plan(si.normalised_coeffs(len(ext), 1, "box", si.rng(31, 1)), ext, "box", prec)
        with pytest.raises(spider.SpiderError) as e:
            p.set_engine(engine)
        assert e.value.status == _native.SPIDER_ERR_UNSUPPORTED
        p.close()


def test_run_host_async_rejects_bad_arguments_without_touching_a_device(lib):
    import stencil_inputs as si
    buf = np.zeros(40 * 72, np.float32)
    ptr = buf.ctypes.data_as(ctypes.c_void_p)
    assert lib.spider_run_host_async(None, ptr, ptr, 1, None) == _native.SPIDER_ERR_INVALID
    p = spider.Plan(si.normalised_coeffs(2, 1, "box", si.rng(32, 0)), (40, 72), "box", "tf32")
    assert lib.spider_run_host_async(p.handle, None, ptr, 1, None) == _native.SPIDER_ERR_INVALID
    assert lib.spider_run_host_async(p.handle, ptr, None, 1, None) == _native.SPIDER_ERR_INVALID
    assert lib.spider_run_host_async(p.handle, ptr, ptr, -1, None) == _native.SPIDER_ERR_INVALID
    size = ctypes.c_size_t(1)
    assert lib.spider_plan_device_bytes(p.handle, ctypes.byref(size)) == 0
    assert size.value == 0                      # nothing was allocated
    p.close()


def test_autotune_arithmetic_rejects_bad_arguments_without_touching_a_device(lib):
    import stencil_inputs as si
    buf = np.zeros(40 * 72, np.float32)
    ptr = buf.ctypes.data_as(ctypes.c_void_p)
    pr, en, rate = ctypes.c_int(), ctypes.c_int(), ctypes.c_double()
    args = (ctypes.byref(pr), ctypes.byref(en), ctypes.byref(rate))
    assert lib.spider_plan_autotune_arithmetic(None, ptr, ptr, 10, 1e-3, None, *args) == _native.SPIDER_ERR_INVALID
    p = spider.Plan(si.normalised_coeffs(2, 1, "box", si.rng(34, 0)), (40, 72), "box", "tf32")
    for steps, target in ((0, 1e-3), (10, 0.0), (10, -1.0), (10, float("nan")), (10, float("inf"))):
        assert lib.spider_plan_autotune_arithmetic(p.handle, ptr, ptr, steps, target, None, *args) == \
            _native.SPIDER_ERR_INVALID, (steps, target)
    p.close()
