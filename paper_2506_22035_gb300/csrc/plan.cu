// Host-side offline transform (Sec. 3.1) and operand packing (Sec. 3.3.2).
//
// For each dz plane and each A index a (see spider_internal.h) the 16 x 16
// matrix A_a is assembled in window coordinates: row m = (s, xo) with
// s = m / 8 the output row (y + s) and xo = m % 8 the output within the
// segment; column p is window position p (input x = x0 - 4 + p).  Its entry
// is w[dz][dy][dx] with dy = a - ry - s and dx = p - 4 - xo when both are in
// range (the banded kernel matrix of Sec. 3.1.1 for kernel row dy, shifted to
// the 16-wide window), else a structural zero.
//
// The MMA's K order is then taken through the strided permutation phi
// (spider_internal.h), which puts the two members of every 1:2 pair / the
// four members of every 2:4 group 8 window positions apart.  A band of
// 2r+1 <= 7 consecutive positions can hold at most one member of a pair and
// at most two of a group, so the permuted matrix is 1:2 and 2:4 structured
// sparse (Sec. 3.1.2).  Compression keeps the band positions in their
// original order with 2-bit indices, increasing, least significant bits
// first; a group with fewer than two band positions is completed with a
// zero placeholder at the next free index (Sec. 3.1.2, stage 3).
//
// Packing (Sec. 3.3.2): every lane's A registers of one MMA are contiguous
// (one 16-byte load), consecutive MMAs follow each other, and the metadata
// word of each lane is stored next to its neighbours, so the kernel fills its
// registers with coalesced loads.
#include <cmath>
#include <cstring>
#include <stdexcept>
#include <vector>
#include <cuda_fp16.h>
#include <cuda_bf16.h>

#include "spider_internal.h"

namespace spider {

uint32_t round_tf32_rna(float x) {
  // Round to the nearest value with a 10-bit mantissa, ties away from zero
  // (the rounding of cvt.rna.tf32.f32): add half of the dropped range to the
  // magnitude bits and clear the 13 low bits.  Inputs are finite.
  uint32_t u;
  std::memcpy(&u, &x, 4);
  u += 0x1000u;
  u &= 0xFFFFE000u;
  return u;
}

float tf32_value(float x) {
  uint32_t u = round_tf32_rna(x);
  float f;
  std::memcpy(&f, &u, 4);
  return f;
}

static uint16_t h_bits(float x) {
  __half h = __float2half_rn(x);
  uint16_t u;
  std::memcpy(&u, &h, 2);
  return u;
}
static float h_value(float x) { return __half2float(__float2half_rn(x)); }
static uint16_t bf_bits(float x) {
  __nv_bfloat16 h = __float2bfloat16_rn(x);
  uint16_t u;
  std::memcpy(&u, &h, 2);
  return u;
}
static float bf_value(float x) { return __bfloat162float(__float2bfloat16_rn(x)); }

int combos_per_plane(spider_precision prec, int ry) {
  switch (prec) {
    case SPIDER_F16X2: return (ry + 1) + (2 * ry + 2);
    case SPIDER_BF16X3: return 2 * ((ry + 1) + (2 * ry + 2));
    default: return 2 * ry + 2;
  }
}

namespace {

// Which part of a coefficient an operand carries: the coefficient itself
// (the cube passed in is then already the part wanted, e.g. the TF32
// rounding or one term of a split).
enum class Part { Full };

float part_value(float w, Part) { return w; }

struct WindowMatrix {
  float v[16][16];
  bool mask[16][16];
};

// TF32 coefficients rounded so that their sum stays as close as possible to
// the sum of the FP32 coefficients.  Each weight takes one of its two TF32
// neighbours: round to nearest first, then flip the weights whose flip best
// reduces the error of the sum.  With round-to-nearest alone the rounding
// errors of the weights add up to a systematic error of the stencil's
// response to the constant mode that grows linearly with the number of steps;
// here it is bounded by the spacing of the smallest weights.  Exactly
// representable weights are unchanged.
std::vector<float> tf32_sum_preserving(const std::vector<float>& w) {
  const size_t n = w.size();
  std::vector<float> out(n), other(n);
  double resid = 0;
  for (size_t i = 0; i < n; ++i) {
    out[i] = tf32_value(w[i]);
    uint32_t u;
    std::memcpy(&u, &w[i], 4);
    const uint32_t t = u & 0xFFFFE000u;  // neighbour toward zero
    float lo, hi;
    std::memcpy(&lo, &t, 4);
    const uint32_t t2 = t + 0x2000u;     // neighbour away from zero
    std::memcpy(&hi, &t2, 4);
    other[i] = (lo == w[i]) ? w[i] : (out[i] == lo ? hi : lo);
    resid += (double)w[i] - (double)out[i];
  }
  std::vector<bool> flipped(n, false);
  for (;;) {
    int best = -1;
    double best_abs = std::fabs(resid), best_cost = 0;
    for (size_t i = 0; i < n; ++i) {
      if (flipped[i] || other[i] == out[i]) continue;
      const double delta = (double)other[i] - (double)out[i];
      const double r2 = std::fabs(resid - delta);
      const double cost = std::fabs((double)w[i] - (double)other[i]);
      if (r2 < best_abs || (best >= 0 && r2 == best_abs && cost < best_cost)) {
        best = (int)i;
        best_abs = r2;
        best_cost = cost;
      }
    }
    if (best < 0) break;
    resid -= (double)other[best] - (double)out[best];
    std::swap(out[best], other[best]);
    flipped[best] = true;
  }
  return out;
}

// The two 16-bit neighbours of x (FP16 or BF16): *near is x rounded to
// nearest, *far the neighbour on the other side of x (equal to *near when x
// is exactly representable, or when the step would leave the finite range).
void neighbours16(float x, bool bf16, float* near, float* far) {
  const uint16_t b = bf16 ? bf_bits(x) : h_bits(x);
  auto value = [&](uint16_t u) {
    if (bf16) {
      const uint32_t f = (uint32_t)u << 16;
      float v;
      std::memcpy(&v, &f, 4);
      return v;
    }
    __half h;
    std::memcpy(&h, &u, 2);
    return __half2float(h);
  };
  *near = value(b);
  *far = *near;
  if (*near == x) return;
  const uint16_t sign = b & 0x8000u, mag = b & 0x7FFFu;
  const uint16_t inf = bf16 ? 0x7F80u : 0x7C00u;
  uint16_t m2;
  if (std::fabs(*near) < std::fabs(x)) {
    m2 = (uint16_t)(mag + 1);
    if (m2 >= inf) return;
  } else {
    m2 = (uint16_t)(mag - 1);  // |near| > |x| >= 0, so mag >= 1
  }
  *far = value((uint16_t)(sign | m2));
}

// Greedy flips that bring sum_i (need_i - scale * out_i) as close to zero as
// possible, each out_i taking one of its two candidates (out_i, other_i).
// The rule of tf32_sum_preserving, for the last term of a split.
void sum_preserving_flips(const std::vector<double>& need, std::vector<float>& out, std::vector<float>& other,
                          double scale) {
  const size_t n = out.size();
  double resid = 0;
  for (size_t i = 0; i < n; ++i) resid += need[i] - scale * (double)out[i];
  std::vector<bool> flipped(n, false);
  for (;;) {
    int best = -1;
    double best_abs = std::fabs(resid), best_cost = 0;
    for (size_t i = 0; i < n; ++i) {
      if (flipped[i] || other[i] == out[i]) continue;
      const double delta = scale * ((double)other[i] - (double)out[i]);
      const double r2 = std::fabs(resid - delta);
      const double cost = std::fabs(need[i] - scale * (double)other[i]);
      if (r2 < best_abs || (best >= 0 && r2 == best_abs && cost < best_cost)) {
        best = (int)i;
        best_abs = r2;
        best_cost = cost;
      }
    }
    if (best < 0) break;
    resid -= scale * ((double)other[best] - (double)out[best]);
    std::swap(out[best], other[best]);
    flipped[best] = true;
  }
}

}  // namespace

// Split weights (see spider_internal.h).  FP16: hi = w rounded to FP16,
// lo = (w - hi) * 2^11 rounded to FP16.  BF16: hi, mid = (w - hi) and
// lo = (w - hi - mid), each rounded to BF16; the differences are exact in
// FP32.  The last term of every weight takes one of its two 16-bit
// neighbours so that the split weights sum as close as possible to the FP32
// weights: a rounding error of the sum multiplies the constant mode every
// step and grows linearly with the step count, where the rounding errors of
// single weights do not.
SplitWeights split_weights(const std::vector<float>& w, spider_precision prec) {
  SplitWeights sw;
  const size_t n = w.size();
  const bool bf = prec == SPIDER_BF16X3;
  sw.hi.resize(n);
  sw.mid.assign(n, 0.f);
  sw.lo.resize(n);
  sw.lo_scale = bf ? 1.0 : 1.0 / 2048.0;
  std::vector<float> other(n);
  std::vector<double> need(n);
  for (size_t i = 0; i < n; ++i) {
    sw.hi[i] = bf ? bf_value(w[i]) : h_value(w[i]);
    float rest = w[i] - sw.hi[i];
    if (bf) {
      sw.mid[i] = bf_value(rest);
      rest = rest - sw.mid[i];
    } else {
      rest = rest * 2048.0f;
    }
    neighbours16(rest, bf, &sw.lo[i], &other[i]);
    need[i] = (double)w[i] - (double)sw.hi[i] - (double)sw.mid[i];
  }
  sum_preserving_flips(need, sw.lo, other, sw.lo_scale);
  return sw;
}

double split_sum_error(const std::vector<float>& w, const SplitWeights& sw) {
  double d = 0;
  for (size_t i = 0; i < w.size(); ++i)
    d += (double)w[i] - ((double)sw.hi[i] + (double)sw.mid[i] + sw.lo_scale * (double)sw.lo[i]);
  return d;
}

namespace {

// A_a for plane dz (index dzi = dz + rz) in window coordinates; `coeffs`
// supplies the cube (the plan's FP32 weights or their TF32 rounding).
WindowMatrix window_matrix(const spider_plan_t* p, const std::vector<float>& coeffs, int dzi, int a, Part part) {
  WindowMatrix A;
  const int wy = 2 * p->ry + 1, wx = 2 * p->rx + 1;
  for (int m = 0; m < 16; ++m) {
    const int s = m / 8, xo = m % 8;
    const int dy = a - p->ry - s;
    for (int q = 0; q < 16; ++q) {
      const int dx = q - kHaloX - xo;
      const bool in = (dy >= -p->ry && dy <= p->ry && dx >= -p->rx && dx <= p->rx);
      A.mask[m][q] = in;
      A.v[m][q] = in ? part_value(coeffs[((size_t)dzi * wy + (dy + p->ry)) * wx + (dx + p->rx)], part) : 0.f;
    }
  }
  return A;
}

uint32_t f32_bits(float x) {
  uint32_t u;
  std::memcpy(&u, &x, 4);
  return u;
}

// TF32 m16n8k16, 1:2 on K pairs (2c, 2c+1).  Fragment maps (verified on the
// device): A compressed 16 x 8 -- a0 (g, q), a1 (g+8, q), a2 (g, q+4),
// a3 (g+8, q+4) with g = lane/4, q = lane%4; metadata (selector 0) -- lanes
// with q in {0,1} hold row g pairs 4q..4q+3 in bits 0-15 and row g+8 in bits
// 16-31, one nibble per pair: 0b0100 keeps the first element, 0b1110 the
// second.
// `K` is in MMA K order (column k = K index).
void pack_tf32_sparse_k(const WindowMatrix& K, uint32_t* words /*32x4*/, uint32_t* meta /*32*/) {
  float cval[16][8];
  int cidx[16][8];
  for (int m = 0; m < 16; ++m) {
    for (int c = 0; c < 8; ++c) {
      const int p0 = 2 * c, p1 = 2 * c + 1;
      if (K.mask[m][p0] && K.mask[m][p1]) throw std::runtime_error("internal: pair not 1:2");
      if (K.mask[m][p1]) { cidx[m][c] = 1; cval[m][c] = K.v[m][p1]; }
      else { cidx[m][c] = 0; cval[m][c] = K.mask[m][p0] ? K.v[m][p0] : 0.f; }
    }
  }
  for (int lane = 0; lane < 32; ++lane) {
    const int g = lane / 4, q = lane % 4;
    words[lane * 4 + 0] = f32_bits(cval[g][q]);
    words[lane * 4 + 1] = f32_bits(cval[g + 8][q]);
    words[lane * 4 + 2] = f32_bits(cval[g][q + 4]);
    words[lane * 4 + 3] = f32_bits(cval[g + 8][q + 4]);
    uint32_t e = 0;
    if (q < 2) {
      for (int i = 0; i < 4; ++i) {
        const uint32_t n0 = cidx[g][4 * q + i] ? 0xEu : 0x4u;
        const uint32_t n1 = cidx[g + 8][4 * q + i] ? 0xEu : 0x4u;
        e |= n0 << (4 * i);
        e |= n1 << (16 + 4 * i);
      }
    }
    meta[lane] = e;
  }
}

// `A` is in window coordinates; its K order is taken through phi_tf32.
void pack_tf32_sparse(const WindowMatrix& A, uint32_t* words /*32x4*/, uint32_t* meta /*32*/) {
  WindowMatrix K;
  for (int m = 0; m < 16; ++m)
    for (int k = 0; k < 16; ++k) {
      K.v[m][k] = A.v[m][phi_tf32(k)];
      K.mask[m][k] = A.mask[m][phi_tf32(k)];
    }
  pack_tf32_sparse_k(K, words, meta);
}

// Wide layout (radius 4..7): K half h of kernel row kr (dy = kr - ry) in K
// order.  Row m is output m of a 16-output segment, window position
// phi_wide(h, k) is input x = x0 - 8 + position; entry w[dy][dx] with
// dx = position - 8 - m when |dx| <= r.  The band of 2r + 1 <= 15 positions
// never holds both p and p + 16, so every pair is 1:2 (Sec. 3.1.2 with
// L = 16, the paper's worked example for r = 7).
WindowMatrix wide_matrix(const spider_plan_t* p, const std::vector<float>& coeffs, int kr, int h) {
  WindowMatrix K;
  const int wx = 2 * p->rx + 1;
  for (int m = 0; m < 16; ++m)
    for (int k = 0; k < 16; ++k) {
      const int dx = phi_wide(h, k) - kWideHalo - m;
      const bool in = dx >= -p->rx && dx <= p->rx;
      K.mask[m][k] = in;
      K.v[m][k] = in ? coeffs[(size_t)kr * wx + (dx + p->rx)] : 0.f;
    }
  return K;
}

// Dense TF32 m16n8k8, two K halves: a0 (g, q), a1 (g+8, q), a2 (g, q+4),
// a3 (g+8, q+4) with column = K-index within the half.
void pack_tf32_dense(const WindowMatrix& A, uint32_t* words /*32x8*/) {
  for (int lane = 0; lane < 32; ++lane) {
    const int g = lane / 4, q = lane % 4;
    for (int h = 0; h < 2; ++h) {
      auto val = [&](int row, int col) { return f32_bits(A.v[row][phi_tf32(8 * h + col)]); };
      words[lane * 8 + 4 * h + 0] = val(g, q);
      words[lane * 8 + 4 * h + 1] = val(g + 8, q);
      words[lane * 8 + 4 * h + 2] = val(g, q + 4);
      words[lane * 8 + 4 * h + 3] = val(g + 8, q + 4);
    }
  }
}

// Group compression of 4 K-indices with the placeholder rule.
void compress_group(const bool in[4], int idx[2]) {
  int n = 0, pos[4];
  for (int j = 0; j < 4; ++j) if (in[j]) pos[n++] = j;
  if (n > 2) throw std::runtime_error("internal: group not 2:4");
  if (n == 2) { idx[0] = pos[0]; idx[1] = pos[1]; }
  else if (n == 1) {
    if (pos[0] < 3) { idx[0] = pos[0]; idx[1] = pos[0] + 1; }
    else { idx[0] = 2; idx[1] = 3; }
  } else { idx[0] = 0; idx[1] = 1; }
}

// 16-bit m16n8k32, 2:4.  K half 0 is window matrix H0, half 1 is H1.
// Fragment maps (verified on the device): A compressed 16 x 16 --
// a0 (g, 2q..2q+1), a1 (g+8, 2q..), a2 (g, 2q+8..), a3 (g+8, 2q+8..);
// metadata (selector 0) -- lanes with q in {0,1}: nibble i = row g, group
// 4q+i; nibble 4+i = row g+8, group 4q+i; nibble = idx0 | idx1 << 2.
void pack_16bit_sparse_k32(const WindowMatrix& H0, const WindowMatrix& H1, bool bf16,
                           uint32_t* words /*32x4*/, uint32_t* meta /*32*/) {
  float cval[16][16];
  int cidx[16][8][2];
  for (int m = 0; m < 16; ++m) {
    for (int c = 0; c < 8; ++c) {
      const WindowMatrix& H = c < 4 ? H0 : H1;
      const int c4 = c % 4;
      bool in[4];
      int pos[4];
      for (int j = 0; j < 4; ++j) { pos[j] = phi_16bit(4 * c4 + j); in[j] = H.mask[m][pos[j]]; }
      int idx[2];
      compress_group(in, idx);
      cidx[m][c][0] = idx[0];
      cidx[m][c][1] = idx[1];
      for (int s = 0; s < 2; ++s) cval[m][2 * c + s] = in[idx[s]] ? H.v[m][pos[idx[s]]] : 0.f;
    }
  }
  auto bits = [&](float x) -> uint32_t { return bf16 ? bf_bits(x) : h_bits(x); };
  auto pack2 = [&](int row, int col) { return bits(cval[row][col]) | (bits(cval[row][col + 1]) << 16); };
  for (int lane = 0; lane < 32; ++lane) {
    const int g = lane / 4, q = lane % 4;
    words[lane * 4 + 0] = pack2(g, 2 * q);
    words[lane * 4 + 1] = pack2(g + 8, 2 * q);
    words[lane * 4 + 2] = pack2(g, 2 * q + 8);
    words[lane * 4 + 3] = pack2(g + 8, 2 * q + 8);
    uint32_t e = 0;
    if (q < 2) {
      for (int i = 0; i < 4; ++i) {
        const int grp = 4 * q + i;
        e |= (uint32_t)(cidx[g][grp][0] | (cidx[g][grp][1] << 2)) << (4 * i);
        e |= (uint32_t)(cidx[g + 8][grp][0] | (cidx[g + 8][grp][1] << 2)) << (16 + 4 * i);
      }
    }
    meta[lane] = e;
  }
}

}  // namespace

spider_status build_operands(spider_plan_t* p) {
  const int planes = 2 * p->rz + 1;
  const int na = 2 * p->ry + 2;
  p->n_arows = planes * na;
  p->a_words.clear();
  p->meta_words.clear();
  try {
    const std::vector<float> w_tf32 = tf32_sum_preserving(p->w);
    // weight-sum errors of every arithmetic, relative to sum |w| (the error
    // model of spider_plan_error_bound)
    double wabs = 0, d_tf32 = 0;
    for (size_t i = 0; i < p->w.size(); ++i) {
      wabs += std::fabs((double)p->w[i]);
      d_tf32 += (double)p->w[i] - (double)w_tf32[i];
    }
    const double scale = wabs > 0 ? 1.0 / wabs : 0.0;
    p->wsum_rel[0] = std::fabs(d_tf32) * scale;
    p->wsum_rel[1] = std::fabs(split_sum_error(p->w, split_weights(p->w, SPIDER_F16X2))) * scale;
    p->wsum_rel[2] = std::fabs(split_sum_error(p->w, split_weights(p->w, SPIDER_BF16X3))) * scale;
    if (p->prec == SPIDER_F16X2 || p->prec == SPIDER_BF16X3) p->split = split_weights(p->w, p->prec);
    if (p->wide()) {
      // wide layout: [kernel row][K half][lane] (sparse TF32 only)
      const int nkr = 2 * p->ry + 1;
      p->n_arows = nkr;
      p->n_combos = 2 * nkr;
      p->a_words.resize((size_t)p->n_combos * 128);
      p->meta_words.resize((size_t)p->n_combos * 32);
      for (int kr = 0; kr < nkr; ++kr)
        for (int h = 0; h < 2; ++h)
          pack_tf32_sparse_k(wide_matrix(p, w_tf32, kr, h), &p->a_words[(size_t)(2 * kr + h) * 128],
                             &p->meta_words[(size_t)(2 * kr + h) * 32]);
      return SPIDER_OK;
    }
    if (p->engine == SPIDER_ENGINE_CUDA_CORE) {
      p->n_combos = 0;
      return SPIDER_OK;
    }
    if (p->engine == SPIDER_ENGINE_DENSE_TC) {
      p->n_combos = p->n_arows;
      p->a_words.resize((size_t)p->n_arows * 32 * 8);
      for (int dzi = 0; dzi < planes; ++dzi)
        for (int a = 0; a < na; ++a)
          pack_tf32_dense(window_matrix(p, w_tf32, dzi, a, Part::Full), &p->a_words[((size_t)dzi * na + a) * 256]);
      return SPIDER_OK;
    }
    const int cpp = combos_per_plane(p->prec, p->ry);
    p->n_combos = planes * cpp;
    p->a_words.resize((size_t)p->n_combos * 128);
    p->meta_words.resize((size_t)p->n_combos * 32);
    for (int dzi = 0; dzi < planes; ++dzi) {
      if (p->prec == SPIDER_TF32 || p->prec == SPIDER_AUTO) {
        for (int a = 0; a < na; ++a) {
          const size_t c = (size_t)dzi * cpp + a;
          pack_tf32_sparse(window_matrix(p, w_tf32, dzi, a, Part::Full), &p->a_words[c * 128], &p->meta_words[c * 32]);
        }
      } else {
        // One pass of combos per split term pair, each (ry + 1) two-row
        // combos [K_x(2c) | K_x(2c+1)] x [X_x(j); X_x(j+1)] followed by na
        // one-row combos [K_hi(a) | K_y(a)] x [X_y(j); X_hi(j)]:
        //   FP16 hi/lo:      x = hi,  y = lo (scaled by 2^11)
        //   BF16 hi/mid/lo:  pass 0 x = hi, y = mid; pass 1 x = mid, y = lo
        const bool bf = p->prec == SPIDER_BF16X3;
        const SplitWeights& sw = p->split;
        const int npass = bf ? 2 : 1;
        const int per_pass = (p->ry + 1) + na;
        for (int pass = 0; pass < npass; ++pass) {
          const std::vector<float>& two_row = pass == 0 ? sw.hi : sw.mid;
          const std::vector<float>& cross = (bf && pass == 0) ? sw.mid : sw.lo;
          for (int c = 0; c <= p->ry; ++c) {
            const size_t ci = (size_t)dzi * cpp + pass * per_pass + c;
            pack_16bit_sparse_k32(window_matrix(p, two_row, dzi, 2 * c, Part::Full),
                                  window_matrix(p, two_row, dzi, 2 * c + 1, Part::Full), bf, &p->a_words[ci * 128],
                                  &p->meta_words[ci * 32]);
          }
          for (int a = 0; a < na; ++a) {
            const size_t ci = (size_t)dzi * cpp + pass * per_pass + (p->ry + 1) + a;
            pack_16bit_sparse_k32(window_matrix(p, sw.hi, dzi, a, Part::Full),
                                  window_matrix(p, cross, dzi, a, Part::Full), bf, &p->a_words[ci * 128],
                                  &p->meta_words[ci * 32]);
          }
        }
      }
    }
  } catch (const std::exception& e) {
    return fail(SPIDER_ERR_INVALID, e.what());
  }
  return SPIDER_OK;
}

}  // namespace spider
