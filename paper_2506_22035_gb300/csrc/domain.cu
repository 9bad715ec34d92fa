// Domain decomposition of one grid into slabs with ghost planes.
//
// The grid is cut into `parts` slabs along its slowest axis (z for 3-D
// stencils, y for 2-D, x for 1-D).  Slab p owns planes [first, first + owned)
// and keeps, on each side that has a neighbour, g ghost planes copied from
// that neighbour.  One exchange period runs E time steps on every slab as an
// ordinary grid of (ghost_lo + owned + ghost_hi) planes with the zero halo
// at its ends.  A slab's ghost planes go wrong from the outside in, r planes
// per step (their own outer neighbours are missing), so with g >= E r the
// owned planes after E steps are exactly those of the undivided run.  Then
// each slab's outermost g owned planes are copied into its neighbours' ghost
// planes and the next period starts.  Only the global grid's two end faces
// carry the zero Dirichlet halo of the stencil (Sec. 1: the HALO region of
// the points next to a tile's edge).
//
// Every slab computes each owned point with the same products in the same
// order as the undivided grid does, so results are bit-identical, provided
// the slab origins keep the points at the same place inside the tensor-core
// tiles where that place changes the arithmetic: 8-point segments along x
// (the output index inside a segment selects the A row), and row pairs along
// y for the split precisions, whose k32 products take two input rows at
// once.  Slab boundaries and ghost depths are therefore multiples of 8 (1-D;
// 16 for the 16-point segments of the wide layout) or 2 (2-D).
//
// On a machine with one GPU per slab each slab would live on its own device
// and the exchange would be a peer copy; here every slab is on the current
// device, which makes the exchange testable on one GPU.
#include <algorithm>
#include <memory>
#include <vector>

#include "spider_internal.h"

struct spider_domain_t {
  struct Slab {
    int64_t first = 0, owned = 0, glo = 0, ghi = 0;
    spider_plan plan = nullptr;
    float* buf[2] = {nullptr, nullptr};
    int64_t planes() const { return glo + owned + ghi; }
  };
  int ndim = 1;
  int64_t extents[3] = {1, 1, 1};
  int64_t axis = 1;    // planes along the split axis
  int64_t plane = 1;   // points per plane
  int exchange = 1;    // E: time steps per exchange period
  int64_t ghost = 0;   // g: ghost planes per interior side
  std::vector<Slab> slabs;
  std::mutex mu;
};

namespace spider {
namespace {

void free_slabs(spider_domain_t* d) {
  for (auto& s : d->slabs) {
    if (s.buf[0]) cudaFree(s.buf[0]);
    if (s.buf[1]) cudaFree(s.buf[1]);
    s.buf[0] = s.buf[1] = nullptr;
    if (s.plan) spider_plan_destroy(s.plan);
    s.plan = nullptr;
  }
}

spider_status ensure_buffers(spider_domain_t* d) {
  for (auto& s : d->slabs) {
    if (s.buf[0]) continue;
    const size_t bytes = (size_t)(s.planes() * d->plane) * sizeof(float);
    cudaError_t e = cudaMalloc(&s.buf[0], bytes);
    if (e == cudaSuccess) e = cudaMalloc(&s.buf[1], bytes);
    if (e != cudaSuccess) {
      cudaGetLastError();
      if (s.buf[0]) cudaFree(s.buf[0]);
      s.buf[0] = s.buf[1] = nullptr;
      return fail(SPIDER_ERR_OOM, "slab grids");
    }
  }
  return SPIDER_OK;
}

}  // namespace
}  // namespace spider

using namespace spider;

extern "C" {

spider_status spider_domain_create(spider_plan plan, int parts, int steps_per_exchange, spider_domain* out) {
  set_error("");
  if (!out) return fail(SPIDER_ERR_INVALID, "out is NULL");
  *out = nullptr;
  if (!plan) return fail(SPIDER_ERR_INVALID, "plan is NULL");
  if (parts < 1) return fail(SPIDER_ERR_INVALID, "parts must be >= 1");
  if (steps_per_exchange < 0) return fail(SPIDER_ERR_INVALID, "steps_per_exchange must be >= 0");
  auto d = std::make_unique<spider_domain_t>();
  d->ndim = plan->ndim;
  for (int i = 0; i < plan->ndim; ++i) d->extents[i] = plan->extents[i];
  d->axis = plan->extents[0];
  d->plane = plan->points() / d->axis;
  d->exchange = steps_per_exchange > 0 ? steps_per_exchange : plan->steps_per_pass;
  // x slabs keep 8-point segments (16-point segments in the wide layout)
  const int64_t align = plan->ndim == 1 ? (plan->wide() ? 16 : 8) : plan->ndim == 2 ? 2 : 1;
  const int64_t need = (int64_t)d->exchange * plan->r;
  d->ghost = parts > 1 ? (need + align - 1) / align * align : 0;
  if (parts > d->axis) return fail(SPIDER_ERR_INVALID, "more parts than planes");
  // slab boundaries: the even split rounded down to the alignment
  std::vector<int64_t> cut(parts + 1);
  for (int p = 0; p <= parts; ++p) cut[p] = (p == parts) ? d->axis : (d->axis * p / parts) / align * align;
  for (int p = 0; p < parts; ++p) {
    spider_domain_t::Slab s;
    s.first = cut[p];
    s.owned = cut[p + 1] - cut[p];
    s.glo = p > 0 ? d->ghost : 0;
    s.ghi = p + 1 < parts ? d->ghost : 0;
    // a neighbour must own every plane of the ghost region it fills
    if (s.owned < 1 || (parts > 1 && s.owned < d->ghost)) {
      return fail(SPIDER_ERR_INVALID, "slabs too thin for the ghost depth (steps_per_exchange * radius)");
    }
    d->slabs.push_back(s);
  }
  for (auto& s : d->slabs) {
    int64_t ext[3];
    for (int i = 0; i < plan->ndim; ++i) ext[i] = plan->extents[i];
    ext[0] = s.planes();
    spider_status st = spider_plan_create(plan->ndim, ext, plan->shape, plan->r, plan->w.data(), plan->prec, &s.plan);
    if (st == SPIDER_OK && plan->engine != SPIDER_ENGINE_SPARSE_TC) st = spider_plan_set_engine(s.plan, plan->engine);
    if (st == SPIDER_OK) {
      s.plan->steps_per_pass = plan->steps_per_pass;
      s.plan->tile_variant = plan->tile_variant;
    } else {
      free_slabs(d.get());
      return st;
    }
  }
  *out = d.release();
  return SPIDER_OK;
}

spider_status spider_domain_slab(spider_domain d, int i, int64_t* first, int64_t* owned, int64_t* ghost_lo,
                                 int64_t* ghost_hi) {
  set_error("");
  if (!d) return fail(SPIDER_ERR_INVALID, "domain is NULL");
  if (i < 0 || i >= (int)d->slabs.size()) return fail(SPIDER_ERR_INVALID, "slab index out of range");
  const auto& s = d->slabs[i];
  if (first) *first = s.first;
  if (owned) *owned = s.owned;
  if (ghost_lo) *ghost_lo = s.glo;
  if (ghost_hi) *ghost_hi = s.ghi;
  return SPIDER_OK;
}

spider_status spider_domain_run(spider_domain d, const float* grid_in, float* grid_out, int64_t steps,
                                cudaStream_t stream) {
  set_error("");
  if (!d) return fail(SPIDER_ERR_INVALID, "domain is NULL");
  if (!grid_in || !grid_out) return fail(SPIDER_ERR_INVALID, "grid pointer is NULL");
  if (steps < 0) return fail(SPIDER_ERR_INVALID, "steps must be >= 0");
  const size_t pbytes = (size_t)d->plane * sizeof(float);
  const size_t total = (size_t)d->axis * pbytes;
  const char* in_c = reinterpret_cast<const char*>(grid_in);
  const char* out_c = reinterpret_cast<const char*>(grid_out);
  if (in_c < out_c + total && out_c < in_c + total) return fail(SPIDER_ERR_INVALID, "grid_in and grid_out overlap");
  std::lock_guard<std::mutex> lock(d->mu);
  spider_status st = ensure_buffers(d);
  if (st != SPIDER_OK) return st;
  auto copy = [&](void* dst, const void* src, size_t bytes) -> spider_status {
    const cudaError_t e = cudaMemcpyAsync(dst, src, bytes, cudaMemcpyDeviceToDevice, stream);
    if (e != cudaSuccess) return fail(SPIDER_ERR_CUDA, cudaGetErrorString(e));
    return SPIDER_OK;
  };
  // scatter: every slab takes its owned and ghost planes from grid_in
  for (auto& s : d->slabs) {
    st = copy(s.buf[0], grid_in + (s.first - s.glo) * d->plane, (size_t)s.planes() * pbytes);
    if (st != SPIDER_OK) return st;
  }
  int cur = 0;
  for (int64_t done = 0; done < steps;) {
    const int64_t e = std::min<int64_t>(d->exchange, steps - done);
    for (auto& s : d->slabs) {
      st = spider_run(s.plan, s.buf[cur], s.buf[1 - cur], e, stream);
      if (st != SPIDER_OK) return st;
    }
    cur = 1 - cur;
    done += e;
    if (done == steps) break;
    // exchange: the outermost g owned planes of each slab fill its
    // neighbour's ghost planes
    for (size_t p = 1; p < d->slabs.size(); ++p) {
      auto& lo = d->slabs[p - 1];
      auto& hi = d->slabs[p];
      const int64_t g = d->ghost;
      st = copy(hi.buf[cur], lo.buf[cur] + (lo.glo + lo.owned - g) * d->plane, (size_t)g * pbytes);
      if (st != SPIDER_OK) return st;
      st = copy(lo.buf[cur] + (lo.glo + lo.owned) * d->plane, hi.buf[cur] + hi.glo * d->plane, (size_t)g * pbytes);
      if (st != SPIDER_OK) return st;
    }
  }
  // gather the owned planes
  for (auto& s : d->slabs) {
    st = copy(grid_out + s.first * d->plane, s.buf[cur] + s.glo * d->plane, (size_t)s.owned * pbytes);
    if (st != SPIDER_OK) return st;
  }
  return SPIDER_OK;
}

spider_status spider_domain_sync(spider_domain d, cudaStream_t stream) {
  set_error("");
  if (!d) return fail(SPIDER_ERR_INVALID, "domain is NULL");
  for (auto& s : d->slabs) {
    const spider_status st = spider_plan_sync(s.plan, stream);
    if (st != SPIDER_OK) return st;
  }
  return SPIDER_OK;
}

void spider_domain_destroy(spider_domain d) {
  if (!d) return;
  {
    std::lock_guard<std::mutex> lock(d->mu);
    free_slabs(d);
  }
  delete d;
}

}  // extern "C"
