/*
 * FP64 direct stencil oracle -- TEST INFRASTRUCTURE ONLY.
 *
 * Only tests, the smoke check and the CPU-baseline leg of the benchmark may
 * load this library.  The product path never calls it and shares no code,
 * header or constant with it.
 *
 * What it computes (SPIDER, Sec. 1 and Sec. 2.2, the stencil definition):
 *
 *     u_{t+1}[i] = sum_{o in S} w[o] * u_t[i + o],   t = 0 .. steps-1,
 *
 * where S is the full (2r+1)^d offset cube (a star stencil is the same cube
 * with its off-axis coefficients equal to 0), i.e. a correlation with
 * offsets o in [-r, r]^d.  Everything is computed in double precision from
 * the caller's double inputs.  Two boundary modes:
 *   periodic == 0 : zero Dirichlet -- every point outside the grid reads as
 *                   0 at every step, and every point of the grid is updated;
 *   periodic == 1 : indices wrap around (used by the Fourier-mode pins).
 *
 * Coefficients are dense, row-major [dz][dy][dx] with each offset running
 * -r..r.  Extents are given slowest axis first, x (contiguous) last.
 * There is no matrix lowering here: every output is the plain sum above,
 * accumulated over the offsets in a fixed order (dz, dy, dx ascending), so
 * the result does not depend on the thread count.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

static int64_t wrap_index(int64_t i, int64_t n) {
  int64_t m = i % n;
  return m < 0 ? m + n : m;
}

/* Returns 0 on success, -1 on invalid arguments, -2 on allocation failure. */
int oracle_stencil_fp64(int ndim, const int64_t* extents, int r, const double* w,
                        const double* in, double* out, int64_t steps, int periodic,
                        int nthreads) {
  if (ndim < 1 || ndim > 3 || r < 0 || steps < 0 || !extents || !w || !in || !out) return -1;
  int64_t nz = 1, ny = 1, nx = extents[ndim - 1];
  if (ndim >= 2) ny = extents[ndim - 2];
  if (ndim >= 3) nz = extents[0];
  if (nx < 1 || ny < 1 || nz < 1) return -1;
  const int rz = ndim >= 3 ? r : 0, ry = ndim >= 2 ? r : 0, rx = r;
  const int wy = 2 * ry + 1, wx = 2 * rx + 1;
  const int64_t n = nz * ny * nx;

  double* a = (double*)malloc((size_t)n * sizeof(double));
  double* b = (double*)malloc((size_t)n * sizeof(double));
  if (!a || !b) { free(a); free(b); return -2; }
  memcpy(a, in, (size_t)n * sizeof(double));
  if (nthreads <= 0) nthreads = 1;

  for (int64_t t = 0; t < steps; ++t) {
    if (!periodic) {
      /* Zero Dirichlet.  For each output row (z, y) accumulate, offset by
       * offset, w[o] * u[z+dz][y+dy][x+dx] over the x for which the input
       * point lies inside the grid; everything outside contributes 0. */
#pragma omp parallel for collapse(2) schedule(static) num_threads(nthreads)
      for (int64_t z = 0; z < nz; ++z) {
        for (int64_t y = 0; y < ny; ++y) {
          double* orow = b + (z * ny + y) * nx;
          for (int64_t x = 0; x < nx; ++x) orow[x] = 0.0;
          for (int dz = -rz; dz <= rz; ++dz) {
            const int64_t zz = z + dz;
            if (zz < 0 || zz >= nz) continue;
            for (int dy = -ry; dy <= ry; ++dy) {
              const int64_t yy = y + dy;
              if (yy < 0 || yy >= ny) continue;
              const double* irow = a + (zz * ny + yy) * nx;
              for (int dx = -rx; dx <= rx; ++dx) {
                const double c = w[((dz + rz) * wy + (dy + ry)) * wx + (dx + rx)];
                const int64_t lo = dx < 0 ? -dx : 0;          /* x + dx >= 0  */
                const int64_t hi = dx > 0 ? nx - dx : nx;     /* x + dx < nx  */
                for (int64_t x = lo; x < hi; ++x) orow[x] += c * irow[x + dx];
              }
            }
          }
        }
      }
    } else {
#pragma omp parallel for collapse(2) schedule(static) num_threads(nthreads)
      for (int64_t z = 0; z < nz; ++z) {
        for (int64_t y = 0; y < ny; ++y) {
          for (int64_t x = 0; x < nx; ++x) {
            double s = 0.0;
            for (int dz = -rz; dz <= rz; ++dz) {
              const int64_t zz = wrap_index(z + dz, nz);
              for (int dy = -ry; dy <= ry; ++dy) {
                const int64_t yy = wrap_index(y + dy, ny);
                for (int dx = -rx; dx <= rx; ++dx) {
                  const int64_t xx = wrap_index(x + dx, nx);
                  s += w[((dz + rz) * wy + (dy + ry)) * wx + (dx + rx)] * a[(zz * ny + yy) * nx + xx];
                }
              }
            }
            b[(z * ny + y) * nx + x] = s;
          }
        }
      }
    }
    double* tmp = a; a = b; b = tmp;
  }
  memcpy(out, a, (size_t)n * sizeof(double));
  free(a);
  free(b);
  return 0;
}

/* Number of OpenMP threads the oracle would use by default (1 without OpenMP). */
int oracle_max_threads(void) {
#ifdef _OPENMP
  return omp_get_max_threads();
#else
  return 1;
#endif
}
