/*
 * Oracle for the stencil sweeps -- TEST INFRASTRUCTURE ONLY.
 *
 * Only the tests, the smoke check and the benchmark's CPU-baseline leg may load this code.  It
 * shares nothing with the CUDA library: no headers, no helpers, no tables.
 *
 * What it computes: T applications of one of the seven stencil operators of Listings 1-4 of
 * Malas et al. (arXiv 1510.04995, Sect. 2.2) to the interior of a padded 3D grid, in FP64, in the
 * plain lexicographic ("naive") order of the 1D example of Sect. 2.1.1: every time step reads the
 * level-t array and writes the level-(t+1) array; the two arrays swap roles after each step.  The
 * halo of width R (R=1 for the 7-point, R=4 for the 25-point stencils) is never written (the
 * listings' loops run from R to N-R-1).  Temporal blocking (wavefront, diamond tiling) only
 * reorders these independent updates, so this plain sweep is the exact definition of the result.
 *
 * Each point is evaluated in the literal left-to-right term order of its listing, one rounding
 * per operation (build with -ffp-contract=off so that no fused multiply-add is formed):
 *   7pt const  (Listing 1): c0*V + c1*(x+1 + x-1) + c1*(y+1 + y-1) + c1*(z+1 + z-1)
 *   7pt var    (Listing 2): C0*V + C1*x+1 + C2*x-1 + C3*y+1 + C4*y-1 + C5*z+1 + C6*z-1
 *   25pt const (Listing 3 with the per-point factor C = 1, second order in time):
 *       (2*V - U) + (c0*V + c1*(x+1 + x-1 + y+1 + y-1 + z+1 + z-1) + ... + c4*(... r=4 ...))
 *   25pt var   (Listing 4's 13 axis-symmetric coefficient grids, with the second-order-in-time
 *       update of Listing 3):  (2*V - U) + (C00*V + C01*(x+1 + x-1) + C02*(y+1 + y-1)
 *       + C03*(z+1 + z-1) + C04*(x+2 pair) + ... + C12*(z+4 pair))
 *   25pt C grid (Listing 3 as printed, with its per-point factor grid C):
 *       (2*V - U) + C * (c0*V + c1*(x+1 + x-1 + y+1 + y-1 + z+1 + z-1) + ... + c4*(... r=4 ...))
 *   27pt box   (the box-shaped operator of Sect. 7: all 26 neighbours at Chebyshev distance 1,
 *       first order in time, constants by neighbour class):
 *       c0*V + c1*(sum of the 6 face neighbours) + c2*(sum of the 12 edge neighbours)
 *            + c3*(sum of the 8 corner neighbours)
 *       each sum taken over the offsets (dx, dy, dz) in lexicographic order (dz outermost, then
 *       dy, then dx, each from -1 to 1).
 *   7pt red-black Gauss-Seidel (Sect. 7): time step t is a half-sweep that updates, in place,
 *       the points whose interior coordinates have (x + y + z + t) even with the 7-point constant
 *       formula (c0*V + c1*(x pair) + c1*(y pair) + c1*(z pair)) and leaves the others; the
 *       updated points' neighbours all have the other colour, so the half-sweep reads only
 *       values of the previous half-step and the in-place order within it does not matter.
 *       Two consecutive time steps make one red-black iteration.
 * For the second-order stencils U is the level t-1 array, overwritten in place by level t+1
 * (Listing 3 writes U = 2V - U + ...).
 *
 * Layout: element (i, j, k) of a padded grid (0 <= i < ldx, 0 <= j < ny+2R, 0 <= k < nz+2R) is
 * at (k*(ny+2R) + j)*ldx + i; interior i in [R, R+nx).  Coefficient grids have the same layout
 * and are stored back to back.  On return u holds level T and u_prev level T-1 (for odd T the
 * two arrays' contents are exchanged at the end); for T = 0 nothing changes.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define IDX(i, j, k) (((int64_t)(k) * sy + (j)) * ldx + (i))

static void step_7c(int64_t nx, int64_t ny, int64_t nz, int64_t ldx, const double* V, double* U,
                    const double* c, int nthreads) {
  const int64_t R = 1, sy = ny + 2 * R;
  const double c0 = c[0], c1 = c[1];
#pragma omp parallel for num_threads(nthreads) schedule(static)
  for (int64_t k = R; k < R + nz; k++)
    for (int64_t j = R; j < R + ny; j++)
      for (int64_t i = R; i < R + nx; i++) {
        U[IDX(i, j, k)] = c0 * V[IDX(i, j, k)]
                        + c1 * (V[IDX(i + 1, j, k)] + V[IDX(i - 1, j, k)])
                        + c1 * (V[IDX(i, j + 1, k)] + V[IDX(i, j - 1, k)])
                        + c1 * (V[IDX(i, j, k + 1)] + V[IDX(i, j, k - 1)]);
      }
}

static void step_7v(int64_t nx, int64_t ny, int64_t nz, int64_t ldx, const double* V, double* U,
                    const double* C, int nthreads) {
  const int64_t R = 1, sy = ny + 2 * R;
  const int64_t g = (nz + 2 * R) * sy * ldx; /* elements per coefficient grid */
  const double *C0 = C, *C1 = C + g, *C2 = C + 2 * g, *C3 = C + 3 * g, *C4 = C + 4 * g,
               *C5 = C + 5 * g, *C6 = C + 6 * g;
#pragma omp parallel for num_threads(nthreads) schedule(static)
  for (int64_t k = R; k < R + nz; k++)
    for (int64_t j = R; j < R + ny; j++)
      for (int64_t i = R; i < R + nx; i++) {
        const int64_t p = IDX(i, j, k);
        U[p] = C0[p] * V[p]
             + C1[p] * V[IDX(i + 1, j, k)]
             + C2[p] * V[IDX(i - 1, j, k)]
             + C3[p] * V[IDX(i, j + 1, k)]
             + C4[p] * V[IDX(i, j - 1, k)]
             + C5[p] * V[IDX(i, j, k + 1)]
             + C6[p] * V[IDX(i, j, k - 1)];
      }
}

static void step_25c(int64_t nx, int64_t ny, int64_t nz, int64_t ldx, const double* V, double* U,
                     const double* c, int nthreads) {
  const int64_t R = 4, sy = ny + 2 * R;
#pragma omp parallel for num_threads(nthreads) schedule(static)
  for (int64_t k = R; k < R + nz; k++)
    for (int64_t j = R; j < R + ny; j++)
      for (int64_t i = R; i < R + nx; i++) {
        const int64_t p = IDX(i, j, k);
        double lap = c[0] * V[p];
        for (int64_t r = 1; r <= 4; r++)
          lap = lap + c[r] * (V[IDX(i + r, j, k)] + V[IDX(i - r, j, k)]
                            + V[IDX(i, j + r, k)] + V[IDX(i, j - r, k)]
                            + V[IDX(i, j, k + r)] + V[IDX(i, j, k - r)]);
        U[p] = 2.0 * V[p] - U[p] + lap;
      }
}

static void step_25v(int64_t nx, int64_t ny, int64_t nz, int64_t ldx, const double* V, double* U,
                     const double* C, int nthreads) {
  const int64_t R = 4, sy = ny + 2 * R;
  const int64_t g = (nz + 2 * R) * sy * ldx;
#pragma omp parallel for num_threads(nthreads) schedule(static)
  for (int64_t k = R; k < R + nz; k++)
    for (int64_t j = R; j < R + ny; j++)
      for (int64_t i = R; i < R + nx; i++) {
        const int64_t p = IDX(i, j, k);
        /* Listing 4: C00 centre; then for r = 1..4 the x, y, z pairs use grids 3r-2, 3r-1, 3r. */
        double acc = C[p] * V[p];
        for (int64_t r = 1; r <= 4; r++) {
          acc = acc + C[(3 * r - 2) * g + p] * (V[IDX(i + r, j, k)] + V[IDX(i - r, j, k)]);
          acc = acc + C[(3 * r - 1) * g + p] * (V[IDX(i, j + r, k)] + V[IDX(i, j - r, k)]);
          acc = acc + C[(3 * r) * g + p] * (V[IDX(i, j, k + r)] + V[IDX(i, j, k - r)]);
        }
        U[p] = 2.0 * V[p] - U[p] + acc;
      }
}

static void step_25cg(int64_t nx, int64_t ny, int64_t nz, int64_t ldx, const double* V, double* U,
                      const double* C, const double* c, int nthreads) {
  const int64_t R = 4, sy = ny + 2 * R;
#pragma omp parallel for num_threads(nthreads) schedule(static)
  for (int64_t k = R; k < R + nz; k++)
    for (int64_t j = R; j < R + ny; j++)
      for (int64_t i = R; i < R + nx; i++) {
        const int64_t p = IDX(i, j, k);
        /* the bracket of Listing 3, then scaled by the factor of this point */
        double lap = c[0] * V[p];
        for (int64_t r = 1; r <= 4; r++)
          lap = lap + c[r] * (V[IDX(i + r, j, k)] + V[IDX(i - r, j, k)]
                            + V[IDX(i, j + r, k)] + V[IDX(i, j - r, k)]
                            + V[IDX(i, j, k + r)] + V[IDX(i, j, k - r)]);
        U[p] = 2.0 * V[p] - U[p] + C[p] * lap;
      }
}

static void step_27b(int64_t nx, int64_t ny, int64_t nz, int64_t ldx, const double* V, double* U,
                     const double* c, int nthreads) {
  const int64_t R = 1, sy = ny + 2 * R;
#pragma omp parallel for num_threads(nthreads) schedule(static)
  for (int64_t k = R; k < R + nz; k++)
    for (int64_t j = R; j < R + ny; j++)
      for (int64_t i = R; i < R + nx; i++) {
        double cls[4] = {0.0, 0.0, 0.0, 0.0}; /* sums by class: 1 = face, 2 = edge, 3 = corner */
        int first[4] = {1, 1, 1, 1};
        for (int dz = -1; dz <= 1; dz++)
          for (int dy = -1; dy <= 1; dy++)
            for (int dx = -1; dx <= 1; dx++) {
              const int m = (dx != 0) + (dy != 0) + (dz != 0);
              if (m == 0) continue;
              const double v = V[IDX(i + dx, j + dy, k + dz)];
              cls[m] = first[m] ? v : cls[m] + v;
              first[m] = 0;
            }
        U[IDX(i, j, k)] = c[0] * V[IDX(i, j, k)] + c[1] * cls[1] + c[2] * cls[2] + c[3] * cls[3];
      }
}

static void step_rbgs(int64_t nx, int64_t ny, int64_t nz, int64_t ldx, const double* V, double* U,
                      const double* c, int64_t t, int nthreads) {
  const int64_t R = 1, sy = ny + 2 * R;
  const double c0 = c[0], c1 = c[1];
#pragma omp parallel for num_threads(nthreads) schedule(static)
  for (int64_t k = R; k < R + nz; k++)
    for (int64_t j = R; j < R + ny; j++)
      for (int64_t i = R; i < R + nx; i++) {
        const int64_t colour = ((i - R) + (j - R) + (k - R) + t) % 2;
        if (colour != 0) {
          U[IDX(i, j, k)] = V[IDX(i, j, k)];
          continue;
        }
        U[IDX(i, j, k)] = c0 * V[IDX(i, j, k)]
                        + c1 * (V[IDX(i + 1, j, k)] + V[IDX(i - 1, j, k)])
                        + c1 * (V[IDX(i, j + 1, k)] + V[IDX(i, j - 1, k)])
                        + c1 * (V[IDX(i, j, k + 1)] + V[IDX(i, j, k - 1)]);
      }
}

/* Returns 0 on success, 1 on invalid arguments. */
int oracle_sweep(int stencil, int64_t nx, int64_t ny, int64_t nz, int64_t ldx, int64_t T,
                 double* u, double* u_prev, const double* coeffs, const double* c, int nthreads) {
  if (stencil < 0 || stencil > 6 || nx < 1 || ny < 1 || nz < 1 || T < 0 || !u || !u_prev) return 1;
  const int64_t R = (stencil >= 2 && stencil <= 4) ? 4 : 1;
  if (ldx < nx + 2 * R) return 1;
  if ((stencil == 1 || stencil == 3 || stencil == 4) && !coeffs) return 1;
  if ((stencil == 0 || stencil == 2 || stencil == 4 || stencil == 5 || stencil == 6) && !c) return 1;
  if (nthreads < 1) nthreads = 1;
  double* buf[2] = {u, u_prev};
  for (int64_t t = 0; t < T; t++) {
    const double* V = buf[t % 2];
    double* U = buf[(t + 1) % 2];
    switch (stencil) {
      case 0: step_7c(nx, ny, nz, ldx, V, U, c, nthreads); break;
      case 1: step_7v(nx, ny, nz, ldx, V, U, coeffs, nthreads); break;
      case 2: step_25c(nx, ny, nz, ldx, V, U, c, nthreads); break;
      case 3: step_25v(nx, ny, nz, ldx, V, U, coeffs, nthreads); break;
      case 4: step_25cg(nx, ny, nz, ldx, V, U, coeffs, c, nthreads); break;
      case 5: step_27b(nx, ny, nz, ldx, V, U, c, nthreads); break;
      default: step_rbgs(nx, ny, nz, ldx, V, U, c, t, nthreads); break;
    }
  }
  if (T % 2 == 1) { /* level T sits in u_prev: exchange contents so that u holds level T */
    const int64_t n = (nz + 2 * R) * (ny + 2 * R) * ldx;
    for (int64_t p = 0; p < n; p++) {
      const double tmp = u[p];
      u[p] = u_prev[p];
      u_prev[p] = tmp;
    }
  }
  return 0;
}
