/*
 * FP64 CPU oracle loops for gridding (G) and degridding (D).  TEST INFRASTRUCTURE ONLY:
 * nothing in the library links or calls this file.
 *
 * G, Eq. IMAGE-MOD (Sec. 2):  grid[p0y+ty][p0x+tx][p] += conj(CF[oy][ox][ty][tx]) * w[p] * V[p]
 * D, Eq. ME-MOD-GRIDDED:      V[p] = sum_{ty,tx} CF[oy][ox][ty][tx] * grid[p0y+ty][p0x+tx][p]
 * for every kept sample, with the optional phase-centre phasor of Eq. CIJ multiplied
 * into w V before G and, conjugated, into V after D.  Complex numbers are interleaved
 * (re, im) doubles.  Gridding splits the grid into row stripes, one per thread, and
 * every thread walks all samples in order, so each pixel is summed in sample order
 * whatever the thread count.  Degridding splits the samples.  Build with
 * -ffp-contract=off so that no multiply-add is fused.
 */
#include <stdint.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

void oracle_grid_rows(int64_t n, const uint8_t* valid, const int32_t* cf, const int64_t* p0x,
                      const int64_t* p0y, const int32_t* ox, const int32_t* oy, const int32_t* support,
                      const double* phasor, int P, const double* vis, const double* wt, const int64_t* cf_off,
                      int OS, const double* cf_data, int N, int64_t row_lo, int64_t row_hi,
                      double* band /* [row_hi - row_lo][N][P][2], accumulated */, int nthreads);

void oracle_grid(int64_t n, const uint8_t* valid, const int32_t* cf, const int64_t* p0x,
                 const int64_t* p0y, const int32_t* ox, const int32_t* oy, const int32_t* support,
                 const double* phasor /* [n][2] or NULL */, int P, const double* vis /* [n][P][2] */,
                 const double* wt /* [n][P] */, const int64_t* cf_off, int OS, const double* cf_data,
                 int N, double* grid /* [N][N][P][2], accumulated */, double* sumwt /* [P] */,
                 int nthreads) {
  for (int64_t s = 0; s < n; ++s) {
    if (!valid[s]) continue;
    for (int p = 0; p < P; ++p) sumwt[p] += wt[s * P + p];
  }
  oracle_grid_rows(n, valid, cf, p0x, p0y, ox, oy, support, phasor, P, vis, wt, cf_off, OS, cf_data, N, 0, N,
                   grid, nthreads);
}

/* G restricted to grid rows [row_lo, row_hi): the same sums, for one band of the grid. */
void oracle_grid_rows(int64_t n, const uint8_t* valid, const int32_t* cf, const int64_t* p0x,
                      const int64_t* p0y, const int32_t* ox, const int32_t* oy, const int32_t* support,
                      const double* phasor, int P, const double* vis, const double* wt, const int64_t* cf_off,
                      int OS, const double* cf_data, int N, int64_t row_lo, int64_t row_hi, double* band,
                      int nthreads) {
#pragma omp parallel num_threads(nthreads)
  {
    int nt = 1, tid = 0;
#ifdef _OPENMP
    nt = omp_get_num_threads();
    tid = omp_get_thread_num();
#endif
    const int64_t span = row_hi - row_lo;
    int64_t y_lo = row_lo + span * tid / nt, y_hi = row_lo + span * (tid + 1) / nt;
    for (int64_t s = 0; s < n; ++s) {
      if (!valid[s]) continue;
      int S = support[s];
      int64_t y0 = p0y[s];
      if (y0 + S <= y_lo || y0 >= y_hi) continue;
      double a_re[4], a_im[4];
      for (int p = 0; p < P; ++p) {
        double vr = vis[(s * P + p) * 2], vi = vis[(s * P + p) * 2 + 1];
        double w = wt[s * P + p];
        double xr = w * vr, xi = w * vi;
        if (phasor) {
          double cr = phasor[2 * s], ci = phasor[2 * s + 1];
          double t = xr * cr - xi * ci;
          xi = xr * ci + xi * cr;
          xr = t;
        }
        a_re[p] = xr;
        a_im[p] = xi;
      }
      const double* tab = cf_data + 2 * (cf_off[cf[s]] + ((int64_t)oy[s] * (OS + 1) + ox[s]) * S * S);
      for (int ty = 0; ty < S; ++ty) {
        int64_t y = y0 + ty;
        if (y < y_lo || y >= y_hi) continue;
        for (int tx = 0; tx < S; ++tx) {
          double cr = tab[2 * (ty * S + tx)], ci = -tab[2 * (ty * S + tx) + 1];   /* conj(CF) */
          double* g = band + (((y - row_lo) * N + p0x[s] + tx) * P) * 2;
          for (int p = 0; p < P; ++p) {
            g[2 * p] += cr * a_re[p] - ci * a_im[p];
            g[2 * p + 1] += cr * a_im[p] + ci * a_re[p];
          }
        }
      }
    }
  }
}

void oracle_degrid(int64_t n, const uint8_t* valid, const int32_t* cf, const int64_t* p0x,
                   const int64_t* p0y, const int32_t* ox, const int32_t* oy, const int32_t* support,
                   const double* phasor, int P, const int64_t* cf_off, int OS, const double* cf_data,
                   int N, const double* grid, double* vis_out /* [n][P][2], overwritten */,
                   int nthreads) {
#pragma omp parallel for schedule(dynamic, 256) num_threads(nthreads)
  for (int64_t s = 0; s < n; ++s) {
    double acc_re[4] = {0, 0, 0, 0}, acc_im[4] = {0, 0, 0, 0};
    if (valid[s]) {
      int S = support[s];
      const double* tab = cf_data + 2 * (cf_off[cf[s]] + ((int64_t)oy[s] * (OS + 1) + ox[s]) * S * S);
      for (int ty = 0; ty < S; ++ty) {
        for (int tx = 0; tx < S; ++tx) {
          double cr = tab[2 * (ty * S + tx)], ci = tab[2 * (ty * S + tx) + 1];
          const double* g = grid + (((p0y[s] + ty) * N + p0x[s] + tx) * P) * 2;
          for (int p = 0; p < P; ++p) {
            acc_re[p] += cr * g[2 * p] - ci * g[2 * p + 1];
            acc_im[p] += cr * g[2 * p + 1] + ci * g[2 * p];
          }
        }
      }
      if (phasor) {
        double cr = phasor[2 * s], ci = -phasor[2 * s + 1];   /* conj(phasor) */
        for (int p = 0; p < P; ++p) {
          double t = acc_re[p] * cr - acc_im[p] * ci;
          acc_im[p] = acc_re[p] * ci + acc_im[p] * cr;
          acc_re[p] = t;
        }
      }
    }
    for (int p = 0; p < P; ++p) {
      vis_out[(s * P + p) * 2] = acc_re[p];
      vis_out[(s * P + p) * 2 + 1] = acc_im[p];
    }
  }
}
