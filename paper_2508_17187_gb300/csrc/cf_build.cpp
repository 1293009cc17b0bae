// Host FP64 construction of the convolution functions (PreCompute / ConvFunc, Sec. 4.1 and
// Tab. AWP-CFSETUP of Sec. 6): prolate spheroidal (PS), A-term and W-term screens, Fourier
// transformed to the oversampled uv-plane tables the gridding kernels read.
//
// PS term: psi_0(c, x), the ground state of d/dx[(1 - x^2) psi'] - c^2 x^2 psi = -chi psi on
// [-1, 1], c = pi W / 2.  Expanded in orthonormal even Legendre functions it is the eigenvector
// of the smallest eigenvalue of a symmetric tridiagonal matrix; the eigenvalue is found by
// Sturm-sequence bisection and the eigenvector by shifted inverse iteration (the shift sits
// just below the eigenvalue, so the shifted matrix is positive definite and the tridiagonal
// solve needs no pivoting).
//
// Transform: c(du, dv) = M^-2 sum_ij s[j][i] exp(-2 pi i (du (i - M/2) + dv (j - M/2)) / M) at
// du = S/2 - tx - ox/OS.  Splitting du into (S/2 - ox/OS) and the integer tx turns the sum over
// i, for one offset, into a pre-twiddled length-M inverse FFT whose first S outputs are the S
// taps; rows first, then columns.
#include <cmath>
#include <complex>
#include <vector>

#include "awg_internal.h"

namespace awg {
namespace {

using cd = std::complex<double>;
constexpr double kPi = 3.14159265358979323846;

class Pswf0 {
 public:
  explicit Pswf0(double c, int n_terms = 60) {
    std::vector<double> d(n_terms), e(n_terms - 1);
    const double c2 = c * c;
    for (int m = 0; m < n_terms; ++m) {
      const double n = 2.0 * m;
      d[m] = n * (n + 1.0) + c2 * (2.0 * n * (n + 1.0) - 1.0) / ((2.0 * n + 3.0) * (2.0 * n - 1.0));
      if (m + 1 < n_terms)
        e[m] = c2 * (n + 1.0) * (n + 2.0) / ((2.0 * n + 3.0) * std::sqrt((2.0 * n + 1.0) * (2.0 * n + 5.0)));
    }
    // Gershgorin bounds, then bisection on the Sturm count for the smallest eigenvalue.
    double lo = 1e300, hi = -1e300;
    for (int m = 0; m < n_terms; ++m) {
      double r = (m > 0 ? std::fabs(e[m - 1]) : 0.0) + (m + 1 < n_terms ? std::fabs(e[m]) : 0.0);
      lo = std::fmin(lo, d[m] - r);
      hi = std::fmax(hi, d[m] + r);
    }
    auto count_below = [&](double lam) {
      int cnt = 0;
      double q = d[0] - lam;
      if (q < 0) ++cnt;
      for (int m = 1; m < n_terms; ++m) {
        if (q == 0.0) q = 1e-300;
        q = d[m] - lam - e[m - 1] * e[m - 1] / q;
        if (q < 0) ++cnt;
      }
      return cnt;
    };
    for (int it = 0; it < 200; ++it) {
      double mid = 0.5 * (lo + hi);
      if (count_below(mid) >= 1) hi = mid; else lo = mid;
      if (hi - lo <= 1e-15 * std::fmax(1.0, std::fabs(hi))) break;
    }
    const double chi0 = 0.5 * (lo + hi);
    const double sigma = chi0 - 1e-9 * std::fmax(1.0, std::fabs(chi0));
    std::vector<double> x(n_terms, 1.0), cp(n_terms), dp(n_terms);
    for (int it = 0; it < 4; ++it) {
      // Thomas algorithm for (B - sigma I) y = x (symmetric positive definite).
      double den = d[0] - sigma;
      cp[0] = (n_terms > 1 ? e[0] : 0.0) / den;
      dp[0] = x[0] / den;
      for (int m = 1; m < n_terms; ++m) {
        den = (d[m] - sigma) - e[m - 1] * cp[m - 1];
        cp[m] = (m + 1 < n_terms ? e[m] : 0.0) / den;
        dp[m] = (x[m] - e[m - 1] * dp[m - 1]) / den;
      }
      x[n_terms - 1] = dp[n_terms - 1];
      for (int m = n_terms - 2; m >= 0; --m) x[m] = dp[m] - cp[m] * x[m + 1];
      double nrm = 0.0;
      for (double v : x) nrm += v * v;
      nrm = std::sqrt(nrm);
      for (double& v : x) v /= nrm;
    }
    // Orthonormal Legendre coefficients -> coefficients of P_{2m}.
    a_.resize(n_terms);
    for (int m = 0; m < n_terms; ++m) a_[m] = x[m] * std::sqrt((4.0 * m + 1.0) / 2.0);
    if (eval(0.0) < 0)
      for (double& v : a_) v = -v;
  }

  double eval(double t) const {
    // sum_m a_m P_{2m}(t) by the three-term Legendre recurrence.
    double p_prev = 1.0, p = t, sum = a_[0];
    const int n_max = 2 * (int)a_.size() - 2;
    for (int n = 1; n < n_max; ++n) {
      double p_next = ((2.0 * n + 1.0) * t * p - n * p_prev) / (n + 1.0);
      p_prev = p;
      p = p_next;
      if (((n + 1) & 1) == 0) sum += a_[(n + 1) / 2] * p;
    }
    return sum;
  }

 private:
  std::vector<double> a_;
};

// In-place radix-2 FFT, sum_i b_i exp(+2 pi i k i / M) (unnormalised inverse transform).
void fft_inverse(std::vector<cd>& b) {
  const int M = (int)b.size();
  for (int i = 1, j = 0; i < M; ++i) {
    int bit = M >> 1;
    for (; j & bit; bit >>= 1) j ^= bit;
    j ^= bit;
    if (i < j) std::swap(b[i], b[j]);
  }
  for (int len = 2; len <= M; len <<= 1) {
    const double ang = 2.0 * kPi / len;
    for (int i = 0; i < M; i += len) {
      for (int k = 0; k < len / 2; ++k) {
        const cd w(std::cos(ang * k), std::sin(ang * k));
        cd u = b[i + k], v = b[i + k + len / 2] * w;
        b[i + k] = u + v;
        b[i + k + len / 2] = u - v;
      }
    }
  }
}

cd expi_turns(double t) {  // exp(2 pi i t) with the argument reduced to [-1/2, 1/2] turns first
  t -= std::nearbyint(t);
  return cd(std::cos(2.0 * kPi * t), std::sin(2.0 * kPi * t));
}

double taper_at(const Pswf0& ps, double t, double norm) { return ps.eval(t) / norm; }

}  // namespace

int support_of_plane(const awg_cf_params& p, int ks) {
  if (!p.use_w) return p.max_support;
  const int k = std::abs(ks - (p.n_wplanes - 1));
  const double q = std::sqrt((double)k / (double)(p.n_wplanes - 1));
  int s = 8 * (int)std::ceil((8.0 + (double)(p.max_support - 8) * q) / 8.0);
  if (s > p.max_support) s = p.max_support;
  if (s < p.ps_support) s = p.ps_support;
  return s;
}

int screen_size(int S) {
  int M = 16;
  while (M < 2 * S) M *= 2;
  return M;
}

void taper_image(const awg_cf_params& p, std::vector<double>& out) {
  const int N = p.grid_n;
  out.assign(N, 1.0);
  if (!p.use_ps) return;
  Pswf0 ps(kPi * p.ps_support / 2.0);
  const double norm = ps.eval(0.0);
  for (int j = 0; j < N; ++j) out[j] = taper_at(ps, 2.0 * (double)(j - N / 2) / N, norm);
}

// Airy voltage pattern 2 J1(z) / z of the dish at frequency nu, for the direction (lr, mr) in the
// frame rotated by the parallactic angle, with the elliptical distortion of the A-term.
static double airy_voltage(const awg_cf_params& p, double lr, double mr, double nu) {
  const double a = lr / (1.0 + p.ellipticity), b = mr / (1.0 - p.ellipticity);
  const double z = kPi * p.dish_diameter_m * std::sqrt(a * a + b * b) * nu / kCLight;
  return z != 0.0 ? 2.0 * std::cyl_bessel_j(1.0, z) / z : 1.0;
}

int mueller_elements(const awg_cf_params& p, int* elem_p, int* elem_q) {
  // pol index -> (a, b): RR = (0, 0), RL = (0, 1), LR = (1, 0), LL = (1, 1); R = 0, L = 1
  const double d = std::hypot(p.leakage_re, p.leakage_im);
  int n = 0;
  for (int pp = 0; pp < 4; ++pp)
    for (int qq = 0; qq < 4; ++qq) {
      const int a = pp >> 1, b = pp & 1, c = qq >> 1, e = qq & 1;
      const int n_leak = (a != c) + (b != e);
      const double mag = n_leak == 0 ? 1.0 : std::pow(d, n_leak);
      if (mag >= p.mueller_threshold || n_leak == 0) {
        elem_p[n] = pp;
        elem_q[n] = qq;
        ++n;
      }
    }
  return n;
}

// Image-plane screen s[j][i] = T(x_i) T(y_j) A W at x_i = (i - M/2) N / M pixels (row j: y).  For a
// Mueller element (elem_p, elem_q >= 0) the A factor is J_ac conj(J_bd) with (a, b) the feeds of
// pol elem_p and (c, d) those of elem_q, J = [[A_R, d A_R], [d A_L, A_L]] (A_R, A_L squinted by
// +-squint_rad); otherwise the pol-shared Airy power pattern.
static void cf_screen(const awg_cf_params& p, const double* pa_centers, const double* sb_freqs, int pa, int sb,
                      int ks, int elem_p, int elem_q, int M, std::vector<cd>& scr) {
  const int N = p.grid_n;
  std::vector<double> t1(M, 1.0);
  if (p.use_ps) {
    Pswf0 ps(kPi * p.ps_support / 2.0);
    const double norm = ps.eval(0.0);
    for (int i = 0; i < M; ++i) t1[i] = taper_at(ps, 2.0 * (double)(i - M / 2) / M, norm);
  }
  const double w = p.use_w ? (double)(ks - (p.n_wplanes - 1)) * p.w_max_lambda / (double)(p.n_wplanes - 1) : 0.0;
  scr.assign((size_t)M * M, cd(0.0));
  const double chi = p.use_a ? pa_centers[pa] : 0.0;
  const double cchi = std::cos(chi), schi = std::sin(chi);
  const double nu = p.use_a ? sb_freqs[sb] : 0.0;
  for (int j = 0; j < M; ++j) {
    const double m = (double)(j - M / 2) * N / M * p.cell_rad;
    for (int i = 0; i < M; ++i) {
      const double l = (double)(i - M / 2) * N / M * p.cell_rad;
      cd v(t1[i] * t1[j], 0.0);
      if (p.use_w) {
        const double r2 = l * l + m * m;
        const double nm1 = -r2 / (1.0 + std::sqrt(1.0 - r2));   // sqrt(1 - r^2) - 1 without cancellation
        v *= expi_turns(-w * nm1);
      }
      if (p.use_a) {
        const double lr = l * cchi + m * schi, mr = -l * schi + m * cchi;
        if (elem_p >= 0) {
          const cd dl(p.leakage_re, p.leakage_im);
          const double vr = airy_voltage(p, lr - p.squint_rad, mr, nu);
          const double vl = airy_voltage(p, lr + p.squint_rad, mr, nu);
          // J[x][y]: row x = output feed, column y = sky feed
          const cd J[2][2] = {{cd(vr, 0.0), dl * vr}, {dl * vl, cd(vl, 0.0)}};
          const int a = elem_p >> 1, b = elem_p & 1, c = elem_q >> 1, e = elem_q & 1;
          v *= J[a][c] * std::conj(J[b][e]);
        } else {
          const double amp = airy_voltage(p, lr, mr, nu);
          v *= amp * amp;
        }
      }
      scr[(size_t)j * M + i] = v;
    }
  }
}

// Twiddles of the axis transform: tw[o][i] = exp(-2 pi i (S/2 - o/OS) (i - M/2) / M).
static void axis_twiddles(int M, int S, int OS, std::vector<cd>& tw) {
  tw.resize((size_t)(OS + 1) * M);
  for (int o = 0; o <= OS; ++o) {
    const double shift = 0.5 * S - (double)o / OS;
    for (int i = 0; i < M; ++i) tw[(size_t)o * M + i] = expi_turns(-shift * (double)(i - M / 2) / M);
  }
}

// One axis of the CF transform: out[o][t] = (1/M) (-1)^t sum_i v_i tw[o][i] exp(2 pi i t i / M), the
// taps t < S of the screen row v at oversampling offset o (shift S/2 - o/OS pixels).
static void axis_transform(const cd* v, int M, int S, int OS, const std::vector<cd>& tw, cd* out) {
  std::vector<cd> b(M);
  for (int o = 0; o <= OS; ++o) {
    for (int i = 0; i < M; ++i) b[i] = v[i] * tw[(size_t)o * M + i];
    fft_inverse(b);
    for (int t = 0; t < S; ++t) out[(size_t)o * S + t] = b[t] * ((t & 1) ? -1.0 : 1.0) / (double)M;
  }
}

void build_cf_table(const awg_cf_params& p, const double* pa_centers, const double* sb_freqs, int pa,
                    int sb, int ks, std::vector<double>& out) {
  const int S = support_of_plane(p, ks);
  const int M = screen_size(S);
  const int OS = p.oversampling;
  std::vector<cd> scr, tw;
  cf_screen(p, pa_centers, sb_freqs, pa, sb, ks, -1, -1, M, scr);
  axis_twiddles(M, S, OS, tw);
  // Pass over rows (u): X[ox][j][tx].
  const int Q = (OS + 1) * S;
  std::vector<cd> X((size_t)(OS + 1) * M * S), row(Q), col(M), colt(Q);
  for (int j = 0; j < M; ++j) {
    axis_transform(&scr[(size_t)j * M], M, S, OS, tw, row.data());
    for (int ox = 0; ox <= OS; ++ox)
      for (int tx = 0; tx < S; ++tx) X[((size_t)ox * M + j) * S + tx] = row[(size_t)ox * S + tx];
  }
  // Pass over columns (v): out[oy][ox][ty][tx].
  out.assign((size_t)2 * (OS + 1) * (OS + 1) * S * S, 0.0);
  for (int ox = 0; ox <= OS; ++ox) {
    for (int tx = 0; tx < S; ++tx) {
      for (int j = 0; j < M; ++j) col[j] = X[((size_t)ox * M + j) * S + tx];
      axis_transform(col.data(), M, S, OS, tw, colt.data());
      for (int oy = 0; oy <= OS; ++oy)
        for (int ty = 0; ty < S; ++ty) {
          const cd c = colt[(size_t)oy * S + ty];
          const size_t at = ((((size_t)oy * (OS + 1) + ox) * S + ty) * S + tx) * 2;
          out[at] = c.real();
          out[at + 1] = c.imag();
        }
    }
  }
}

// Greedy rank-1 terms of a rows x cols matrix E (row-major), subtracted in place: alternating
// least squares from the strongest column (power iteration on E^H E) for the leading pair.
static void leading_term(std::vector<cd>& E, int rows, int cols, std::vector<cd>& g, std::vector<cd>& f) {
  g.assign(rows, cd(0.0));
  f.assign(cols, cd(0.0));
  double emax = 0.0;
  int jbest = 0;
  for (size_t i = 0; i < E.size(); ++i) {
    const double a = std::abs(E[i]);
    if (a > emax) { emax = a; jbest = (int)(i % cols); }
  }
  if (emax == 0.0) return;
  for (int r = 0; r < rows; ++r) g[r] = E[(size_t)r * cols + jbest];
  double prev = 0.0;
  for (int it = 0; it < 40; ++it) {
    double gg = 0.0;
    for (const cd& v : g) gg += std::norm(v);
    std::fill(f.begin(), f.end(), cd(0.0));
    for (int r = 0; r < rows; ++r) {
      const cd cg = std::conj(g[r]);
      const cd* e = &E[(size_t)r * cols];
      for (int c = 0; c < cols; ++c) f[c] += cg * e[c];
    }
    for (cd& v : f) v /= gg;
    double ff = 0.0;
    for (const cd& v : f) ff += std::norm(v);
    double g2 = 0.0;
    for (int r = 0; r < rows; ++r) {
      cd acc = 0.0;
      const cd* e = &E[(size_t)r * cols];
      for (int c = 0; c < cols; ++c) acc += e[c] * std::conj(f[c]);
      g[r] = acc / ff;
      g2 += std::norm(g[r]);
    }
    const double sigma = std::sqrt(g2 * ff);
    if (it >= 3 && std::fabs(sigma - prev) <= 1e-13 * sigma) break;
    prev = sigma;
  }
  for (int r = 0; r < rows; ++r) {
    cd* e = &E[(size_t)r * cols];
    for (int c = 0; c < cols; ++c) e[c] -= g[r] * f[c];
  }
}

int build_cf_factors(const awg_cf_params& p, const double* pa_centers, const double* sb_freqs, int pa, int sb,
                     int ks, int elem_p, int elem_q, double tol, int r_max, std::vector<double>& fx,
                     std::vector<double>& fy) {
  // The CF is the 2-D transform of the screen, separable as C = Fy scr Fx^T with one axis
  // transform per axis; a term g f^T of the screen therefore gives the CF term (Fy g)(Fx f)^T.
  // Terms are taken greedily from the screen's residual; after each term the CF residual is
  // evaluated on the offset slices (oy, ox) in {0, OS/2, OS}^2 (each S x S: the CF's own slices,
  // computed directly from the screen, minus the terms so far) and the fit stops once it is
  // within tol of the CF's peak there.
  const int S = support_of_plane(p, ks);
  const int M = screen_size(S);
  const int OS = p.oversampling;
  const int Q = (OS + 1) * S;
  std::vector<cd> E, tw;
  cf_screen(p, pa_centers, sb_freqs, pa, sb, ks, elem_p, elem_q, M, E);
  axis_twiddles(M, S, OS, tw);
  // axis transform as explicit rows for the checked offsets: Fo[t][i]
  const int chk[3] = {0, OS / 2, OS};
  std::vector<cd> Fo((size_t)3 * S * M);
  {
    std::vector<cd> e(M, cd(0.0)), o((size_t)Q);
    for (int i = 0; i < M; ++i) {
      e[i] = 1.0;
      axis_transform(e.data(), M, S, OS, tw, o.data());
      for (int c = 0; c < 3; ++c)
        for (int t = 0; t < S; ++t) Fo[((size_t)c * S + t) * M + i] = o[(size_t)chk[c] * S + t];
      e[i] = 0.0;
    }
  }
  // slices of a screen-space matrix: out[cy][cx][ty][tx] = sum_j Fo[cy][ty][j] sum_i Z[j][i] Fo[cx][tx][i]
  auto slices = [&](const std::vector<cd>& Z, std::vector<cd>& out) {
    std::vector<cd> A((size_t)3 * M * S, cd(0.0));   // A[cx][j][tx]
    for (int cx = 0; cx < 3; ++cx)
      for (int j = 0; j < M; ++j)
        for (int tx = 0; tx < S; ++tx) {
          cd acc = 0.0;
          const cd* z = &Z[(size_t)j * M];
          const cd* fo = &Fo[((size_t)cx * S + tx) * M];
          for (int i = 0; i < M; ++i) acc += z[i] * fo[i];
          A[((size_t)cx * M + j) * S + tx] = acc;
        }
    out.assign((size_t)9 * S * S, cd(0.0));
    for (int cy = 0; cy < 3; ++cy)
      for (int cx = 0; cx < 3; ++cx)
        for (int ty = 0; ty < S; ++ty) {
          const cd* fo = &Fo[((size_t)cy * S + ty) * M];
          for (int tx = 0; tx < S; ++tx) {
            cd acc = 0.0;
            for (int j = 0; j < M; ++j) acc += fo[j] * A[((size_t)cx * M + j) * S + tx];
            out[(((size_t)cy * 3 + cx) * S + ty) * S + tx] = acc;
          }
        }
  };
  std::vector<cd> sl;
  slices(E, sl);
  double peak = 0.0;
  for (const cd& v : sl) peak = std::fmax(peak, std::abs(v));
  fx.clear();
  fy.clear();
  if (peak == 0.0) {   // an all-zero CF (e.g. a leakage element with d = 0): one zero term
    fx.assign(2 * (size_t)Q, 0.0);
    fy.assign(2 * (size_t)Q, 0.0);
    return 1;
  }
  std::vector<cd> g, f, tg(Q), tf(Q);
  for (int r = 0; r < r_max; ++r) {
    leading_term(E, M, M, g, f);
    axis_transform(g.data(), M, S, OS, tw, tg.data());
    axis_transform(f.data(), M, S, OS, tw, tf.data());
    for (int q = 0; q < Q; ++q) {
      fx.push_back(tf[q].real());
      fx.push_back(tf[q].imag());
    }
    for (int q = 0; q < Q; ++q) {
      fy.push_back(tg[q].real());
      fy.push_back(tg[q].imag());
    }
    // the term's own slices are outer products of its transformed factors
    double res = 0.0;
    for (int cy = 0; cy < 3; ++cy)
      for (int cx = 0; cx < 3; ++cx)
        for (int ty = 0; ty < S; ++ty)
          for (int tx = 0; tx < S; ++tx) {
            cd& v = sl[(((size_t)cy * 3 + cx) * S + ty) * S + tx];
            v -= tg[(size_t)chk[cy] * S + ty] * tf[(size_t)chk[cx] * S + tx];
            res = std::fmax(res, std::abs(v));
          }
    if (res <= tol * peak) return r + 1;
  }
  fx.clear();
  fy.clear();
  return 0;
}

int factor_low_rank(const std::vector<double>& tab, int S, int OS, double tol, int r_max, std::vector<double>& fx,
                    std::vector<double>& fy) {
  // The table seen as a Q x Q matrix C[(oy, ty)][(ox, tx)], Q = (OS + 1) S.  A separable CF
  // c(du, dv) = g(dv) f(du) makes C = g f^T; a sum of r such terms makes C = sum_k g_k f_k^T.
  // Terms are taken greedily from the residual E (starting at E = C): alternating least squares
  // from E's strongest column (power iteration on E^H E) gives the leading pair, which is
  // subtracted.  The fit stops at the first r with max |E| <= tol max |C|.
  const int Q = (OS + 1) * S;
  std::vector<cd> E((size_t)Q * Q);
  double cmax = 0.0;
  for (int oy = 0; oy <= OS; ++oy)
    for (int ox = 0; ox <= OS; ++ox)
      for (int ty = 0; ty < S; ++ty)
        for (int tx = 0; tx < S; ++tx) {
          const size_t i = ((((size_t)oy * (OS + 1) + ox) * S + ty) * S + tx) * 2;
          const cd v(tab[i], tab[i + 1]);
          E[(size_t)(oy * S + ty) * Q + ox * S + tx] = v;
          cmax = std::fmax(cmax, std::abs(v));
        }
  fx.clear();
  fy.clear();
  if (cmax == 0.0) {   // the zero table: one zero term
    fx.assign(2 * (size_t)Q, 0.0);
    fy.assign(2 * (size_t)Q, 0.0);
    return 1;
  }
  std::vector<cd> g(Q), f(Q);
  for (int r = 0; r < r_max; ++r) {
    double emax = 0.0;
    int jbest = 0;
    for (size_t i = 0; i < E.size(); ++i) {
      const double a = std::abs(E[i]);
      if (a > emax) { emax = a; jbest = (int)(i % Q); }
    }
    for (int qy = 0; qy < Q; ++qy) g[qy] = E[(size_t)qy * Q + jbest];
    double prev = 0.0;
    for (int it = 0; it < 40; ++it) {
      double gg = 0.0;
      for (const cd& v : g) gg += std::norm(v);
      std::fill(f.begin(), f.end(), cd(0.0));
      for (int qy = 0; qy < Q; ++qy) {
        const cd cg = std::conj(g[qy]);
        const cd* row = &E[(size_t)qy * Q];
        for (int qx = 0; qx < Q; ++qx) f[qx] += cg * row[qx];
      }
      for (cd& v : f) v /= gg;
      double ff = 0.0;
      for (const cd& v : f) ff += std::norm(v);
      for (int qy = 0; qy < Q; ++qy) {
        cd acc = 0.0;
        const cd* row = &E[(size_t)qy * Q];
        for (int qx = 0; qx < Q; ++qx) acc += row[qx] * std::conj(f[qx]);
        g[qy] = acc / ff;
      }
      // sigma of the current pair; stop once it no longer moves
      double g2 = 0.0;
      for (const cd& v : g) g2 += std::norm(v);
      const double sigma = std::sqrt(g2 * ff);
      if (it >= 3 && std::fabs(sigma - prev) <= 1e-13 * sigma) break;
      prev = sigma;
    }
    // balance the two factors' magnitudes
    double gm = 0.0, fm = 0.0;
    for (const cd& v : g) gm = std::fmax(gm, std::abs(v));
    for (const cd& v : f) fm = std::fmax(fm, std::abs(v));
    if (gm > 0.0 && fm > 0.0) {
      const double sc = std::sqrt(fm / gm);
      for (cd& v : g) v *= sc;
      for (cd& v : f) v /= sc;
    }
    double res = 0.0;
    for (int qy = 0; qy < Q; ++qy) {
      cd* row = &E[(size_t)qy * Q];
      for (int qx = 0; qx < Q; ++qx) {
        row[qx] -= g[qy] * f[qx];
        res = std::fmax(res, std::abs(row[qx]));
      }
    }
    for (int q = 0; q < Q; ++q) {
      fx.push_back(f[q].real());
      fx.push_back(f[q].imag());
    }
    for (int q = 0; q < Q; ++q) {
      fy.push_back(g[q].real());
      fy.push_back(g[q].imag());
    }
    if (res <= tol * cmax) return r + 1;
  }
  fx.clear();
  fy.clear();
  return 0;
}

}  // namespace awg
