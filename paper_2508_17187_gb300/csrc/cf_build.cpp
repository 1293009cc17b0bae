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

void build_cf_table(const awg_cf_params& p, const double* pa_centers, const double* sb_freqs, int pa,
                    int sb, int ks, std::vector<double>& out) {
  const int S = support_of_plane(p, ks);
  const int M = screen_size(S);
  const int OS = p.oversampling;
  const int N = p.grid_n;
  // Image-plane screen s[j][i]: T(x_i) T(y_j) A W at x_i = (i - M/2) N / M pixels.
  std::vector<double> t1(M, 1.0);
  if (p.use_ps) {
    Pswf0 ps(kPi * p.ps_support / 2.0);
    const double norm = ps.eval(0.0);
    for (int i = 0; i < M; ++i) t1[i] = taper_at(ps, 2.0 * (double)(i - M / 2) / M, norm);
  }
  const double w = p.use_w ? (double)(ks - (p.n_wplanes - 1)) * p.w_max_lambda / (double)(p.n_wplanes - 1) : 0.0;
  std::vector<cd> scr((size_t)M * M);
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
        const double a = lr / (1.0 + p.ellipticity), b = mr / (1.0 - p.ellipticity);
        const double z = kPi * p.dish_diameter_m * std::sqrt(a * a + b * b) * nu / kCLight;
        double amp = 1.0;
        if (z != 0.0) {
          const double j1 = std::cyl_bessel_j(1.0, z);
          amp = (2.0 * j1 / z) * (2.0 * j1 / z);
        }
        v *= amp;
      }
      scr[(size_t)j * M + i] = v;
    }
  }
  // Pass over rows (u): X[ox][j][tx].
  std::vector<cd> X((size_t)(OS + 1) * M * S), b(M), tw(M);
  for (int ox = 0; ox <= OS; ++ox) {
    const double shift = 0.5 * S - (double)ox / OS;
    for (int i = 0; i < M; ++i) tw[i] = expi_turns(-shift * (double)(i - M / 2) / M);
    for (int j = 0; j < M; ++j) {
      for (int i = 0; i < M; ++i) b[i] = scr[(size_t)j * M + i] * tw[i];
      fft_inverse(b);
      for (int tx = 0; tx < S; ++tx) X[((size_t)ox * M + j) * S + tx] = b[tx] * ((tx & 1) ? -1.0 : 1.0) / (double)M;
    }
  }
  // Pass over columns (v): out[oy][ox][ty][tx].
  out.assign((size_t)2 * (OS + 1) * (OS + 1) * S * S, 0.0);
  for (int oy = 0; oy <= OS; ++oy) {
    const double shift = 0.5 * S - (double)oy / OS;
    for (int j = 0; j < M; ++j) tw[j] = expi_turns(-shift * (double)(j - M / 2) / M);
    for (int ox = 0; ox <= OS; ++ox) {
      for (int tx = 0; tx < S; ++tx) {
        for (int j = 0; j < M; ++j) b[j] = X[((size_t)ox * M + j) * S + tx] * tw[j];
        fft_inverse(b);
        for (int ty = 0; ty < S; ++ty) {
          const cd c = b[ty] * ((ty & 1) ? -1.0 : 1.0) / (double)M;
          const size_t at = ((((size_t)oy * (OS + 1) + ox) * S + ty) * S + tx) * 2;
          out[at] = c.real();
          out[at + 1] = c.imag();
        }
      }
    }
  }
}

bool factor_rank1(const std::vector<double>& tab, int S, int OS, double tol, std::vector<double>& fx,
                  std::vector<double>& fy) {
  // The table seen as a Q x Q matrix C[(oy, ty)][(ox, tx)], Q = (OS + 1) S.  A separable CF
  // c(du, dv) = g(dv) f(du) makes C = g f^T; alternating least squares from the strongest column
  // finds g and f, and the fit is accepted when max |C - g f^T| <= tol max |C|.
  const int Q = (OS + 1) * S;
  auto at = [&](int qy, int qx) {
    const int oy = qy / S, ty = qy - oy * S, ox = qx / S, tx = qx - ox * S;
    const size_t i = ((((size_t)oy * (OS + 1) + ox) * S + ty) * S + tx) * 2;
    return cd(tab[i], tab[i + 1]);
  };
  double cmax = 0.0;
  int jbest = 0;
  for (int qy = 0; qy < Q; ++qy)
    for (int qx = 0; qx < Q; ++qx) {
      const double a = std::abs(at(qy, qx));
      if (a > cmax) { cmax = a; jbest = qx; }
    }
  if (cmax == 0.0) return false;
  std::vector<cd> g(Q), f(Q);
  for (int qy = 0; qy < Q; ++qy) g[qy] = at(qy, jbest);
  for (int it = 0; it < 4; ++it) {
    double gg = 0.0;
    for (const cd& v : g) gg += std::norm(v);
    for (int qx = 0; qx < Q; ++qx) {
      cd acc = 0.0;
      for (int qy = 0; qy < Q; ++qy) acc += std::conj(g[qy]) * at(qy, qx);
      f[qx] = acc / gg;
    }
    double ff = 0.0;
    for (const cd& v : f) ff += std::norm(v);
    for (int qy = 0; qy < Q; ++qy) {
      cd acc = 0.0;
      for (int qx = 0; qx < Q; ++qx) acc += at(qy, qx) * std::conj(f[qx]);
      g[qy] = acc / ff;
    }
  }
  // balance the two factors' magnitudes
  double gm = 0.0, fm = 0.0;
  for (const cd& v : g) gm = std::fmax(gm, std::abs(v));
  for (const cd& v : f) fm = std::fmax(fm, std::abs(v));
  const double sc = std::sqrt(fm / gm);
  for (cd& v : g) v *= sc;
  for (cd& v : f) v /= sc;
  double res = 0.0;
  for (int qy = 0; qy < Q; ++qy)
    for (int qx = 0; qx < Q; ++qx) res = std::fmax(res, std::abs(at(qy, qx) - g[qy] * f[qx]));
  if (res > tol * cmax) return false;
  fx.resize(2 * (size_t)Q);
  fy.resize(2 * (size_t)Q);
  for (int q = 0; q < Q; ++q) {
    fx[2 * q] = f[q].real();
    fx[2 * q + 1] = f[q].imag();
    fy[2 * q] = g[q].real();
    fy[2 * q + 1] = g[q].imag();
  }
  return true;
}

}  // namespace awg
