// FP64 CPU oracle of the strong-lens log-posterior.
//
// TEST INFRASTRUCTURE ONLY. This file is the plain, slow, obviously correct
// definition that the CUDA path is checked against. Only the test suite, the
// smoke check and the CPU-baseline leg of the benchmark load it. It shares no
// code, header, table or helper with the CUDA library, and the library never
// calls it.
//
// Every quantity is double precision. The gradient is forward-mode automatic
// differentiation with dual numbers (one partial per parameter), so it is
// independent of the CUDA path's hand-written adjoint.
//
// What is computed (the paper defers the model to its predecessor; the
// readings below are those of the lensing literature, named where used):
//   * Grid: pixel (i, j) has centre x = (j - (nx-1)/2) D, y = (i - (ny-1)/2) D
//     (D = pixel scale); sub-pixel (k, l) of supersampling s is offset by
//     ((l + 1/2)/s - 1/2) D in x and ((k + 1/2)/s - 1/2) D in y.
//   * Ellipticity (e1, e2): position angle phi = atan2(e2, e1)/2, c = |e|,
//     axis ratio q = (1 - c)/(1 + c); lens frame x' = cos(phi) dx + sin(phi) dy,
//     y' = -sin(phi) dx + cos(phi) dy about the component's centre.
//   * EPL mass (Sec. 3, parameters theta_E, gamma, e1, e2, x, y), deflection
//     after Tessore & Metcalf (2015): t = gamma - 1, b = theta_E sqrt(q),
//     R = sqrt(q^2 x'^2 + y'^2), e^{i varphi} = (q x' + i y')/R,
//     f = (1-q)/(1+q), alpha' = 2b/(1+q) (b/R)^(t-1) Sum_n Omega_n with
//     Omega_0 = e^{i varphi} and Omega_n = -f (2n-(2-t))/(2n+(2-t))
//     e^{2 i varphi} Omega_{n-1}; alpha' is rotated back by +phi. The
//     convergence this deflects with is kappa = (2-t)/2 (b/R)^t.
//     The sum stops once the tail bound (N+2)^2 f^N/(1-f)^2 is below 1e-17.
//   * External shear (Sec. 3): alpha = (g1 x + g2 y, g2 x - g1 y), origin-centred.
//   * Elliptical Sersic light (lens light on the image plane, source light on
//     the source plane beta = theta - alpha): R = sqrt(q x'^2 + y'^2/q),
//     I = I_e exp(-b_n ((R/R_e)^(1/n) - 1)), b_n = 1.9992 n - 0.3271
//     (Capaccioli 1989); I_e is the half-light intensity (Eq. sim-dist).
//   * Both radii are clamped below at R_MIN = 1e-6 arcsec.
//   * Binning: model pixel = D^2 x mean over the s x s sub-pixels.
//   * PSF: true 2-D convolution ("same" size, zero padding), PSF normalised
//     to unit sum.
//   * Likelihood: log L = -1/2 Sum ((d - m)/sigma)^2 with a fixed noise map.
//   * Prior (Eq. sim-dist): sum of normalised 1-D log densities; |e| < emax
//     pairs restrict the support only. Outside the support, or outside the
//     model's domain (theta_E > 0, 1 < gamma < 3, every |e| < 0.8, R_e > 0,
//     n >= 0.2), log p = -inf and its gradient is 0. A NaN parameter gives NaN.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <limits>
#include <vector>
#ifdef _OPENMP
#include <omp.h>
#endif

namespace {

constexpr double R_MIN = 1e-6;
constexpr double E_DOMAIN = 0.8;
constexpr double N_MIN = 0.2;
constexpr double SERIES_TOL = 1e-17;
constexpr double PI = 3.14159265358979323846;

// ------------------------------------------------------------ dual numbers
template <int NP>
struct Dual {
  double v;
  double d[NP];
};

inline double val(double x) { return x; }
template <int NP> inline double val(const Dual<NP>& x) { return x.v; }

template <int NP> inline Dual<NP> cst(double v) {
  Dual<NP> r;
  r.v = v;
  for (int i = 0; i < NP; ++i) r.d[i] = 0.0;
  return r;
}
// r = function value v with derivative dv/da, chained through a
template <int NP> inline Dual<NP> chain(const Dual<NP>& a, double v, double dvda) {
  Dual<NP> r;
  r.v = v;
  for (int i = 0; i < NP; ++i) r.d[i] = dvda * a.d[i];
  return r;
}
template <int NP> inline Dual<NP> operator+(const Dual<NP>& a, const Dual<NP>& b) {
  Dual<NP> r; r.v = a.v + b.v;
  for (int i = 0; i < NP; ++i) r.d[i] = a.d[i] + b.d[i];
  return r;
}
template <int NP> inline Dual<NP> operator-(const Dual<NP>& a, const Dual<NP>& b) {
  Dual<NP> r; r.v = a.v - b.v;
  for (int i = 0; i < NP; ++i) r.d[i] = a.d[i] - b.d[i];
  return r;
}
template <int NP> inline Dual<NP> operator*(const Dual<NP>& a, const Dual<NP>& b) {
  Dual<NP> r; r.v = a.v * b.v;
  for (int i = 0; i < NP; ++i) r.d[i] = a.d[i] * b.v + a.v * b.d[i];
  return r;
}
template <int NP> inline Dual<NP> operator/(const Dual<NP>& a, const Dual<NP>& b) {
  Dual<NP> r; r.v = a.v / b.v;
  for (int i = 0; i < NP; ++i) r.d[i] = (a.d[i] * b.v - a.v * b.d[i]) / (b.v * b.v);
  return r;
}
template <int NP> inline Dual<NP> operator-(const Dual<NP>& a) {
  Dual<NP> r; r.v = -a.v;
  for (int i = 0; i < NP; ++i) r.d[i] = -a.d[i];
  return r;
}
template <int NP> inline Dual<NP> operator+(const Dual<NP>& a, double b) { Dual<NP> r = a; r.v += b; return r; }
template <int NP> inline Dual<NP> operator+(double a, const Dual<NP>& b) { return b + a; }
template <int NP> inline Dual<NP> operator-(const Dual<NP>& a, double b) { Dual<NP> r = a; r.v -= b; return r; }
template <int NP> inline Dual<NP> operator-(double a, const Dual<NP>& b) { return -b + a; }
template <int NP> inline Dual<NP> operator*(const Dual<NP>& a, double b) {
  Dual<NP> r; r.v = a.v * b;
  for (int i = 0; i < NP; ++i) r.d[i] = a.d[i] * b;
  return r;
}
template <int NP> inline Dual<NP> operator*(double a, const Dual<NP>& b) { return b * a; }
template <int NP> inline Dual<NP> operator/(const Dual<NP>& a, double b) { return a * (1.0 / b); }
template <int NP> inline Dual<NP> operator/(double a, const Dual<NP>& b) {
  return chain(b, a / b.v, -a / (b.v * b.v));
}
template <int NP> inline Dual<NP> exp(const Dual<NP>& a) { double e = std::exp(a.v); return chain(a, e, e); }
template <int NP> inline Dual<NP> log(const Dual<NP>& a) { return chain(a, std::log(a.v), 1.0 / a.v); }
template <int NP> inline Dual<NP> sqrt(const Dual<NP>& a) {
  double s = std::sqrt(a.v); return chain(a, s, 0.5 / s);
}
template <int NP> inline Dual<NP> sin(const Dual<NP>& a) { return chain(a, std::sin(a.v), std::cos(a.v)); }
template <int NP> inline Dual<NP> cos(const Dual<NP>& a) { return chain(a, std::cos(a.v), -std::sin(a.v)); }
template <int NP> inline Dual<NP> atan2(const Dual<NP>& y, const Dual<NP>& x) {
  Dual<NP> r; r.v = std::atan2(y.v, x.v);
  double den = x.v * x.v + y.v * y.v;
  for (int i = 0; i < NP; ++i) r.d[i] = (x.v * y.d[i] - y.v * x.d[i]) / den;
  return r;
}
// a^b for a > 0, both dual
template <int NP> inline Dual<NP> pow(const Dual<NP>& a, const Dual<NP>& b) { return exp(b * log(a)); }

using std::atan2;
using std::cos;
using std::exp;
using std::log;
using std::pow;
using std::sin;
using std::sqrt;

// a value clamped below at lo; the clamped branch is a constant
inline double clamp_below(double a, double lo) { return a < lo ? lo : a; }
template <int NP> inline Dual<NP> clamp_below(const Dual<NP>& a, double lo) {
  return a.v < lo ? cst<NP>(lo) : a;
}
template <class T> inline T zero_like(const T&) { return T(0.0); }
template <int NP> inline Dual<NP> zero_like(const Dual<NP>&) { return cst<NP>(0.0); }
template <class T> inline T as_T(double v, const T& like) { return zero_like(like) + v; }

template <class T> struct Cx { T re, im; };
template <class T> inline Cx<T> cmul(const Cx<T>& a, const Cx<T>& b) {
  return {a.re * b.re - a.im * b.im, a.re * b.im + a.im * b.re};
}

// ------------------------------------------------------------------ model
// Ellipticity to axis ratio and position angle.
template <class T> inline void ellipticity(const T& e1, const T& e2, T& q, T& phi) {
  T c = sqrt(e1 * e1 + e2 * e2);
  q = (1.0 - c) / (1.0 + c);
  phi = 0.5 * atan2(e2, e1);
}

// Number of series terms: tail bound (N+2)^2 f^N/(1-f)^2 below SERIES_TOL
// (it bounds the tails of the sum and of its first derivatives).
inline int series_terms(double f) {
  int n = 0;
  while ((n + 2.0) * (n + 2.0) * std::pow(f, n) / ((1.0 - f) * (1.0 - f)) >= SERIES_TOL) ++n;
  return n;
}

// Sum_n Omega_n for t, f and e^{i varphi} (Tessore & Metcalf 2015).
template <class T>
Cx<T> epl_series(const T& t, const T& f, const Cx<T>& eiv) {
  Cx<T> e2iv = cmul(eiv, eiv);
  Cx<T> term = eiv, sum = eiv;
  const int nmax = series_terms(val(f));
  for (int n = 1; n <= nmax; ++n) {
    T ratio = -f * (2.0 * n - (2.0 - t)) / (2.0 * n + (2.0 - t));
    term = cmul(term, e2iv);
    term.re = term.re * ratio;
    term.im = term.im * ratio;
    sum.re = sum.re + term.re;
    sum.im = sum.im + term.im;
  }
  return sum;
}

// EPL deflection at (x, y); p = [theta_E, gamma, e1, e2, x0, y0].
template <class T, class X>
void epl_deflection(const T* p, const X& x, const X& y, T& ax, T& ay) {
  T q, phi;
  ellipticity(p[2], p[3], q, phi);
  T t = p[1] - 1.0;
  T b = p[0] * sqrt(q);
  T f = (1.0 - q) / (1.0 + q);
  T cs = cos(phi), sn = sin(phi);
  T dx = x - p[4], dy = y - p[5];
  T xp = cs * dx + sn * dy;
  T yp = -sn * dx + cs * dy;
  T R = clamp_below(sqrt(q * q * xp * xp + yp * yp), R_MIN);
  Cx<T> eiv = {q * xp / R, yp / R};
  Cx<T> om = epl_series(t, f, eiv);
  T pref = 2.0 * b / (1.0 + q) * pow(b / R, t - 1.0);
  T alr = pref * om.re, ali = pref * om.im;
  ax = cs * alr - sn * ali;
  ay = sn * alr + cs * ali;
}

// Elliptical Sersic surface brightness at (x, y); p = [R_e, n, e1, e2, x0, y0, I_e].
template <class T, class X>
T sersic(const T* p, const X& x, const X& y) {
  T q, phi;
  ellipticity(p[2], p[3], q, phi);
  T cs = cos(phi), sn = sin(phi);
  T dx = x - p[4], dy = y - p[5];
  T xp = cs * dx + sn * dy;
  T yp = -sn * dx + cs * dy;
  T R = clamp_below(sqrt(q * xp * xp + yp * yp / q), R_MIN);
  T bn = 1.9992 * p[1] - 0.3271;
  return p[6] * exp(-bn * (pow(R / p[0], 1.0 / p[1]) - 1.0));
}

}  // namespace

extern "C" {

// System description, the oracle's own layout (double precision).
typedef struct {
  int ny, nx;
  double pixel_scale;
  int supersample;
  const double* data;   // [ny*nx]
  const double* sigma;  // [ny*nx]
  const double* psf;    // [psf_ny*psf_nx], any positive sum (normalised here)
  int psf_ny, psf_nx;
  int n_lens_light, n_source;
  const int* prior_kind;  // [P]: 0 flat, 1 uniform, 2 normal, 3 truncnorm, 4 lognormal
  const double* prior_a;
  const double* prior_b;
  const double* prior_lo;
  const double* prior_hi;
  const double* emax;  // [1 + n_lens_light + n_source], 0 = no disc constraint
} or_system;

}  // extern "C"

namespace {

inline int num_params(int nl, int ns) { return 8 + 7 * (nl + ns); }

// Surface brightness (lens light + lensed source) at image-plane (x, y).
template <class T>
T surface_brightness(const or_system& s, const T* th, double x, double y) {
  T ax, ay;
  epl_deflection(th, x, y, ax, ay);
  const T& g1 = th[6];
  const T& g2 = th[7];
  T bx = x - ax - (g1 * x + g2 * y);
  T by = y - ay - (g2 * x - g1 * y);
  T sb = zero_like(th[0]);
  for (int c = 0; c < s.n_lens_light; ++c) sb = sb + sersic(th + 8 + 7 * c, x, y);
  for (int c = 0; c < s.n_source; ++c) sb = sb + sersic(th + 8 + 7 * (s.n_lens_light + c), bx, by);
  return sb;
}

// Supersampled, binned image (before the PSF).
template <class T>
void binned_image(const or_system& s, const T* th, std::vector<T>& img) {
  const int ny = s.ny, nx = s.nx, ss = s.supersample;
  const double D = s.pixel_scale;
  img.assign((size_t)ny * nx, zero_like(th[0]));
  for (int i = 0; i < ny; ++i)
    for (int j = 0; j < nx; ++j) {
      T acc = zero_like(th[0]);
      for (int k = 0; k < ss; ++k)
        for (int l = 0; l < ss; ++l) {
          double x = (j - (nx - 1) / 2.0 + (l + 0.5) / ss - 0.5) * D;
          double y = (i - (ny - 1) / 2.0 + (k + 0.5) / ss - 0.5) * D;
          acc = acc + surface_brightness(s, th, x, y);
        }
      img[(size_t)i * nx + j] = acc * (D * D / (ss * ss));
    }
}

// "same" true convolution with zero padding; psf normalised to unit sum.
template <class T>
void convolve_same(const std::vector<T>& img, int ny, int nx, const double* psf, int ky, int kx,
                   std::vector<T>& out) {
  double sum = 0.0;
  for (int u = 0; u < ky * kx; ++u) sum += psf[u];
  const int cy = (ky - 1) / 2, cx = (kx - 1) / 2;
  out.assign((size_t)ny * nx, zero_like(img[0]));
  for (int i = 0; i < ny; ++i)
    for (int j = 0; j < nx; ++j) {
      T acc = zero_like(img[0]);
      for (int u = 0; u < ky; ++u)
        for (int v = 0; v < kx; ++v) {
          int ii = i + cy - u, jj = j + cx - v;
          if (ii < 0 || ii >= ny || jj < 0 || jj >= nx) continue;
          acc = acc + img[(size_t)ii * nx + jj] * (psf[u * kx + v] / sum);
        }
      out[(size_t)i * nx + j] = acc;
    }
}

template <class T>
void model_image(const or_system& s, const T* th, std::vector<T>& m) {
  std::vector<T> b;
  binned_image(s, th, b);
  convolve_same(b, s.ny, s.nx, s.psf, s.psf_ny, s.psf_nx, m);
}

inline double normal_cdf(double z) { return 0.5 * std::erfc(-z / std::sqrt(2.0)); }

// True if th lies in the model's domain and the prior's support.
template <class T>
bool in_support(const or_system& s, const T* th) {
  const int nc = s.n_lens_light + s.n_source;
  const int P = num_params(s.n_lens_light, s.n_source);
  if (!(val(th[0]) > 0.0)) return false;
  if (!(val(th[1]) > 1.0 && val(th[1]) < 3.0)) return false;
  for (int c = 0; c <= nc; ++c) {
    int i1 = c == 0 ? 2 : 8 + 7 * (c - 1) + 2;
    double e = std::sqrt(val(th[i1]) * val(th[i1]) + val(th[i1 + 1]) * val(th[i1 + 1]));
    if (!(e < E_DOMAIN)) return false;
    if (s.emax && s.emax[c] > 0.0 && !(e < s.emax[c])) return false;
    if (c > 0) {
      if (!(val(th[i1 - 2]) > 0.0)) return false;
      if (!(val(th[i1 - 1]) >= N_MIN)) return false;
    }
  }
  for (int k = 0; k < P; ++k) {
    double x = val(th[k]);
    switch (s.prior_kind[k]) {
      case 0: case 1: case 3:
        if (!(x >= s.prior_lo[k] && x <= s.prior_hi[k])) return false;
        break;
      case 4:
        if (!(x > 0.0)) return false;
        break;
      default: break;
    }
  }
  return true;
}

// Normalised log prior density (caller has checked the support).
template <class T>
T log_prior(const or_system& s, const T* th) {
  const int P = num_params(s.n_lens_light, s.n_source);
  T lp = zero_like(th[0]);
  const double ls2p = 0.5 * std::log(2.0 * PI);
  for (int k = 0; k < P; ++k) {
    const double a = s.prior_a[k], b = s.prior_b[k];
    switch (s.prior_kind[k]) {
      case 1:
        lp = lp - std::log(s.prior_hi[k] - s.prior_lo[k]);
        break;
      case 2: {
        T z = (th[k] - a) / b;
        lp = lp - 0.5 * z * z - (std::log(b) + ls2p);
        break;
      }
      case 3: {
        T z = (th[k] - a) / b;
        double mass = normal_cdf((s.prior_hi[k] - a) / b) - normal_cdf((s.prior_lo[k] - a) / b);
        lp = lp - 0.5 * z * z - (std::log(b) + ls2p) - std::log(mass);
        break;
      }
      case 4: {
        T lx = log(th[k]);
        T z = (lx - a) / b;
        lp = lp - 0.5 * z * z - lx - (std::log(b) + ls2p);
        break;
      }
      default: break;
    }
  }
  return lp;
}

template <class T>
T log_likelihood(const or_system& s, const T* th) {
  std::vector<T> m;
  model_image(s, th, m);
  T chi2 = zero_like(th[0]);
  for (size_t p = 0; p < m.size(); ++p) {
    T r = (s.data[p] - m[p]) / s.sigma[p];
    chi2 = chi2 + r * r;
  }
  return -0.5 * chi2;
}

bool any_nan(const double* th, int P) {
  for (int k = 0; k < P; ++k)
    if (std::isnan(th[k])) return true;
  return false;
}

double logp_value(const or_system& s, const double* th) {
  const int P = num_params(s.n_lens_light, s.n_source);
  if (any_nan(th, P)) return std::numeric_limits<double>::quiet_NaN();
  if (!in_support(s, th)) return -std::numeric_limits<double>::infinity();
  return log_likelihood(s, th) + log_prior(s, th);
}

template <int NP>
void logp_grad_one(const or_system& s, const double* th, double* logp, double* grad) {
  const int P = num_params(s.n_lens_light, s.n_source);
  if (any_nan(th, P)) {
    *logp = std::numeric_limits<double>::quiet_NaN();
    for (int k = 0; k < P; ++k) grad[k] = std::numeric_limits<double>::quiet_NaN();
    return;
  }
  if (!in_support(s, th)) {
    *logp = -std::numeric_limits<double>::infinity();
    for (int k = 0; k < P; ++k) grad[k] = 0.0;
    return;
  }
  std::vector<Dual<NP>> x(P);
  for (int k = 0; k < P; ++k) {
    x[k] = cst<NP>(th[k]);
    x[k].d[k] = 1.0;
  }
  Dual<NP> lp = log_likelihood(s, x.data()) + log_prior(s, x.data());
  *logp = lp.v;
  for (int k = 0; k < P; ++k) grad[k] = lp.d[k];
}

void logp_grad_dispatch(const or_system& s, const double* th, double* logp, double* grad) {
  switch (s.n_lens_light + s.n_source) {
    case 1: logp_grad_one<15>(s, th, logp, grad); break;
    case 2: logp_grad_one<22>(s, th, logp, grad); break;
    case 3: logp_grad_one<29>(s, th, logp, grad); break;
    case 4: logp_grad_one<36>(s, th, logp, grad); break;
    case 5: logp_grad_one<43>(s, th, logp, grad); break;
    case 6: logp_grad_one<50>(s, th, logp, grad); break;
    default: {
      const int P = num_params(s.n_lens_light, s.n_source);
      *logp = std::numeric_limits<double>::quiet_NaN();
      for (int k = 0; k < P; ++k) grad[k] = std::numeric_limits<double>::quiet_NaN();
    }
  }
}

template <int NP>
void jacobian_one(const or_system& s, const double* th, double* m, double* J) {
  const int P = num_params(s.n_lens_light, s.n_source);
  std::vector<Dual<NP>> x(P);
  for (int k = 0; k < P; ++k) {
    x[k] = cst<NP>(th[k]);
    x[k].d[k] = 1.0;
  }
  std::vector<Dual<NP>> img;
  model_image(s, x.data(), img);
  for (size_t p = 0; p < img.size(); ++p) {
    m[p] = img[p].v;
    for (int k = 0; k < P; ++k) J[p * P + k] = img[p].d[k];
  }
}

void jacobian_dispatch(const or_system& s, const double* th, double* m, double* J) {
  switch (s.n_lens_light + s.n_source) {
    case 1: jacobian_one<15>(s, th, m, J); break;
    case 2: jacobian_one<22>(s, th, m, J); break;
    case 3: jacobian_one<29>(s, th, m, J); break;
    case 4: jacobian_one<36>(s, th, m, J); break;
    case 5: jacobian_one<43>(s, th, m, J); break;
    case 6: jacobian_one<50>(s, th, m, J); break;
    default: break;
  }
}

void set_threads(int nthreads) {
#ifdef _OPENMP
  if (nthreads > 0) omp_set_num_threads(nthreads);
#else
  (void)nthreads;
#endif
}

}  // namespace

extern "C" {

int or_num_params(int n_lens_light, int n_source) { return num_params(n_lens_light, n_source); }

int or_series_terms(double f) { return series_terms(f); }

// F = 2F1(1, t/2; 2 - t/2; -f e^{2 i varphi}) from the EPL series: Sum Omega_n
// divided by Omega_0 = e^{i varphi}.
void or_hyp2f1_series(double t, double f, double varphi, double* re, double* im) {
  Cx<double> eiv = {std::cos(varphi), std::sin(varphi)};
  Cx<double> om = epl_series(t, f, eiv);
  Cx<double> emiv = {eiv.re, -eiv.im};
  Cx<double> F = cmul(om, emiv);
  *re = F.re;
  *im = F.im;
}

void or_epl_deflection(const double* p6, int n, const double* x, const double* y, double* ax,
                       double* ay) {
  for (int k = 0; k < n; ++k) epl_deflection(p6, x[k], y[k], ax[k], ay[k]);
}

void or_sersic(const double* p7, int n, const double* x, const double* y, double* out) {
  for (int k = 0; k < n; ++k) out[k] = sersic(p7, x[k], y[k]);
}

void or_surface_brightness(const or_system* s, const double* theta, int n, const double* x,
                           const double* y, double* out) {
  for (int k = 0; k < n; ++k) out[k] = surface_brightness(*s, theta, x[k], y[k]);
}

void or_convolve_same(const double* img, int ny, int nx, const double* psf, int ky, int kx,
                      double* out) {
  std::vector<double> in(img, img + (size_t)ny * nx), o;
  convolve_same(in, ny, nx, psf, ky, kx, o);
  std::memcpy(out, o.data(), sizeof(double) * o.size());
}

void or_binned_image(const or_system* s, const double* theta, double* img) {
  std::vector<double> b;
  binned_image(*s, theta, b);
  std::memcpy(img, b.data(), sizeof(double) * b.size());
}

// Model image m (binned, PSF-convolved) for B parameter vectors [B][P].
void or_model_image(const or_system* s, const double* theta, int B, double* img, int nthreads) {
  const int P = num_params(s->n_lens_light, s->n_source);
  const size_t npix = (size_t)s->ny * s->nx;
  set_threads(nthreads);
#pragma omp parallel for schedule(dynamic, 1)
  for (int b = 0; b < B; ++b) {
    std::vector<double> m;
    model_image(*s, theta + (size_t)b * P, m);
    std::memcpy(img + b * npix, m.data(), sizeof(double) * npix);
  }
}

// Returns 1 if theta is in the domain and prior support, 0 otherwise.
int or_in_support(const or_system* s, const double* theta) { return in_support(*s, theta) ? 1 : 0; }

double or_log_prior(const or_system* s, const double* theta) {
  if (!in_support(*s, theta)) return -std::numeric_limits<double>::infinity();
  return log_prior(*s, theta);
}

double or_log_likelihood(const or_system* s, const double* theta) {
  return log_likelihood(*s, theta);
}

void or_logp(const or_system* s, const double* theta, int B, double* logp, int nthreads) {
  const int P = num_params(s->n_lens_light, s->n_source);
  set_threads(nthreads);
#pragma omp parallel for schedule(dynamic, 1)
  for (int b = 0; b < B; ++b) logp[b] = logp_value(*s, theta + (size_t)b * P);
}

void or_logp_grad(const or_system* s, const double* theta, int B, double* logp, double* grad,
                  int nthreads) {
  const int P = num_params(s->n_lens_light, s->n_source);
  set_threads(nthreads);
#pragma omp parallel for schedule(dynamic, 1)
  for (int b = 0; b < B; ++b)
    logp_grad_dispatch(*s, theta + (size_t)b * P, logp + b, grad + (size_t)b * P);
}

// Model image m [ny*nx] and its Jacobian J [ny*nx][P] = d m / d theta (dual
// numbers) for one parameter vector.
void or_model_jacobian(const or_system* s, const double* theta, double* m, double* J) {
  jacobian_dispatch(*s, theta, m, J);
}

int or_max_threads(void) {
#ifdef _OPENMP
  return omp_get_max_threads();
#else
  return 1;
#endif
}

}  // extern "C"
