// host.cu -- C ABI of the engine (include/pmc.h): physics-table construction in
// double precision (Sec. II.A.2, II.A.4-5), device memory, the per-run kernel
// sequence captured in a CUDA graph (Sec. II.B.2: phase space and transport of
// the primaries, the event stage of their non-elastic collisions, the drain of
// every later generation until no secondary proton is left, then the dose
// statistics), and the result read-back.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <condition_variable>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <new>
#include <numeric>
#include <string>
#include <thread>
#include <complex>
#include <vector>

#include "../../include/pmc.h"
#include "pmc_kernels.cuh"

using namespace pmc;

namespace {

constexpr double kNA = 6.02214076e23;

// ---------------------------------------------------------------------------
// physics used to build the tables (double precision)
// ---------------------------------------------------------------------------
double bethe_mass(double E, double ZA, double I_eV) {
  // Bethe mass stopping power without shell or density corrections; below
  // 1 MeV continued as S(1 MeV) sqrt(E).
  const double me = 0.51099895, mp = 938.272088, K = 0.307075;
  const double e = E < 1.0 ? 1.0 : E;
  const double g = 1.0 + e / mp, b2 = 1.0 - 1.0 / (g * g), bg2 = b2 * g * g, r = me / mp;
  const double tmax = 2.0 * me * bg2 / (1.0 + 2.0 * g * r + r * r);
  const double I = I_eV * 1e-6;
  const double s = K * ZA / b2 * (0.5 * std::log(2.0 * me * bg2 * tmax / (I * I)) - b2);
  return E < 1.0 ? s * std::sqrt(E) : s;
}

double tsai_x0(int Z, double A) {
  double Lr, Lp;
  if (Z == 1) { Lr = 5.31; Lp = 6.144; }
  else if (Z == 2) { Lr = 4.79; Lp = 5.621; }
  else if (Z == 3) { Lr = 4.74; Lp = 5.805; }
  else if (Z == 4) { Lr = 4.71; Lp = 5.924; }
  else { Lr = std::log(184.15 * std::pow(Z, -1.0 / 3.0)); Lp = std::log(1194.0 * std::pow(Z, -2.0 / 3.0)); }
  const double a = Z / 137.035999084, a2 = a * a;
  const double f = a2 * (1.0 / (1.0 + a2) + 0.20206 - 0.0369 * a2 + 0.0083 * a2 * a2 - 0.002 * a2 * a2 * a2);
  return 716.408 * A / (Z * Z * (Lr - f) + Z * Lp);
}

double binding_energy(int Z, int A) {
  const int N = A - Z;
  if (A <= 1 || Z < 0 || N < 0) return 0.0;
  if (A == 2) return Z == 1 ? 2.224566 : 0.0;
  if (A == 3) return Z == 1 ? 8.481798 : (Z == 2 ? 7.718043 : 0.0);
  if (A == 4) return Z == 2 ? 28.295660 : 0.0;
  // Weizsaecker: volume, surface, Coulomb, asymmetry and pairing terms
  const double a = A;
  double b = 15.75 * a - 17.8 * std::cbrt(a * a) - 0.711 * Z * (Z - 1.0) / std::cbrt(a) -
             23.7 * (N - Z) * double(N - Z) / a;
  if (Z % 2 == 0 && N % 2 == 0) b += 11.18 / std::sqrt(a);
  if (Z % 2 == 1 && N % 2 == 1) b -= 11.18 / std::sqrt(a);
  return b > 0.0 ? b : 0.0;
}

double nuclear_mass(int Z, int A) { return Z * 938.272088 + (A - Z) * 939.565420 - binding_energy(Z, A); }

double sigma_nn_h(double T, bool like) {
  const double t = T < 10.0 ? 10.0 : T, g = 1.0 + t / 938.272088, b = std::sqrt(1.0 - 1.0 / (g * g));
  return like ? 10.63 / (b * b) - 29.92 / b + 42.9 : 34.10 / (b * b) - 82.2 / b + 82.2;
}

// High-energy limit of the non-elastic cross-section (mb): the empirical fit of Letaw,
// Silberberg & Tsao (ApJS 51, 1983) to measured proton reaction cross-sections.
double sigma_inel_he(int A) {
  return 45.0 * std::pow(double(A), 0.7) * (1.0 + 0.016 * std::sin(5.3 - 2.63 * std::log(double(A))));
}

// Non-elastic cross-section (mb): the fit's energy shape 1 - 0.62 e^(-E/200) sin(10.9 E^-0.28),
// closed below the Coulomb barrier by (1 - B_c/E).
double sigma_inel_h(int Z, int A, double E) {
  if (A <= 1 || E <= 0.0) return 0.0;
  const double a13 = std::cbrt(double(A)), bc = 1.439964548 * Z / (1.16 * (a13 + 1.0));
  if (E <= bc) return 0.0;
  return sigma_inel_he(A) * (1.0 - 0.62 * std::exp(-E / 200.0) * std::sin(10.9 * std::pow(E, -0.28))) * (1.0 - bc / E);
}

double sigma_el_h(int A, double E) {
  if (E <= 0.0) return 0.0;
  if (A == 1) return sigma_nn_h(E, true);
  return 12.0 * std::pow(double(A), 2.0 / 3.0) * (1.0 + 20.0 / (E + 10.0));
}

const double GL8X[4] = {0.1834346424956498, 0.5255324099163290, 0.7966664774136267, 0.9602898564975363};
const double GL8W[4] = {0.3626837833783620, 0.3137066458778873, 0.2223810344533745, 0.1012285362903763};

// Moliere distribution functions (Bethe's form) at kMolN nodes v = i * kMolVmax/(kMolN-1):
// F0 = 1 - exp(-v^2) and, for n = 1, 2,
//   F_n(v) = (1/n!) int_0^inf v J1(v u) exp(-u^2/4) [(u^2/4) ln(u^2/4)]^n du,
// by 8-point Gauss-Legendre on 896 panels of [0, 14].  The fourth component of node i holds
// B(b_i), the root of B - ln B = b_i at b_i = kMolB0 + i / kMolBScale (Newton in double).
std::vector<float4> moliere_table() {
  std::vector<float4> t(kMolN);
  const int panels = 896;
  const double U = 14.0, h = U / panels;
  for (int i = 0; i < kMolN; ++i) {
    const double v = static_cast<double>(kMolVmax) * i / (kMolN - 1);
    double s1 = 0.0, s2 = 0.0;
    for (int k = 0; k < panels; ++k) {
      const double c = (k + 0.5) * h, r = 0.5 * h;
      for (int q = 0; q < 8; ++q) {
        const double u = c + (q < 4 ? -1.0 : 1.0) * r * GL8X[q & 3], w = r * GL8W[q & 3];
        const double y = 0.25 * u * u, L = y * std::log(y);
        const double g = v * ::j1(v * u) * std::exp(-y);
        s1 += w * g * L;
        s2 += w * g * L * L;
      }
    }
    const double b = static_cast<double>(kMolB0) + i / static_cast<double>(kMolBScale);
    double B = std::max(4.5, b + std::log(b));
    for (int it = 0; it < 40; ++it) {
      const double d = (B - std::log(B) - b) / (1.0 - 1.0 / B);
      B -= d;
      if (std::fabs(d) < 1e-15 * B) break;
    }
    t[i] = make_float4(static_cast<float>(1.0 - std::exp(-v * v)), static_cast<float>(s1),
                       static_cast<float>(0.5 * s2), static_cast<float>(i == 0 ? 4.5 : B));
  }
  return t;
}

// Brackets for inverting F = F0 + x F1 + x^2 F2, x = 1/B in (0, 1/4.5]: per node the least
// and greatest F over x (F is quadratic in x), both increasing along the nodes as F is for
// each B; for u in [u_k, u_k+1) the node below u lies at or above the last node whose
// greatest F is <= u_k, and at or below the last node whose least F is <= u_k+1.  Two
// nodes of margin each side cover single-precision evaluation on the device.
std::vector<unsigned> moliere_guide(const std::vector<float4>& t) {
  std::vector<double> flo(kMolN), fhi(kMolN);
  const double xm = 1.0 / 4.5;
  for (int i = 0; i < kMolN; ++i) {
    const double a = t[i].x, b = t[i].y, c = t[i].z;
    auto F = [&](double x) { return a + x * (b + x * c); };
    double lo = std::min(F(0.0), F(xm)), hi = std::max(F(0.0), F(xm));
    if (c != 0.0) {
      const double xs = -b / (2.0 * c);
      if (xs > 0.0 && xs < xm) { lo = std::min(lo, F(xs)); hi = std::max(hi, F(xs)); }
    }
    flo[i] = lo;
    fhi[i] = hi;
  }
  for (int i = 1; i < kMolN; ++i) {        // enforce monotone bounds (conservative)
    flo[i] = std::max(flo[i], flo[i - 1]);
  }
  for (int i = kMolN - 2; i >= 0; --i) fhi[i] = std::min(fhi[i], fhi[i + 1]);
  std::vector<unsigned> g(kMolGuide);
  for (int k = 0; k < kMolGuide; ++k) {
    const double ua = static_cast<double>(k) / kMolGuide, ub = static_cast<double>(k + 1) / kMolGuide;
    int llo = 0, lhi = 0;
    for (int i = 0; i < kMolN; ++i) {
      if (fhi[i] <= ua) llo = i;
      if (flo[i] <= ub) lhi = i;
    }
    const int lo = std::max(0, llo - 2), hi = std::min(kMolN - 1, lhi + 3);
    g[k] = static_cast<unsigned>(lo) | (static_cast<unsigned>(hi) << 16);
  }
  return g;
}

// ---- Vavilov straggling table -------------------------------------------------
// The fluctuation of the loss about its mean, for the Bethe spectrum of transfers to free
// electrons xi (1/eps^2 - beta^2 / (eps eps_max)) on (0, eps_max], has in units of eps_max the
// characteristic function ln phi(tau) = kappa (I2(tau) - beta^2 I1(tau)) with
// I1 = -Cin + i (Si - tau), I2 = -(e^{i tau} - 1 - i tau) + i tau (-Cin + i Si) and
// Cin = gamma + ln tau - Ci.  Its density comes from a discrete Fourier inversion; the table
// holds quantiles of z = (loss - mean) / xi (see kVav* in pmc_device.cuh).

// Sine and cosine integrals: power series up to 4; beyond, the continued fraction of
// E1(i x) = -Ci(x) + i (Si(x) - pi/2) evaluated by the modified Lentz method.
void sine_cosine_integrals(double x, double& si, double& ci) {
  if (x <= 4.0) {
    double p = x, s = x;                                  // x^(2k+1) / (2k+1)!
    for (int k = 1; k < 40; ++k) {
      p *= -x * x / ((2.0 * k) * (2.0 * k + 1.0));
      s += p / (2.0 * k + 1.0);
    }
    double q = 1.0, c = 0.0;                              // x^(2k) / (2k)!
    for (int k = 1; k < 40; ++k) {
      q *= -x * x / ((2.0 * k - 1.0) * (2.0 * k));
      c += q / (2.0 * k);
    }
    si = s;
    ci = 0.57721566490153286 + std::log(x) + c;
    return;
  }
  using cd = std::complex<double>;
  cd b(1.0, x), c(1e300, 0.0), d = 1.0 / b, h = d;
  for (int k = 1; k < 100000; ++k) {
    const double a = -static_cast<double>(k) * k;
    b += 2.0;
    d = 1.0 / (a * d + b);
    c = b + a / c;
    const cd del = c * d;
    h *= del;
    if (std::abs(del - 1.0) < 1e-16) break;
  }
  h *= cd(std::cos(x), -std::sin(x));
  ci = -h.real();
  si = 1.5707963267948966 + h.imag();
}

// In-place radix-2 DFT X_j = sum_k x_k exp(-2 pi i j k / n), n a power of two.
void dft_forward(std::vector<std::complex<double>>& a) {
  const size_t n = a.size();
  for (size_t i = 1, j = 0; i < n; ++i) {
    size_t bit = n >> 1;
    for (; j & bit; bit >>= 1) j ^= bit;
    j ^= bit;
    if (i < j) std::swap(a[i], a[j]);
  }
  for (size_t len = 2; len <= n; len <<= 1) {
    const double ang = -2.0 * 3.14159265358979323846 / static_cast<double>(len);
    const std::complex<double> wl(std::cos(ang), std::sin(ang));
    for (size_t i = 0; i < n; i += len) {
      std::complex<double> w(1.0, 0.0);
      for (size_t k = 0; k < len / 2; ++k) {
        const std::complex<double> u = a[i + k], v = a[i + k + len / 2] * w;
        a[i + k] = u + v;
        a[i + k + len / 2] = u - v;
        w *= wl;
      }
    }
  }
}

// One table row: the kVavNU quantiles of z at (kappa, beta^2), shifted to mean zero.
std::vector<double> vavilov_row(double kappa, double b2) {
  // the distribution's core is about kappa wide (units of eps_max) and the grid spans a few
  // eps_max: thin layers (kappa < 0.01) get a finer grid, keeping its step under 0.06 xi
  const int n = kappa >= 0.01 ? 1 << 14 : 1 << 16;
  const double sd = std::sqrt(kappa * (1.0 - 0.5 * b2));
  const double ylo = -10.0 * sd - 0.05, yhi = 10.0 * sd + 3.0, L = yhi - ylo, dy = L / n;
  std::vector<std::complex<double>> a(n);
  for (int k = 0; k < n; ++k) {
    const int kk = k < n / 2 ? k : k - n;
    const double tau = 2.0 * 3.14159265358979323846 * kk / L;
    std::complex<double> lp(0.0, 0.0);
    if (kk != 0) {
      const double t = std::fabs(tau);
      double si, ci;
      sine_cosine_integrals(t, si, ci);
      const double cin = 0.57721566490153286 + std::log(t) - ci;
      const std::complex<double> i1(-cin, si - t);
      const std::complex<double> i2 = -(std::complex<double>(std::cos(t) - 1.0, std::sin(t) - t)) +
                                      std::complex<double>(-t * si, -t * cin);
      lp = kappa * (i2 - b2 * i1);
      if (tau < 0.0) lp = std::conj(lp);
    }
    a[k] = std::exp(lp) * std::polar(1.0, -tau * ylo);
  }
  dft_forward(a);
  std::vector<double> cdf(n + 1, 0.0);
  for (int j = 0; j < n; ++j) cdf[j + 1] = cdf[j] + std::max(a[j].real() / L, 0.0) * dy;
  for (int j = 0; j <= n; ++j) cdf[j] /= cdf[n];
  for (int j = 1; j <= n; ++j) cdf[j] = std::max(cdf[j], cdf[j - 1]);
  std::vector<double> z(kVavNU);
  int j = 0;
  for (int i = 0; i < kVavNU; ++i) {
    const double u = kVavU0 + i * (1.0 - 2.0 * kVavU0) / (kVavNU - 1);
    while (j < n - 1 && cdf[j + 1] < u) ++j;
    const double w = cdf[j + 1] > cdf[j] ? (u - cdf[j]) / (cdf[j + 1] - cdf[j]) : 0.0;
    z[i] = (ylo - 0.5 * dy + (j + w) * dy) / kappa;
  }
  double mean = 0.5 * (z.front() + z.back());
  for (int i = 1; i < kVavNU - 1; ++i) mean += z[i];
  mean /= (kVavNU - 1);
  for (double& v : z) v -= mean;
  return z;
}

// The table [kVavNB][kVavNK][kVavNU], built once per process.
const std::vector<float>& vavilov_table() {
  static const std::vector<float> tab = [] {
    std::vector<float> t(static_cast<size_t>(kVavNB) * kVavNK * kVavNU);
    for (int ib = 0; ib < kVavNB; ++ib)
      for (int ik = 0; ik < kVavNK; ++ik) {
        const double b2 = kVavB2Max * ib / (kVavNB - 1);
        const double kappa =
            std::exp(std::log(kVavK0) + (std::log(kVavK1) - std::log(kVavK0)) * ik / (kVavNK - 1));
        const std::vector<double> row = vavilov_row(kappa, b2);
        for (int i = 0; i < kVavNU; ++i)
          t[(static_cast<size_t>(ib) * kVavNK + ik) * kVavNU + i] = static_cast<float>(row[i]);
      }
    return t;
  }();
  return tab;
}

double integrate_inv_s(double a, double b, double ZA, double I) {
  const double m = 0.5 * (a + b), h = 0.5 * (b - a);
  double s = 0.0;
  for (int k = 0; k < 4; ++k)
    s += GL8W[k] * (1.0 / bethe_mass(m - h * GL8X[k], ZA, I) + 1.0 / bethe_mass(m + h * GL8X[k], ZA, I));
  return s * h;
}

// Clamped cubic spline on a uniform grid: returns (y, M h^2/6) pairs.
std::vector<float2> spline(const std::vector<double>& y, double h, double d0, double dn) {
  const int n = static_cast<int>(y.size());
  std::vector<double> a(n), b(n), c(n), r(n), M(n);
  b[0] = 2.0; c[0] = 1.0; r[0] = 6.0 / h * ((y[1] - y[0]) / h - d0);
  for (int i = 1; i < n - 1; ++i) {
    a[i] = 1.0; b[i] = 4.0; c[i] = 1.0;
    r[i] = 6.0 * (y[i + 1] - 2.0 * y[i] + y[i - 1]) / (h * h);
  }
  a[n - 1] = 1.0; b[n - 1] = 2.0; r[n - 1] = 6.0 / h * (dn - (y[n - 1] - y[n - 2]) / h);
  for (int i = 1; i < n; ++i) {
    const double w = a[i] / b[i - 1];
    b[i] -= w * c[i - 1];
    r[i] -= w * r[i - 1];
  }
  M[n - 1] = r[n - 1] / b[n - 1];
  for (int i = n - 2; i >= 0; --i) M[i] = (r[i] - c[i] * M[i + 1]) / b[i];
  std::vector<float2> out(n);
  for (int i = 0; i < n; ++i) out[i] = make_float2(static_cast<float>(y[i]), static_cast<float>(M[i] * h * h / 6.0));
  return out;
}

struct RangeClass {
  double ZA, I;
  std::vector<double> E, R;     // forward nodes: ln E = j / 64
  double range(double e) const {  // accurate range at any energy >= 1 MeV
    int j = static_cast<int>(std::log(e) * 64.0);
    j = std::max(0, std::min(j, kNE - 1));
    while (j > 0 && E[j] > e) --j;
    return R[j] + integrate_inv_s(E[j], e, ZA, I);
  }
};

// Range and inverse-range splines of one stopping-power class (Sec. II.A.2):
// R(E) = R(1 MeV) + integral of 1/S from 1 MeV, with R(1 MeV) = 2/S(1 MeV) from
// the sqrt(E) continuation below 1 MeV; nodes uniform in ln E and ln R with
// spacing 2^-6; clamped splines with the exact end slopes.
int build_range_class(double ZA, double I, std::vector<float2>& rt, std::vector<float2>& et, float& S1, float& R1,
                      float& lnR0, int& nR) {
  RangeClass rc;
  rc.ZA = ZA; rc.I = I;
  const double h = 1.0 / 64.0;
  rc.E.resize(kNE); rc.R.resize(kNE);
  const double s1 = bethe_mass(1.0, ZA, I);
  for (int j = 0; j < kNE; ++j) rc.E[j] = std::exp(j * h);
  rc.E[0] = 1.0;
  rc.R[0] = 2.0 / s1;
  for (int j = 1; j < kNE; ++j) rc.R[j] = rc.R[j - 1] + integrate_inv_s(rc.E[j - 1], rc.E[j], ZA, I);
  rt = spline(rc.R, h, rc.E[0] / bethe_mass(rc.E[0], ZA, I), rc.E[kNE - 1] / bethe_mass(rc.E[kNE - 1], ZA, I));
  const double y0 = std::floor(std::log(rc.R[0]) * 64.0) / 64.0;
  const int n = static_cast<int>(std::ceil((std::log(rc.R[kNE - 1]) - y0) * 64.0)) + 1;
  if (n > kNR) return -1;
  std::vector<double> Ey(n);
  for (int j = 0; j < n; ++j) {
    const double Rt = std::exp(y0 + j * h);
    if (Rt <= rc.R[0]) { const double q = 0.5 * Rt * s1; Ey[j] = q * q; continue; }
    int lo = 0, hi = kNE - 1;
    while (hi - lo > 1) { const int mid = (lo + hi) / 2; if (rc.R[mid] <= Rt) lo = mid; else hi = mid; }
    double e = Rt < rc.R[kNE - 1] ? rc.E[lo] + (rc.E[hi] - rc.E[lo]) * (Rt - rc.R[lo]) / (rc.R[hi] - rc.R[lo])
                                  : rc.E[kNE - 1];
    for (int it = 0; it < 40; ++it) {   // Newton on R(E) - Rt, dR/dE = 1/S
      const double de = (rc.range(e) - Rt) * bethe_mass(e, ZA, I);
      e -= de;
      if (std::fabs(de) < 1e-14 * e) break;
    }
    Ey[j] = e;
  }
  const double d0 = std::exp(y0) * (Ey[0] < 1.0 ? s1 * std::sqrt(Ey[0]) : bethe_mass(Ey[0], ZA, I));
  const double dn = std::exp(y0 + (n - 1) * h) * bethe_mass(Ey[n - 1], ZA, I);
  et = spline(Ey, h, d0, dn);
  et.resize(kNR, make_float2(0.0f, 0.0f));
  S1 = static_cast<float>(s1);
  R1 = static_cast<float>(rc.R[0]);
  lnR0 = static_cast<float>(y0);
  nR = n;
  return 0;
}

void build_nucleus(int Z, int A, NucleusModel& nm) {
  std::memset(&nm, 0, sizeof(nm));
  nm.Z = Z; nm.A = A;
  const double a13 = std::cbrt(double(A));
  const double R = 1.16 * a13 * (1.0 - 1.16 / (a13 * a13)), aws = 0.55;
  const double Rout = R + aws * std::log(99.0);
  double norm = 0.0, f[kShells], r[kShells + 1];
  for (int i = 0; i <= kShells; ++i) r[i] = Rout * i / kShells;
  for (int i = 0; i < kShells; ++i) {
    f[i] = 1.0 / (1.0 + std::exp((0.5 * (r[i] + r[i + 1]) - R) / aws));
    norm += f[i] * 4.0 / 3.0 * M_PI * (r[i + 1] * r[i + 1] * r[i + 1] - r[i] * r[i] * r[i]);
  }
  const double Sn = nuclear_mass(Z, A - 1) + 939.565420 - nuclear_mass(Z, A);
  const double Sp = nuclear_mass(Z - 1, A - 1) + 938.272088 - nuclear_mass(Z, A);
  for (int i = 0; i <= kShells; ++i) nm.r[i] = static_cast<float>(r[i]);
  for (int i = 0; i < kShells; ++i) {
    const double rho = f[i] * A / norm;
    for (int q = 0; q < 2; ++q) {
      const double rq = rho * (q ? double(Z) / A : double(A - Z) / A);
      const double m = q ? 938.272088 : 939.565420;
      const double pF = 197.3269804 * std::cbrt(3.0 * M_PI * M_PI * rq);
      const double TF = std::sqrt(pF * pF + m * m) - m;
      nm.rho[q][i] = static_cast<float>(rq);
      nm.pF[q][i] = static_cast<float>(pF);
      nm.TF[q][i] = static_cast<float>(TF);
      nm.V[q][i] = static_cast<float>(TF + (q ? Sp : Sn));
    }
  }
  nm.Rout = static_cast<float>(Rout);
}

// ---------------------------------------------------------------------------
// device memory
// ---------------------------------------------------------------------------
struct DevBuf {
  void* p = nullptr;
  size_t n = 0;
};

}  // namespace

constexpr int kQueues = 6;

struct pmc_ctx {
  pmc_options opt{};
  cudaMemPool_t pool = nullptr;          // stream-ordered allocation from this pool when set
  int n_sm = 0;
  cudaStream_t stream = nullptr;
  cudaStream_t stream2 = nullptr;      // second stream of the pipelined sub-groups
  cudaEvent_t fork_ev = nullptr, join_ev = nullptr;
  std::string err;
  // physics
  bool have_materials = false;
  Physics phys{};
  std::vector<pmc_material> mats;
  std::vector<pmc_nuclide> nucs;
  std::vector<pmc_hu_bin> hus;
  DevBuf d_phys, d_rt, d_et, d_st, d_nuclei, d_btab, d_mol, d_vav;
  // geometry
  bool have_phantom = false;
  Geometry geo{};
  long long n_vox = 0;
  DevBuf d_mat, d_rho, d_hu;
  // spots
  std::vector<pmc_spot> spots;
  int n_spots_dev = 0;                  // spots in the device table of the last run (those with histories)
  // run buffers
  // queues of stream A [0..2] and B [3..5]: phase space of the primaries, protons for the
  // drain, events
  DevBuf d_tally, d_dose, d_sigma, d_counters, d_counts, d_seed, d_spots, d_q[kQueues];
  DevBuf d_hist, d_esc;
  uint64_t hist_n = 0, esc_cap = 0;
  bool let_on = false, let_valid = false;
  DevBuf d_yields;                      // event-generator totals
  cudaEvent_t ev_a = nullptr, ev_b = nullptr;
  DevBuf d_let_num, d_let_den, d_let, d_let_sigma;   // dose-averaged LET tallies and results
  DevBuf d_dlog, d_dlog_cnt;            // debug deposit log and its record count
  uint64_t dlog_cap = 0;
  size_t q_cap = 0;
  int block = 0;
  int64_t chunk = 0;
  bool tuned = false;                  // launch shape fixed (by the caller or the autotuner)
  // kernel timing
  int profile = 0;                  // 0 off, 1 every launch, 2 primary-transport launches only
  std::vector<cudaEvent_t> events;      // pairs around launches
  std::vector<int> event_kind;          // kind per pair
  std::vector<int> event_kernels;       // kernels launched inside each pair
  size_t n_events_used = 0;
  double prof_ms[4] = {0, 0, 0, 0};
  double prof_span[4] = {0, 0, 0, 0};   // first start to last end per kind (launches may overlap)
  int64_t prof_launches[4] = {0, 0, 0, 0};
  int64_t prof_kernels[4] = {0, 0, 0, 0};
  int64_t steps_primary = 0;
  // learned stand-in of the event generator
  bool surr_trained = false;
  int n_slots = 0;                      // non-elastic target slots (nuclides with A >= 2, in order)
  DevBuf d_sp, d_sg, d_sm, d_sv;        // parameters, gradients, Adam moments
  DevBuf d_swb;                         // BF16 inference weights, packed in streaming order
  DevBuf d_gws, d_gerr;                 // training GEMMs: split-K workspace, tensor-core wait errors
  DevBuf d_slot_nuc, d_nuc_slot;        // slot -> nuclide, nuclide -> slot
  DevBuf d_rec[2];               // residual nuclei between cascade and evaporation, per stream
  DevBuf d_drain;                // per stream: drain control block, ready marks of its two queues
  size_t drain_qcap = 0;         // the queue capacity the marks are laid out for
  bool drain_debug = false;      // next drain: one phantom item and short waits (they run out)
  size_t surr_cap = 0;
  int mode = PMC_FULL_CASCADE;          // mode of the captured graph
  // graph
  cudaGraphExec_t gexec = nullptr;
  std::string gkey;
  bool have_run = false;
  pmc_ledger last{};
};

namespace {

int fail(pmc_ctx* c, int code, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  std::vsnprintf(buf, sizeof(buf), fmt, ap);
  va_end(ap);
  if (c) c->err = buf;
  return code;
}

#define CK(call)                                                                               \
  do {                                                                                         \
    cudaError_t e_ = (call);                                                                   \
    if (e_ != cudaSuccess) return fail(ctx, PMC_E_CUDA, "%s: %s", #call, cudaGetErrorString(e_)); \
  } while (0)

void release(pmc_ctx* ctx, void* p) {
  if (ctx->pool) cudaFreeAsync(p, ctx->stream);
  else if (ctx->opt.free) ctx->opt.free(p, ctx->opt.alloc_user);
  else cudaFree(p);
}

int dalloc(pmc_ctx* ctx, DevBuf& b, size_t bytes) {
  if (b.p && b.n >= bytes) return PMC_OK;
  if (b.p) {
    release(ctx, b.p);
    b.p = nullptr;
    b.n = 0;
  }
  if (bytes == 0) return PMC_OK;
  if (ctx->pool) {
    // stream-ordered: no device-wide synchronisation, so plans on other streams keep running
    if (cudaMallocFromPoolAsync(&b.p, bytes, ctx->pool, ctx->stream) != cudaSuccess) {
      cudaGetLastError();
      b.p = nullptr;
      return fail(ctx, PMC_E_OOM, "pool allocation of %zu bytes failed", bytes);
    }
  } else if (ctx->opt.alloc) {
    b.p = ctx->opt.alloc(bytes, ctx->opt.alloc_user);
    if (!b.p) return fail(ctx, PMC_E_OOM, "allocator returned NULL for %zu bytes", bytes);
    if (reinterpret_cast<uintptr_t>(b.p) & 255u) {
      release(ctx, b.p);
      b.p = nullptr;
      return fail(ctx, PMC_E_OOM, "allocator returned a block not aligned to 256 bytes");
    }
  } else if (cudaMalloc(&b.p, bytes) != cudaSuccess) {
    cudaGetLastError();
    b.p = nullptr;
    return fail(ctx, PMC_E_OOM, "cudaMalloc of %zu bytes failed", bytes);
  }
  b.n = bytes;
  // any captured graph may point at the old buffer
  if (ctx->gexec) { cudaGraphExecDestroy(ctx->gexec); ctx->gexec = nullptr; ctx->gkey.clear(); }
  return PMC_OK;
}

void dfree(pmc_ctx* ctx, DevBuf& b) {
  if (!b.p) return;
  release(ctx, b.p);
  b.p = nullptr;
  b.n = 0;
}

int upload(pmc_ctx* ctx, DevBuf& b, const void* src, size_t bytes) {
  int rc = dalloc(ctx, b, bytes);
  if (rc) return rc;
  if (bytes) CK(cudaMemcpyAsync(b.p, src, bytes, cudaMemcpyHostToDevice, ctx->stream));
  CK(cudaStreamSynchronize(ctx->stream));
  return PMC_OK;
}

// Histories per spot in proportion to weight, largest remainder (ties to the lower index).
std::vector<uint64_t> split_histories(const std::vector<pmc_spot>& sp, uint64_t n) {
  double W = 0.0;
  for (const auto& s : sp) W += s.weight;
  std::vector<uint64_t> cnt(sp.size());
  std::vector<double> rem(sp.size());
  uint64_t used = 0;
  for (size_t i = 0; i < sp.size(); ++i) {
    const double q = static_cast<double>(n) * sp[i].weight / W;
    cnt[i] = static_cast<uint64_t>(std::floor(q));
    rem[i] = q - std::floor(q);
    used += cnt[i];
  }
  while (used < n) {
    size_t best = 0;
    for (size_t i = 1; i < sp.size(); ++i) if (rem[i] > rem[best]) best = i;
    cnt[best]++;
    rem[best] = -1.0;
    ++used;
  }
  return cnt;
}

}  // namespace

extern "C" {

int pmc_create(pmc_ctx** out, const pmc_options* opt) {
  if (!out) return PMC_E_INVALID;
  *out = nullptr;
  pmc_ctx* ctx = new (std::nothrow) pmc_ctx();
  if (!ctx) return PMC_E_OOM;
  if (opt) ctx->opt = *opt;
  if (ctx->opt.n_batches == 0) ctx->opt.n_batches = 10;
  // the allocator hooks come as a pair: a block from one must go back to the other
  if (ctx->opt.n_batches < 2 || ctx->opt.n_batches > 1024 || (ctx->opt.alloc == nullptr) != (ctx->opt.free == nullptr)) {
    delete ctx;
    return PMC_E_INVALID;
  }
  if (cudaSetDevice(ctx->opt.device) != cudaSuccess ||
      cudaDeviceGetAttribute(&ctx->n_sm, cudaDevAttrMultiProcessorCount, ctx->opt.device) != cudaSuccess ||
      cudaStreamCreateWithFlags(&ctx->stream, cudaStreamNonBlocking) != cudaSuccess ||
      cudaStreamCreateWithFlags(&ctx->stream2, cudaStreamNonBlocking) != cudaSuccess ||
      cudaEventCreateWithFlags(&ctx->fork_ev, cudaEventDisableTiming) != cudaSuccess ||
      cudaEventCreateWithFlags(&ctx->join_ev, cudaEventDisableTiming) != cudaSuccess) {
    cudaGetLastError();
    delete ctx;
    return PMC_E_CUDA;
  }
  ctx->block = ctx->opt.block_size > 0 ? ctx->opt.block_size : 256;
  ctx->chunk = ctx->opt.chunk;
  ctx->tuned = ctx->opt.block_size > 0;
  *out = ctx;
  return PMC_OK;
}

void pmc_destroy(pmc_ctx* ctx) {
  if (!ctx) return;
  cudaSetDevice(ctx->opt.device);
  cudaStreamSynchronize(ctx->stream);
  if (ctx->gexec) cudaGraphExecDestroy(ctx->gexec);
  for (cudaEvent_t e : ctx->events) cudaEventDestroy(e);
  DevBuf* bufs[] = {&ctx->d_phys, &ctx->d_rt, &ctx->d_et, &ctx->d_st, &ctx->d_nuclei, &ctx->d_btab, &ctx->d_mol, &ctx->d_vav, &ctx->d_mat,
                    &ctx->d_rho, &ctx->d_hu, &ctx->d_tally, &ctx->d_dose, &ctx->d_sigma, &ctx->d_counters,
                    &ctx->d_counts, &ctx->d_seed, &ctx->d_spots, &ctx->d_q[0], &ctx->d_q[1], &ctx->d_q[2],
                    &ctx->d_q[3], &ctx->d_q[4], &ctx->d_q[5], &ctx->d_hist, &ctx->d_esc,
                    &ctx->d_let_num, &ctx->d_let_den, &ctx->d_let, &ctx->d_let_sigma, &ctx->d_yields,
                    &ctx->d_dlog, &ctx->d_dlog_cnt};
  if (ctx->ev_a) cudaEventDestroy(ctx->ev_a);
  if (ctx->ev_b) cudaEventDestroy(ctx->ev_b);
  for (DevBuf* b : bufs) dfree(ctx, *b);
  DevBuf* sbufs[] = {&ctx->d_swb, &ctx->d_sp, &ctx->d_sg, &ctx->d_sm, &ctx->d_sv, &ctx->d_slot_nuc, &ctx->d_nuc_slot,
                     &ctx->d_rec[0], &ctx->d_rec[1], &ctx->d_gws, &ctx->d_gerr, &ctx->d_drain};
  for (DevBuf* b : sbufs) dfree(ctx, *b);
  if (ctx->pool) cudaStreamSynchronize(ctx->stream);   // the stream-ordered frees have run
  cudaStreamDestroy(ctx->stream);
  cudaStreamDestroy(ctx->stream2);
  cudaEventDestroy(ctx->fork_ev);
  cudaEventDestroy(ctx->join_ev);
  delete ctx;
}

const char* pmc_last_error(const pmc_ctx* ctx) { return ctx ? ctx->err.c_str() : "no context"; }

int pmc_load_materials(pmc_ctx* ctx, const pmc_nuclide* nuc, int n_nuc, const pmc_material* mat, int n_mat,
                       const pmc_hu_bin* hu, int n_hu) {
  if (!ctx) return PMC_E_INVALID;
  try {
    if (!nuc || !mat || n_nuc < 1 || n_nuc > PMC_MAX_NUCLIDES || n_mat < 1 || n_mat > PMC_MAX_MATERIALS ||
        n_hu < 0 || n_hu > PMC_MAX_HU_BINS || (n_hu > 0 && !hu))
      return fail(ctx, PMC_E_INVALID, "material counts out of range");
    if (mat[0].own_table) return fail(ctx, PMC_E_INVALID, "material 0 must be the scaled reference water");
    cudaSetDevice(ctx->opt.device);
    Physics& ph = ctx->phys;
    std::memset(&ph, 0, sizeof(ph));
    ph.n_mat = n_mat; ph.n_nuc = n_nuc; ph.n_hu = n_hu;
    ph.flags = ctx->opt.physics_flags;
    for (int i = 0; i < n_nuc; ++i) {
      const pmc_nuclide& q = nuc[i];
      if (q.Z < 1 || q.A < q.Z || q.A >= kMaxA - 1 || q.Z >= kMaxZ - 1 || q.mass_u <= 0.0 || q.I_eV <= 0.0)
        return fail(ctx, PMC_E_INVALID, "nuclide %d invalid", i);
      NucConst& c = ph.nuc[i];
      c.Z = q.Z; c.A = q.A;
      const double a13 = std::cbrt(double(q.A));
      c.a13 = static_cast<float>(a13);
      c.bc = static_cast<float>(q.A > 1 ? 1.439964548 * q.Z / (1.16 * (a13 + 1.0)) : 0.0);
      c.sig_he = static_cast<float>(q.A > 1 ? sigma_inel_he(q.A) : 0.0);
      c.el = static_cast<float>(12.0 * a13 * a13);
      c.mass = static_cast<float>(nuclear_mass(q.Z, q.A));
    }
    // materials: Z/A, mean excitation energy, Eq. 1 factor, radiation length, classes
    std::vector<double> ZA(n_mat), Iv(n_mat), mol_zz(n_mat, 0.0);
    for (int m = 0; m < n_mat; ++m) {
      const pmc_material& M = mat[m];
      if (M.n < 1 || M.n > PMC_MAX_NUC_PER_MAT || M.rho <= 0.0) return fail(ctx, PMC_E_INVALID, "material %d invalid", m);
      double wsum = 0.0, za = 0.0, lnI = 0.0, ix0 = 0.0;
      for (int k = 0; k < M.n; ++k) {
        if (M.nuc[k] < 0 || M.nuc[k] >= n_nuc || M.w[k] < 0.0) return fail(ctx, PMC_E_INVALID, "material %d entry %d", m, k);
        const pmc_nuclide& q = nuc[M.nuc[k]];
        wsum += M.w[k];
        za += M.w[k] * q.Z / q.mass_u;
        lnI += M.w[k] * q.Z / q.mass_u * std::log(q.I_eV);
        ix0 += M.w[k] / tsai_x0(q.Z, q.mass_u);
      }
      if (std::fabs(wsum - 1.0) > 1e-6) return fail(ctx, PMC_E_INVALID, "material %d fractions sum to %g", m, wsum);
      ZA[m] = za;
      Iv[m] = M.I_eV > 0.0 ? M.I_eV : std::exp(lnI / za);
      MatConst& mc = ph.mat[m];
      mc.ZA = static_cast<float>(za);
      mc.inv_X0 = static_cast<float>(ix0);
      mc.bohr_k = static_cast<float>(0.307075 * 0.51099895 * za);
      mc.n = M.n;
      for (int k = 0; k < M.n; ++k) {
        mc.nuc[k] = M.nuc[k];
        mc.n_per_g[k] = static_cast<float>(M.w[k] * kNA / nuc[M.nuc[k]].mass_u * 1e-27);
      }
      // Moliere: chi_c^2 = K m_e c^2 x sum w Z(Z+1)/A / (p beta)^2; screening angle
      // chi_a^2 = chi_0^2 (1.13 + 3.76 alpha^2), chi_0 = hbar c Z^(1/3) / (0.885 a0 p),
      // alpha = Z / (137.036 beta), log-averaged over the elements with weights w Z(Z+1)/A
      double zz = 0.0;
      for (int k = 0; k < M.n; ++k) {
        const double Z = nuc[M.nuc[k]].Z;
        zz += M.w[k] * Z * (Z + 1.0) / nuc[M.nuc[k]].mass_u;
      }
      mc.mol_K = static_cast<float>(0.307075 * 0.51099895 * zz);
      mol_zz[m] = zz;
    }
    int ncls = 1;
    for (int m = 0; m < n_mat; ++m) {
      MatConst& mc = ph.mat[m];
      if (m > 0 && mat[m].own_table) {
        if (ncls >= kMaxCls) return fail(ctx, PMC_E_INVALID, "at most %d own-table materials", kMaxCls - 1);
        mc.cls = ncls++;
        mc.f = 1.0f;
      } else {
        mc.cls = 0;
        mc.f = static_cast<float>(m == 0 ? 1.0 : bethe_mass(100.0, ZA[m], Iv[m]) / bethe_mass(100.0, ZA[0], Iv[0]));
      }
    }
    ph.n_cls = ncls;
    std::vector<float2> rt(ncls * kNE), et(ncls * kNR);
    for (int m = 0; m < n_mat; ++m) {
      const int c = ph.mat[m].cls;
      if (m > 0 && c == 0) continue;
      std::vector<float2> a, b;
      if (build_range_class(ZA[m], Iv[m], a, b, ph.S1[c], ph.R1[c], ph.lnR0[c], ph.nR[c]))
        return fail(ctx, PMC_E_INVALID, "material %d: range table exceeds %d nodes", m, kNR);
      std::copy(a.begin(), a.end(), rt.begin() + c * kNE);
      std::copy(b.begin(), b.end(), et.begin() + c * kNR);
    }
    std::vector<float> st(n_mat * kNS);
    for (int m = 0; m < n_mat; ++m) {
      for (int j = 0; j < kNS; ++j) {
        const double E = std::exp(static_cast<double>(kLnS0) + j / 64.0);
        double s = 0.0;
        for (int k = 0; k < mat[m].n; ++k) {
          const pmc_nuclide& q = nuc[mat[m].nuc[k]];
          double sg = 0.0;
          if (!(ph.flags & kNoInelastic)) sg += sigma_inel_h(q.Z, q.A, E);
          if (!(ph.flags & kNoElastic)) sg += sigma_el_h(q.A, E);
          s += mat[m].w[k] * kNA / q.mass_u * sg * 1e-27;
        }
        st[m * kNS + j] = static_cast<float>(s);
      }
    }
    for (int i = 0; i < n_hu; ++i) {
      if (hu[i].material < 0 || hu[i].material >= n_mat || hu[i].hi <= hu[i].lo)
        return fail(ctx, PMC_E_INVALID, "HU bin %d invalid", i);
      ph.hu[i].lo = hu[i].lo; ph.hu[i].hi = hu[i].hi; ph.hu[i].mat = hu[i].material;
      ph.hu[i].a = static_cast<float>(hu[i].rho_a); ph.hu[i].b = static_cast<float>(hu[i].rho_b);
    }
    std::vector<NucleusModel> nm(n_nuc);
    for (int i = 0; i < n_nuc; ++i) {
      if (nuc[i].A >= 2) build_nucleus(nuc[i].Z, nuc[i].A, nm[i]);
      else std::memset(&nm[i], 0, sizeof(NucleusModel));
    }
    // binding energies [Z][A], then the cube roots A^(1/3) of the mass numbers
    std::vector<float> bt(kBtabFloats);
    for (int z = 0; z < kMaxZ; ++z)
      for (int a = 0; a < kMaxA; ++a) bt[z * kMaxA + a] = static_cast<float>(binding_energy(z, a));
    for (int a = 0; a < kMaxA; ++a) bt[kMaxZ * kMaxA + a] = static_cast<float>(std::cbrt(static_cast<double>(a)));
    int rc;
    if ((rc = upload(ctx, ctx->d_phys, &ph, sizeof(Physics)))) return rc;
    if ((rc = upload(ctx, ctx->d_rt, rt.data(), rt.size() * sizeof(float2)))) return rc;
    if ((rc = upload(ctx, ctx->d_et, et.data(), et.size() * sizeof(float2)))) return rc;
    if ((rc = upload(ctx, ctx->d_st, st.data(), st.size() * sizeof(float)))) return rc;
    if ((rc = upload(ctx, ctx->d_nuclei, nm.data(), nm.size() * sizeof(NucleusModel)))) return rc;
    if ((rc = upload(ctx, ctx->d_btab, bt.data(), bt.size() * sizeof(float)))) return rc;
    if (ph.flags & kMoliere) {
      // the distribution table, then per material G_m(E) = ln chi_c^2 - ln x - ln(1.167 chi_a^2)
      // on the cross-section grid: chi_c^2 = K x / (p beta)^2, and the screening angle
      // chi_a^2 = chi_0^2 (1.13 + 3.76 alpha^2), chi_0 = hbar c Z^(1/3) / (0.885 a0 p),
      // alpha = Z / (137.036 beta), log-averaged over the elements with weights w Z(Z+1)/A
      const std::vector<float4> mt = moliere_table();
      std::vector<float> tab(moliere_table_bytes(n_mat) / sizeof(float));
      std::memcpy(tab.data(), mt.data(), mt.size() * sizeof(float4));
      const std::vector<unsigned> guide = moliere_guide(mt);
      std::memcpy(tab.data() + kMolN * 4, guide.data(), guide.size() * sizeof(unsigned));
      const double q0 = 197.3269804 / (0.885 * 52917.721090);   // hbar c / (0.885 a0), MeV
      const double mp = 938.272088;
      for (int m = 0; m < n_mat; ++m) {
        const pmc_material& M = mat[m];
        for (int j = 0; j < kNS; ++j) {
          const double E = std::exp(static_cast<double>(kLnS0) + j / 64.0);
          const double pc = std::sqrt(E * E + 2.0 * E * mp), beta = pc / (E + mp);
          double lna = -2.0 * std::log(pc);
          for (int k = 0; k < M.n; ++k) {
            const double Z = nuc[M.nuc[k]].Z;
            const double c = M.w[k] * Z * (Z + 1.0) / nuc[M.nuc[k]].mass_u / mol_zz[m];
            const double al = Z / (137.035999 * beta);
            lna += c * std::log(q0 * q0 * std::pow(Z, 2.0 / 3.0) * (1.13 + 3.76 * al * al));
          }
          const double lnK = std::log(0.307075 * 0.51099895 * mol_zz[m]);
          tab[kMolN * 4 + kMolGuide + m * kNS + j] =
              static_cast<float>(lnK - 2.0 * std::log(pc * beta) - lna - (2.0 * 0.57721566490153286 - 1.0));
        }
      }
      if ((rc = upload(ctx, ctx->d_mol, tab.data(), tab.size() * sizeof(float)))) return rc;
    } else {
      dfree(ctx, ctx->d_mol);
    }
    if (ph.flags & kVavilov) {
      const std::vector<float>& vt = vavilov_table();
      if ((rc = upload(ctx, ctx->d_vav, vt.data(), vt.size() * sizeof(float)))) return rc;
    } else {
      dfree(ctx, ctx->d_vav);
    }
    std::vector<int> slot_nuc, nuc_slot(n_nuc, -1);
    for (int i = 0; i < n_nuc; ++i)
      if (nuc[i].A >= 2) { nuc_slot[i] = static_cast<int>(slot_nuc.size()); slot_nuc.push_back(i); }
    if ((rc = upload(ctx, ctx->d_nuc_slot, nuc_slot.data(), nuc_slot.size() * sizeof(int)))) return rc;
    if (!slot_nuc.empty() && (rc = upload(ctx, ctx->d_slot_nuc, slot_nuc.data(), slot_nuc.size() * sizeof(int)))) return rc;
    ctx->n_slots = static_cast<int>(slot_nuc.size());
    ctx->surr_trained = false;
    ctx->mats.assign(mat, mat + n_mat);
    ctx->nucs.assign(nuc, nuc + n_nuc);
    ctx->hus.assign(hu, hu + n_hu);
    ctx->have_materials = true;
    if (ctx->gexec) { cudaGraphExecDestroy(ctx->gexec); ctx->gexec = nullptr; ctx->gkey.clear(); }
    return PMC_OK;
  } catch (...) {
    return fail(ctx, PMC_E_INVALID, "exception while building tables");
  }
}

int pmc_load_phantom(pmc_ctx* ctx, int nx, int ny, int nz, double dx, double dy, double dz, double x0, double y0,
                     double z0, const int16_t* hu, const uint8_t* mat, const float* rho) {
  if (!ctx) return PMC_E_INVALID;
  if (nx < 1 || ny < 1 || nz < 1 || dx <= 0 || dy <= 0 || dz <= 0)
    return fail(ctx, PMC_E_INVALID, "bad grid");
  if (!hu && !(mat && rho)) return fail(ctx, PMC_E_INVALID, "give hu, or mat and rho");
  if (hu && !ctx->have_materials) return fail(ctx, PMC_E_INVALID, "load materials (with HU bins) first");
  if (hu && ctx->phys.n_hu < 1) return fail(ctx, PMC_E_INVALID, "HU phantom needs HU bins");
  const long long n = static_cast<long long>(nx) * ny * nz;
  if (n > (1ll << 31) - 1) return fail(ctx, PMC_E_INVALID, "at most 2^31-1 voxels");
  cudaSetDevice(ctx->opt.device);
  const bool shape_changed = n != ctx->n_vox || (hu != nullptr) != (ctx->geo.hu != nullptr);
  Geometry& g = ctx->geo;
  g.nx = nx; g.ny = ny; g.nz = nz;
  g.dx = static_cast<float>(dx); g.dy = static_cast<float>(dy); g.dz = static_cast<float>(dz);
  g.x0 = static_cast<float>(x0); g.y0 = static_cast<float>(y0); g.z0 = static_cast<float>(z0);
  g.idx = static_cast<float>(1.0 / dx); g.idy = static_cast<float>(1.0 / dy); g.idz = static_cast<float>(1.0 / dz);
  int rc;
  if (hu) {
    if ((rc = dalloc(ctx, ctx->d_hu, n * sizeof(int16_t)))) return rc;
    CK(cudaMemcpyAsync(ctx->d_hu.p, hu, n * sizeof(int16_t), cudaMemcpyHostToDevice, ctx->stream));
    g.hu = static_cast<const int16_t*>(ctx->d_hu.p);
    g.mat = nullptr; g.rho = nullptr;
  } else {
    if ((rc = dalloc(ctx, ctx->d_mat, n))) return rc;
    if ((rc = dalloc(ctx, ctx->d_rho, n * sizeof(float)))) return rc;
    CK(cudaMemcpyAsync(ctx->d_mat.p, mat, n, cudaMemcpyHostToDevice, ctx->stream));
    CK(cudaMemcpyAsync(ctx->d_rho.p, rho, n * sizeof(float), cudaMemcpyHostToDevice, ctx->stream));
    g.mat = static_cast<const uint8_t*>(ctx->d_mat.p);
    g.rho = static_cast<const float*>(ctx->d_rho.p);
    g.hu = nullptr;
  }
  CK(cudaStreamSynchronize(ctx->stream));
  ctx->n_vox = n;
  ctx->have_phantom = true;
  if (shape_changed) {
    // results of an earlier run belong to the old grid (and its buffer sizes)
    ctx->have_run = false;
    ctx->let_valid = false;
    if (ctx->gexec) { cudaGraphExecDestroy(ctx->gexec); ctx->gexec = nullptr; ctx->gkey.clear(); }
  }
  return PMC_OK;
}

int pmc_add_spots(pmc_ctx* ctx, const pmc_spot* s, int n) {
  if (!ctx || n < 0 || (n > 0 && !s)) return PMC_E_INVALID;
  for (int i = 0; i < n; ++i) {
    const double dn = std::sqrt(s[i].u * s[i].u + s[i].v * s[i].v + s[i].w * s[i].w);
    if (!(s[i].weight >= 0.0) || !(s[i].E >= 0.0) || !(dn > 0.0))
      return fail(ctx, PMC_E_INVALID, "spot %d invalid", i);
  }
  ctx->spots.insert(ctx->spots.end(), s, s + n);
  return PMC_OK;
}

int pmc_clear_spots(pmc_ctx* ctx) {
  if (!ctx) return PMC_E_INVALID;
  ctx->spots.clear();
  return PMC_OK;
}

int pmc_set_launch(pmc_ctx* ctx, int block_size, int64_t chunk) {
  if (!ctx) return PMC_E_INVALID;
  if (block_size != 0 && (block_size < 32 || block_size > 256 || block_size % 32))
    return fail(ctx, PMC_E_INVALID, "block size must be a multiple of 32 in [32, 256]");
  if (chunk < 0) return fail(ctx, PMC_E_INVALID, "chunk must be >= 0");
  if (block_size) ctx->block = block_size;
  if (chunk) ctx->chunk = chunk;
  if (block_size) ctx->tuned = true;
  return PMC_OK;
}

int pmc_enable_profile(pmc_ctx* ctx, int on) {
  if (!ctx) return PMC_E_INVALID;
  if (on < 0 || on > 2) return fail(ctx, PMC_E_INVALID, "profile mode must be 0, 1 or 2");
  ctx->profile = on;
  return PMC_OK;
}

int pmc_read_profile(pmc_ctx* ctx, double* ms, int64_t* launches, int64_t* primary_steps) {
  if (!ctx) return PMC_E_INVALID;
  for (int k = 0; k < 4; ++k) {
    if (ms) { ms[k] = ctx->prof_ms[k]; ms[4 + k] = ctx->prof_span[k]; }
    if (launches) { launches[k] = ctx->prof_launches[k]; launches[4 + k] = ctx->prof_kernels[k]; }
  }
  if (primary_steps) *primary_steps = ctx->steps_primary;
  return PMC_OK;
}

int pmc_enable_history_ledger(pmc_ctx* ctx, uint64_t max_histories) {
  if (!ctx) return PMC_E_INVALID;
  cudaSetDevice(ctx->opt.device);
  if (max_histories == 0) { dfree(ctx, ctx->d_hist); ctx->hist_n = 0; }
  else {
    int rc = dalloc(ctx, ctx->d_hist, max_histories * 4 * sizeof(long long));
    if (rc) return rc;
    ctx->hist_n = max_histories;
  }
  if (ctx->gexec) { cudaGraphExecDestroy(ctx->gexec); ctx->gexec = nullptr; ctx->gkey.clear(); }
  return PMC_OK;
}

int pmc_enable_let(pmc_ctx* ctx, int on) {
  if (!ctx) return PMC_E_INVALID;
  cudaSetDevice(ctx->opt.device);
  ctx->let_on = on != 0;
  if (!ctx->let_on) {
    dfree(ctx, ctx->d_let_num);
    dfree(ctx, ctx->d_let_den);
    dfree(ctx, ctx->d_let);
    dfree(ctx, ctx->d_let_sigma);
  }
  ctx->let_valid = false;
  if (ctx->gexec) { cudaGraphExecDestroy(ctx->gexec); ctx->gexec = nullptr; ctx->gkey.clear(); }
  return PMC_OK;
}

int pmc_enable_escape_record(pmc_ctx* ctx, uint64_t cap) {
  if (!ctx) return PMC_E_INVALID;
  cudaSetDevice(ctx->opt.device);
  if (cap == 0) { dfree(ctx, ctx->d_esc); ctx->esc_cap = 0; }
  else {
    int rc = dalloc(ctx, ctx->d_esc, cap * 8 * sizeof(float));
    if (rc) return rc;
    ctx->esc_cap = cap;
  }
  if (ctx->gexec) { cudaGraphExecDestroy(ctx->gexec); ctx->gexec = nullptr; ctx->gkey.clear(); }
  return PMC_OK;
}

int pmc_enable_deposit_log(pmc_ctx* ctx, uint64_t cap) {
  if (!ctx) return PMC_E_INVALID;
  if (cap > (1ull << 30)) return fail(ctx, PMC_E_INVALID, "deposit log capacity above 2^30 records");
  cudaSetDevice(ctx->opt.device);
  int rc;
  if (cap == 0) {
    dfree(ctx, ctx->d_dlog);
    dfree(ctx, ctx->d_dlog_cnt);
  } else {
    if ((rc = dalloc(ctx, ctx->d_dlog, cap * sizeof(DepositRecord)))) return rc;
    if ((rc = dalloc(ctx, ctx->d_dlog_cnt, sizeof(unsigned long long)))) return rc;
    CK(cudaMemsetAsync(ctx->d_dlog_cnt.p, 0, sizeof(unsigned long long), ctx->stream));
    CK(cudaStreamSynchronize(ctx->stream));
  }
  ctx->dlog_cap = cap;
  if (ctx->gexec) { cudaGraphExecDestroy(ctx->gexec); ctx->gexec = nullptr; ctx->gkey.clear(); }
  return PMC_OK;
}

int pmc_read_deposit_log(pmc_ctx* ctx, pmc_deposit* out, uint64_t cap, uint64_t* n) {
  if (!ctx || !n || (cap && !out)) return PMC_E_INVALID;
  if (!ctx->dlog_cap) return fail(ctx, PMC_E_INVALID, "the deposit log is not enabled");
  static_assert(sizeof(pmc_deposit) == sizeof(DepositRecord), "deposit record layout");
  cudaSetDevice(ctx->opt.device);
  unsigned long long cnt = 0;
  CK(cudaMemcpy(&cnt, ctx->d_dlog_cnt.p, sizeof(cnt), cudaMemcpyDeviceToHost));
  *n = cnt;
  const uint64_t k = std::min<uint64_t>(std::min<uint64_t>(cnt, ctx->dlog_cap), cap);
  if (k) CK(cudaMemcpy(out, ctx->d_dlog.p, k * sizeof(DepositRecord), cudaMemcpyDeviceToHost));
  if (cnt > ctx->dlog_cap)
    return fail(ctx, PMC_E_QUEUE_OVERFLOW, "%llu deposits, the log holds %llu", cnt, (unsigned long long)ctx->dlog_cap);
  return PMC_OK;
}

}  // extern "C"

namespace {

struct RunPlan {
  uint64_t n;
  int64_t chunk;
  int n_chunks;
  int grid_t, grid_c;           // grids of the primary transport and of the cascade
  size_t smem;
  int grid_d;                   // the drain's grid and shared memory
  size_t smem_d;
};



// Records a timing event opening (open) or closing a pair around a launch of the given kind,
// when that kind is profiled.
int mark(pmc_ctx* ctx, cudaStream_t s, int kind, bool open, int kernels = 1) {
  if (!ctx->profile || (ctx->profile == 2 && kind != 0)) return PMC_OK;
  if (ctx->n_events_used == ctx->events.size()) {
    cudaEvent_t e;
    CK(cudaEventCreate(&e));
    ctx->events.push_back(e);
  }
  cudaEvent_t e = ctx->events[ctx->n_events_used++];
  if (open) ctx->event_kind.push_back(kind);
  else ctx->event_kernels.push_back(kernels);
  CK(cudaEventRecordWithFlags(e, s, cudaEventRecordExternal));
  return PMC_OK;
}

// Parameter layout of the quantile network: W_l [out x in] row-major, then b_l.
constexpr int kLayerIn[kSurrLayers] = {kSurrIn, kSurrHidden, kSurrHidden, kSurrHidden, kSurrHidden};
constexpr int kLayerOut[kSurrLayers] = {kSurrHidden, kSurrHidden, kSurrHidden, kSurrHidden, kSurrOut};
size_t w_off(int l) {
  size_t o = 0;
  for (int i = 0; i < l; ++i) o += static_cast<size_t>(kLayerIn[i]) * kLayerOut[i] + kLayerOut[i];
  return o;
}
size_t b_off(int l) { return w_off(l) + static_cast<size_t>(kLayerIn[l]) * kLayerOut[l]; }
constexpr size_t kSurrParams = 32 * 256 + 256 + 3 * (256 * 256 + 256) + 256 * 16 + 16;
static_assert(kSurrParams == PMC_SURROGATE_PARAMS, "parameter count stated in pmc.h");

// The training GEMMs run on the tensor cores (launch_gemm_tc); their split-K workspace
// (room for 128 splits of a 256 x 256 weight gradient) and wait-error flag.
constexpr size_t kGemmWsFloats = 128ull * 256 * 256;
int gemm_buffers(pmc_ctx* ctx) {
  int rc;
  if ((rc = dalloc(ctx, ctx->d_gws, kGemmWsFloats * sizeof(float)))) return rc;
  if (!ctx->d_gerr.p) {
    if ((rc = dalloc(ctx, ctx->d_gerr, sizeof(int)))) return rc;
    CK(cudaMemset(ctx->d_gerr.p, 0, sizeof(int)));
  }
  return PMC_OK;
}

int gemm(pmc_ctx* ctx, int M, int N, int K, const float* A, long long sam, long long sak, const float* B, long long sbk,
         long long sbn, float* C, long long ldc, const float* bias, bool relu, const float* mask, bool accumulate,
         cudaStream_t s) {
  CK(launch_gemm_tc(M, N, K, A, sam, sak, B, sbk, sbn, C, ldc, bias, relu, mask, accumulate,
                    static_cast<float*>(ctx->d_gws.p), kGemmWsFloats, static_cast<int*>(ctx->d_gerr.p), ctx->n_sm, s));
  return PMC_OK;
}

// Forward pass over rows: act[l] = layer l output (ReLU for l < 4).
int mlp_forward(pmc_ctx* ctx, const float* P, int rows, const float* X, float* const* act, cudaStream_t s) {
  int rc;
  if ((rc = gemm_buffers(ctx))) return rc;
  for (int l = 0; l < kSurrLayers; ++l) {
    const float* in = l == 0 ? X : act[l - 1];
    const int di = kLayerIn[l], dO = kLayerOut[l];
    if ((rc = gemm(ctx, rows, dO, di, in, di, 1, P + w_off(l), 1, di, act[l], dO, P + b_off(l), l < kSurrLayers - 1,
                   nullptr, false, s)))
      return rc;
  }
  return PMC_OK;
}

// Backward pass from G = d loss / d output; gradients into Gp (same layout as P).
int mlp_backward(pmc_ctx* ctx, const float* P, float* Gp, int rows, const float* X, float* const* act, float* g0,
                 float* g1, cudaStream_t s) {
  int rc;
  if ((rc = gemm_buffers(ctx))) return rc;
  const float* G = act[kSurrLayers];   // d loss / d yhat (rows x 16)
  float* bufs[2] = {g0, g1};
  for (int l = kSurrLayers - 1; l >= 0; --l) {
    const float* in = l == 0 ? X : act[l - 1];
    const int di = kLayerIn[l], dO = kLayerOut[l];
    // dW = G^T in (K = rows, split over the workspace)
    if ((rc = gemm(ctx, dO, di, rows, G, 1, dO, in, di, 1, Gp + w_off(l), di, nullptr, false, nullptr, false, s)))
      return rc;
    CK(launch_colsum(rows, dO, G, Gp + b_off(l), s));
    if (l > 0) {
      // dX = G W, masked by the ReLU of the layer below
      float* Gn = bufs[l & 1];
      if ((rc = gemm(ctx, rows, di, dO, G, dO, 1, P + w_off(l), di, 1, Gn, di, nullptr, false, act[l - 1], false, s)))
        return rc;
      G = Gn;
    }
  }
  return PMC_OK;
}

// Raises the tensor-core wait errors of the training GEMMs since the last call.
int gemm_errors(pmc_ctx* ctx) {
  if (!ctx->d_gerr.p) return PMC_OK;
  int e = 0;
  CK(cudaMemcpy(&e, ctx->d_gerr.p, sizeof(int), cudaMemcpyDeviceToHost));
  if (!e) return PMC_OK;
  CK(cudaMemset(ctx->d_gerr.p, 0, sizeof(int)));
  return fail(ctx, PMC_E_TIMEOUT, "%d training GEMM tiles: tensor-core waits timed out", e);
}

// Kernel arguments of the primaries' transport.
TransportArgs transport_args(pmc_ctx* ctx) {
  TransportArgs a{};
  a.phys = static_cast<const Physics*>(ctx->d_phys.p);
  a.rtab = static_cast<const float2*>(ctx->d_rt.p);
  a.etab = static_cast<const float2*>(ctx->d_et.p);
  a.stab = static_cast<const float*>(ctx->d_st.p);
  a.mol = static_cast<const float4*>(ctx->d_mol.p);
  a.vav = static_cast<const float*>(ctx->d_vav.p);
  a.g = ctx->geo;
  a.tally = static_cast<unsigned long long*>(ctx->d_tally.p);
  a.B = ctx->opt.n_batches;
  a.seed = static_cast<const unsigned long long*>(ctx->d_seed.p);
  a.spots = static_cast<const SpotDev*>(ctx->d_spots.p);
  a.n_spots = ctx->n_spots_dev;
  a.cnt = static_cast<Counters*>(ctx->d_counters.p);
  a.hist = static_cast<long long*>(ctx->d_hist.p);
  a.hist_n = ctx->hist_n;
  a.esc = static_cast<float*>(ctx->d_esc.p);
  a.esc_cap = ctx->esc_cap;
  if (ctx->let_on) {
    a.let_num = static_cast<unsigned long long*>(ctx->d_let_num.p);
    a.let_den = static_cast<unsigned long long*>(ctx->d_let_den.p);
  }
  if (ctx->dlog_cap) {
    a.dlog = static_cast<DepositRecord*>(ctx->d_dlog.p);
    a.dlog_count = static_cast<unsigned long long*>(ctx->d_dlog_cnt.p);
    a.dlog_cap = ctx->dlog_cap;
  }
  return a;
}

CascadeArgs cascade_args(pmc_ctx* ctx) {
  CascadeArgs c{};
  c.nuclei = static_cast<const NucleusModel*>(ctx->d_nuclei.p);
  c.btab = static_cast<const float*>(ctx->d_btab.p);
  c.n_nuc = ctx->phys.n_nuc;
  c.g = ctx->geo;
  c.tally = static_cast<unsigned long long*>(ctx->d_tally.p);
  c.B = ctx->opt.n_batches;
  c.seed = static_cast<const unsigned long long*>(ctx->d_seed.p);
  c.cnt = static_cast<Counters*>(ctx->d_counters.p);
  c.hist = static_cast<long long*>(ctx->d_hist.p);
  c.hist_n = ctx->hist_n;
  if (ctx->dlog_cap) {
    c.dlog = static_cast<DepositRecord*>(ctx->d_dlog.p);
    c.dlog_count = static_cast<unsigned long long*>(ctx->d_dlog_cnt.p);
    c.dlog_cap = ctx->dlog_cap;
  }
  return c;
}

// Enqueues the primaries w0..w1-1 (phase space into qin, transport) and the event stage of
// their non-elastic collisions (cascade + evaporation, or the learned stand-in); secondary
// protons go to qout, counted in *qout_count, for the drain.
int enqueue_primaries(pmc_ctx* ctx, const RunPlan& rp, cudaStream_t s, uint64_t w0, uint64_t w1, Particle* qin,
                      Particle* qout, unsigned* qout_count, Particle* qne, unsigned* qne_count, unsigned* work,
                      unsigned* cwork, unsigned* rcount) {
  TransportArgs a = transport_args(ctx);
  a.w_begin = w0;
  a.w_end = w1;
  a.qin = qin;
  a.qin_cap = static_cast<unsigned>(ctx->q_cap);
  a.qsec = qout;
  a.qsec_count = qout_count;
  a.qsec_cap = static_cast<unsigned>(ctx->q_cap);
  a.qne = qne;
  a.qne_count = qne_count;
  a.qne_cap = static_cast<unsigned>(ctx->q_cap);
  a.work = work;
  int rc;
  if ((rc = mark(ctx, s, 0, true))) return rc;
  CK(launch_transport(a, rp.grid_t, ctx->block, rp.smem, s));
  if ((rc = mark(ctx, s, 0, false, 2))) return rc;   // phase space + transport
  if (ctx->mode == PMC_SURROGATE) {
    const float* P = static_cast<const float*>(ctx->d_sp.p);
    const unsigned cap = static_cast<unsigned>(ctx->q_cap);
    const int grid = ctx->n_sm * 2;   // two blocks per SM: 112 KB of shared memory and 256 TMEM columns each
    if ((rc = mark(ctx, s, 2, true))) return rc;
    CK(launch_surrogate_events(qne_count, cap, qne, static_cast<const int*>(ctx->d_nuc_slot.p), a.seed, ctx->d_swb.p,
                               P, a.tally, a.B, qout, qout_count, cap, a.cnt, a.hist, a.hist_n, grid, s));
    if ((rc = mark(ctx, s, 2, false))) return rc;
    return PMC_OK;
  }
  CascadeArgs c = cascade_args(ctx);
  c.qne = qne;
  c.qne_count = qne_count;
  c.qne_cap = static_cast<unsigned>(ctx->q_cap);
  c.qsec = qout;
  c.qsec_count = qout_count;
  c.qsec_cap = static_cast<unsigned>(ctx->q_cap);
  const int ri = (qne == static_cast<Particle*>(ctx->d_q[5].p)) ? 1 : 0;   // which stream's buffers
  c.rec = static_cast<EvapRecord*>(ctx->d_rec[ri].p);
  c.rec_cap = static_cast<unsigned>(ctx->d_rec[ri].n / sizeof(EvapRecord));
  c.rec_count = rcount;
  c.work = cwork;
  if ((rc = mark(ctx, s, 2, true))) return rc;
  CK(launch_cascade(c, s));
  if ((rc = mark(ctx, s, 2, false, 2))) return rc;   // cascade + evaporation
  return PMC_OK;
}

// The drain's buffers of queue set qs (0, 1): its control block and the ready marks of its
// particle, event and residual-nucleus queues.
DrainCtl* drain_ctl(pmc_ctx* ctx, int qs) {
  return reinterpret_cast<DrainCtl*>(static_cast<unsigned char*>(ctx->d_drain.p) + qs * sizeof(DrainCtl));
}
unsigned* drain_ready(pmc_ctx* ctx, int qs, int which) {
  unsigned* r = reinterpret_cast<unsigned*>(static_cast<unsigned char*>(ctx->d_drain.p) + 2 * sizeof(DrainCtl));
  return r + (3 * qs + which) * ctx->q_cap;
}
size_t drain_buffer_bytes(size_t q_cap) { return 2 * sizeof(DrainCtl) + 6 * q_cap * sizeof(unsigned); }

// Enqueues the drain of a sub-group: its particle queue pq already holds *pq_n the protons of
// the first generation; its events, if eq_n is given, are still queued in eq.
int enqueue_drain(pmc_ctx* ctx, const RunPlan& rp, cudaStream_t s, int qs, Particle* pq, const unsigned* pq_n,
                  Particle* eq, const unsigned* eq_n) {
  DrainArgs d{};
  d.t = transport_args(ctx);
  d.c = cascade_args(ctx);
  d.pq = pq;
  d.pq_ready = drain_ready(ctx, qs, 0);
  d.pq_cap = static_cast<unsigned>(ctx->q_cap);
  d.pq_n0 = pq_n;
  d.eq = eq;
  d.eq_ready = drain_ready(ctx, qs, 1);
  d.eq_cap = static_cast<unsigned>(ctx->q_cap);
  d.eq_n0 = eq_n;
  d.xq = static_cast<EvapRecord*>(ctx->d_rec[qs].p);   // free again: the evaporation kernel has run
  d.xq_ready = drain_ready(ctx, qs, 2);
  d.xq_cap = static_cast<unsigned>(ctx->d_rec[qs].n / sizeof(EvapRecord));
  d.ctl = drain_ctl(ctx, qs);
  if (ctx->drain_debug) {
    d.phantom = 1;
    d.idle_limit = 4096;
  }
  int rc;
  if ((rc = mark(ctx, s, 1, true))) return rc;
  CK(launch_drain(d, rp.grid_d, ctx->block, rp.smem_d, s));
  if ((rc = mark(ctx, s, 1, false, 2))) return rc;   // control block set-up + drain
  return PMC_OK;
}

StatsArgs stats_args(pmc_ctx* ctx) {
  StatsArgs sa{};
  sa.tally = static_cast<const unsigned long long*>(ctx->d_tally.p);
  sa.B = ctx->opt.n_batches;
  sa.n_vox = ctx->n_vox;
  sa.g = ctx->geo;
  sa.phys = static_cast<const Physics*>(ctx->d_phys.p);
  sa.dose = static_cast<double*>(ctx->d_dose.p);
  sa.sigma = static_cast<double*>(ctx->d_sigma.p);
  if (ctx->let_on) {
    sa.let_num = static_cast<const unsigned long long*>(ctx->d_let_num.p);
    sa.let_den = static_cast<const unsigned long long*>(ctx->d_let_den.p);
    sa.let = static_cast<double*>(ctx->d_let.p);
    sa.let_sigma = static_cast<double*>(ctx->d_let_sigma.p);
  }
  return sa;
}

// Count slots per sub-group: [0] unused (the primaries' count is the work range), [1] protons
// queued for the drain, [2] events of the primaries, [3] transport work counter, [4] cascade
// work counter, [5] residual nuclei.
constexpr int kSlots = 8;

int enqueue_run(pmc_ctx* ctx, const RunPlan& rp, cudaStream_t s) {
  ctx->n_events_used = 0;
  ctx->event_kind.clear();
  ctx->event_kernels.clear();
  CK(cudaMemsetAsync(ctx->d_tally.p, 0, static_cast<size_t>(ctx->n_vox) * ctx->opt.n_batches * 8, s));
  CK(cudaMemsetAsync(ctx->d_counters.p, 0, sizeof(Counters), s));
  CK(cudaMemsetAsync(ctx->d_counts.p, 0, static_cast<size_t>(rp.n_chunks) * kSlots * sizeof(unsigned), s));
  if (ctx->d_hist.p) CK(cudaMemsetAsync(ctx->d_hist.p, 0, ctx->hist_n * 4 * sizeof(long long), s));
  if (ctx->dlog_cap) CK(cudaMemsetAsync(ctx->d_dlog_cnt.p, 0, sizeof(unsigned long long), s));
  if (ctx->let_on) {
    CK(cudaMemsetAsync(ctx->d_let_num.p, 0, static_cast<size_t>(ctx->n_vox) * ctx->opt.n_batches * 8, s));
    CK(cudaMemsetAsync(ctx->d_let_den.p, 0, static_cast<size_t>(ctx->n_vox) * ctx->opt.n_batches * 8, s));
  }
  unsigned* counts = static_cast<unsigned*>(ctx->d_counts.p);
  Particle* q[kQueues];
  for (int i = 0; i < kQueues; ++i) q[i] = static_cast<Particle*>(ctx->d_q[i].p);
  // Per sub-group: the primaries (phase space, transport), the event stage of their
  // non-elastic collisions (cascade and evaporation, or the learned stand-in), then the drain
  // of everything that left (every later generation, with the full cascade, in one launch).
  // Sub-groups alternate between two streams (forked and joined inside the graph): the
  // latency-bound drain of one sub-group overlaps the full-width launches of the next.  Each
  // stream has its own three queues; tallies and counters are shared through atomics.
  const bool two = rp.n_chunks > 1;
  if (two) {
    CK(cudaEventRecord(ctx->fork_ev, s));
    CK(cudaStreamWaitEvent(ctx->stream2, ctx->fork_ev, 0));
  }
  for (int c = 0; c < rp.n_chunks; ++c) {
    cudaStream_t sc = (two && (c & 1)) ? ctx->stream2 : s;
    Particle** qs = q + 3 * ((two && (c & 1)) ? 1 : 0);
    unsigned* cs = counts + static_cast<size_t>(c) * kSlots;
    const uint64_t w0 = static_cast<uint64_t>(c) * rp.chunk;
    const uint64_t w1 = std::min<uint64_t>(rp.n, w0 + rp.chunk);
    int rc = enqueue_primaries(ctx, rp, sc, w0, w1, qs[0], qs[1], cs + 1, qs[2], cs + 2, cs + 3, cs + 4, cs + 5);
    if (rc) return rc;
    rc = enqueue_drain(ctx, rp, sc, (two && (c & 1)) ? 1 : 0, qs[1], cs + 1, qs[2], nullptr);
    if (rc) return rc;
  }
  if (two) {
    CK(cudaEventRecord(ctx->join_ev, ctx->stream2));
    CK(cudaStreamWaitEvent(s, ctx->join_ev, 0));
  }
  int rc;
  if ((rc = mark(ctx, s, 3, true))) return rc;
  CK(launch_stats(stats_args(ctx), s));
  if ((rc = mark(ctx, s, 3, false))) return rc;
  return PMC_OK;
}

}  // namespace

extern "C" {

int pmc_transport(pmc_ctx* ctx, uint64_t n_histories, uint64_t seed, int mode, void* stream) {
  if (!ctx) return PMC_E_INVALID;
  if (!ctx->tuned && ctx->have_materials && ctx->have_phantom && !ctx->spots.empty() &&
      (mode == PMC_FULL_CASCADE || mode == PMC_SURROGATE) && n_histories > 0 && n_histories <= 0xFFFFFFFFull) {
    const int rc = pmc_autotune(ctx, n_histories, seed ^ 0x5bd1e995ull, nullptr, nullptr);
    if (rc) return rc;
  }
  if (!ctx->have_materials || !ctx->have_phantom) return fail(ctx, PMC_E_INVALID, "load materials and phantom first");
  if (ctx->spots.empty()) return fail(ctx, PMC_E_INVALID, "no spots");
  if (mode != PMC_FULL_CASCADE && mode != PMC_SURROGATE) return fail(ctx, PMC_E_INVALID, "unknown mode %d", mode);
  if (mode == PMC_SURROGATE && !ctx->surr_trained)
    return fail(ctx, PMC_E_INVALID, "the surrogate is not trained (pmc_train_surrogate or pmc_surrogate_load)");
  if (ctx->dlog_cap && (mode != PMC_FULL_CASCADE || ctx->let_on || ctx->d_mol.p || ctx->d_vav.p))
    return fail(ctx, PMC_E_INVALID, "the deposit log runs the full cascade with Highland, Bohr and no LET only");
  if (n_histories == 0) return fail(ctx, PMC_E_INVALID, "n_histories must be > 0");
  if (n_histories > 0xFFFFFFFFull) return fail(ctx, PMC_E_INVALID, "at most 2^32-1 histories per call");
  double wsum = 0.0;
  for (const auto& sp : ctx->spots) wsum += sp.weight;
  if (!(wsum > 0.0)) return fail(ctx, PMC_E_INVALID, "spot weights sum to zero");
  try {
    cudaSetDevice(ctx->opt.device);
    cudaStream_t s = stream ? static_cast<cudaStream_t>(stream) : ctx->stream;
    // spots in work order (highest energy first; long histories start early)
    std::vector<uint64_t> cnt = split_histories(ctx->spots, n_histories);
    std::vector<uint64_t> hfirst(ctx->spots.size());
    uint64_t acc = 0;
    for (size_t i = 0; i < cnt.size(); ++i) { hfirst[i] = acc; acc += cnt[i]; }
    std::vector<size_t> order(ctx->spots.size());
    std::iota(order.begin(), order.end(), 0);
    std::stable_sort(order.begin(), order.end(), [&](size_t a, size_t b) { return ctx->spots[a].E > ctx->spots[b].E; });
    std::vector<SpotDev> sd;
    uint64_t wacc = 0;
    for (size_t k : order) {
      if (cnt[k] == 0) continue;
      const pmc_spot& p = ctx->spots[k];
      const double dn = std::sqrt(p.u * p.u + p.v * p.v + p.w * p.w);
      SpotDev d{};
      d.E = static_cast<float>(p.E); d.sE = static_cast<float>(p.sigma_E);
      d.x = static_cast<float>(p.x); d.y = static_cast<float>(p.y);
      d.sx = static_cast<float>(p.sigma_x); d.sy = static_cast<float>(p.sigma_y);
      d.u = static_cast<float>(p.u / dn); d.v = static_cast<float>(p.v / dn); d.w = static_cast<float>(p.w / dn);
      d.h_first = hfirst[k];
      d.w_first = wacc;
      wacc += cnt[k];
      sd.push_back(d);
    }
    RunPlan rp{};
    rp.n = n_histories;
    // default sub-group: the whole run up to 2^22 histories (measured on GB300: for
    // 1e6 histories one sub-group is as fast as two and faster than four)
    int64_t chunk = ctx->chunk > 0 ? ctx->chunk : (1ll << 22);
    rp.chunk = std::min<int64_t>(chunk, static_cast<int64_t>(n_histories));
    rp.n_chunks = static_cast<int>((n_histories + rp.chunk - 1) / rp.chunk);
    rp.smem = transport_smem_bytes(ctx->phys.n_cls, ctx->phys.n_mat, ctx->d_mol.p != nullptr);
    int bps = 0;
    CK(transport_occupancy(ctx->block, rp.smem, &bps));
    if (bps < 1)
      return fail(ctx, PMC_E_CUDA, "transport kernel does not fit (block %d, smem %zu)", ctx->block, rp.smem);
    rp.grid_t = ctx->n_sm * bps;
    rp.grid_c = ctx->n_sm * 8;      // one tile of 128 events per block for typical event counts
    rp.smem_d = drain_smem_bytes(ctx->phys.n_cls, ctx->phys.n_mat, ctx->d_mol.p != nullptr, ctx->phys.n_nuc);
    int bpd = 0;
    CK(drain_occupancy(ctx->block, rp.smem_d, &bpd));
    if (bpd < 1) return fail(ctx, PMC_E_CUDA, "drain kernel does not fit (block %d, smem %zu)", ctx->block, rp.smem_d);
    rp.grid_d = ctx->n_sm * bpd;
    // buffers
    int rc;
    const size_t B = ctx->opt.n_batches;
    if ((rc = dalloc(ctx, ctx->d_tally, static_cast<size_t>(ctx->n_vox) * B * 8))) return rc;
    if ((rc = dalloc(ctx, ctx->d_dose, static_cast<size_t>(ctx->n_vox) * 8))) return rc;
    if ((rc = dalloc(ctx, ctx->d_sigma, static_cast<size_t>(ctx->n_vox) * 8))) return rc;
    if (ctx->let_on) {
      if ((rc = dalloc(ctx, ctx->d_let_num, static_cast<size_t>(ctx->n_vox) * B * 8))) return rc;
      if ((rc = dalloc(ctx, ctx->d_let_den, static_cast<size_t>(ctx->n_vox) * B * 8))) return rc;
      if ((rc = dalloc(ctx, ctx->d_let, static_cast<size_t>(ctx->n_vox) * 8))) return rc;
      if ((rc = dalloc(ctx, ctx->d_let_sigma, static_cast<size_t>(ctx->n_vox) * 8))) return rc;
    }
    if ((rc = dalloc(ctx, ctx->d_counters, sizeof(Counters)))) return rc;
    if ((rc = dalloc(ctx, ctx->d_counts, static_cast<size_t>(rp.n_chunks) * kSlots * sizeof(unsigned)))) return rc;
    if ((rc = dalloc(ctx, ctx->d_seed, sizeof(uint64_t)))) return rc;
    if ((rc = dalloc(ctx, ctx->d_spots, sd.size() * sizeof(SpotDev)))) return rc;
    ctx->n_spots_dev = static_cast<int>(sd.size());   // spots without histories are not in the table
    const size_t qcap = static_cast<size_t>(std::max<int64_t>(rp.chunk, 1024));
    for (int i = 0; i < kQueues; ++i)
      if ((rc = dalloc(ctx, ctx->d_q[i], qcap * sizeof(Particle)))) return rc;
    ctx->q_cap = ctx->d_q[0].n / sizeof(Particle);
    if (!ctx->d_drain.p || ctx->drain_qcap != ctx->q_cap) {
      // control blocks and ready marks start at zero together (the stamps count up from
      // there), again whenever the marks' layout changes with the queue capacity
      if ((rc = dalloc(ctx, ctx->d_drain, drain_buffer_bytes(ctx->q_cap)))) return rc;
      CK(cudaMemsetAsync(ctx->d_drain.p, 0, ctx->d_drain.n, s));
      ctx->drain_qcap = ctx->q_cap;
    }
    // residual nuclei between cascade and evaporation (and inside the drain, in either mode)
    for (int si = 0; si < 2; ++si)
      if ((rc = dalloc(ctx, ctx->d_rec[si], ctx->q_cap * sizeof(EvapRecord)))) return rc;
    ctx->mode = mode;
    CK(cudaMemcpyAsync(ctx->d_spots.p, sd.data(), sd.size() * sizeof(SpotDev), cudaMemcpyHostToDevice, s));
    CK(cudaMemcpyAsync(ctx->d_seed.p, &seed, sizeof(uint64_t), cudaMemcpyHostToDevice, s));
    // graph of the whole run, rebuilt when its shape changes
    char key[256];
    std::snprintf(key, sizeof(key), "%llu/%lld/%zu/%d/%d/%lld/%p/%p/%p/%d/%p/%d", (unsigned long long)n_histories,
                  (long long)rp.chunk, sd.size(), ctx->block, ctx->opt.n_batches, ctx->n_vox, ctx->d_tally.p,
                  ctx->d_hist.p, ctx->let_on ? ctx->d_let_num.p : nullptr, ctx->profile + 3 * mode,
                  ctx->dlog_cap ? ctx->d_dlog.p : nullptr, ctx->drain_debug ? 1 : 0);
    if (!ctx->gexec || ctx->gkey != key) {
      if (ctx->gexec) { cudaGraphExecDestroy(ctx->gexec); ctx->gexec = nullptr; }
      cudaGraph_t graph;
      CK(cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal));
      rc = enqueue_run(ctx, rp, s);
      cudaError_t e = cudaStreamEndCapture(s, &graph);
      if (rc) { if (e == cudaSuccess) cudaGraphDestroy(graph); return rc; }
      if (e != cudaSuccess) return fail(ctx, PMC_E_CUDA, "graph capture: %s", cudaGetErrorString(e));
      e = cudaGraphInstantiate(&ctx->gexec, graph, 0);
      cudaGraphDestroy(graph);
      if (e != cudaSuccess) { ctx->gexec = nullptr; return fail(ctx, PMC_E_CUDA, "graph instantiate: %s", cudaGetErrorString(e)); }
      ctx->gkey = key;
    }
    CK(cudaGraphLaunch(ctx->gexec, s));
    CK(cudaStreamSynchronize(s));
    for (int k = 0; k < 4; ++k) {
      ctx->prof_ms[k] = 0.0;
      ctx->prof_launches[k] = 0;
      ctx->prof_kernels[k] = 0;
      ctx->prof_span[k] = 0.0;
    }
    if (ctx->profile && !ctx->event_kind.empty()) {
      double lo[4] = {1e300, 1e300, 1e300, 1e300}, hi[4] = {-1e300, -1e300, -1e300, -1e300};
      for (size_t i = 0; i < ctx->event_kind.size(); ++i) {
        float ms = 0.0f, t0 = 0.0f, t1 = 0.0f;
        const int k = ctx->event_kind[i];
        CK(cudaEventElapsedTime(&ms, ctx->events[2 * i], ctx->events[2 * i + 1]));
        CK(cudaEventElapsedTime(&t0, ctx->events[0], ctx->events[2 * i]));
        CK(cudaEventElapsedTime(&t1, ctx->events[0], ctx->events[2 * i + 1]));
        ctx->prof_ms[k] += ms;
        ctx->prof_launches[k] += 1;
        ctx->prof_kernels[k] += i < ctx->event_kernels.size() ? ctx->event_kernels[i] : 1;
        lo[k] = std::min(lo[k], static_cast<double>(t0));
        hi[k] = std::max(hi[k], static_cast<double>(t1));
      }
      for (int k = 0; k < 4; ++k)
        if (ctx->prof_launches[k]) ctx->prof_span[k] = hi[k] - lo[k];
    }
    Counters hc{};
    CK(cudaMemcpyAsync(&hc, ctx->d_counters.p, sizeof(Counters), cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    CK(cudaGetLastError());
    pmc_ledger& L = ctx->last;
    L.incident = static_cast<int64_t>(hc.incident);
    L.deposited = static_cast<int64_t>(hc.deposited);
    L.escaped = static_cast<int64_t>(hc.escaped);
    L.binding = static_cast<int64_t>(hc.binding);
    L.histories = static_cast<int64_t>(n_histories);
    L.steps = static_cast<int64_t>(hc.steps);
    L.elastic = static_cast<int64_t>(hc.elastic);
    L.inelastic = static_cast<int64_t>(hc.inelastic);
    L.secondaries = static_cast<int64_t>(hc.secondaries);
    L.transparent = static_cast<int64_t>(hc.transparent);
    L.inc_retries = static_cast<int64_t>(hc.inc_retries);
    L.queue_high_water = 0;
    L.generations = 2;   // the primaries, then the drain of all later generations
    L.dropped = static_cast<int64_t>(hc.dropped);
    L.errors = static_cast<int64_t>(hc.errors);
    L.surrogate_events = static_cast<int64_t>(hc.surrogate_events);
    ctx->steps_primary = static_cast<int64_t>(hc.steps_primary);
    ctx->have_run = true;
    ctx->let_valid = ctx->let_on;
    if (hc.dropped) return fail(ctx, PMC_E_QUEUE_OVERFLOW, "%llu particles did not fit a queue", (unsigned long long)hc.dropped);
    if (hc.errors)
      return fail(ctx, PMC_E_TIMEOUT, "%llu particles exceeded the step limit or device waits timed out",
                  (unsigned long long)hc.errors);
    return PMC_OK;
  } catch (...) {
    return fail(ctx, PMC_E_INVALID, "exception in transport");
  }
}

int pmc_autotune(pmc_ctx* ctx, uint64_t n_histories, uint64_t seed, int* block_out, int64_t* chunk_out) {
  if (!ctx) return PMC_E_INVALID;
  const int blocks[3] = {128, 192, 256};
  const int64_t n = static_cast<int64_t>(n_histories);
  std::vector<int64_t> chunks = {n};
  if (n >= (1ll << 17)) chunks.push_back((n + 1) / 2);
  double best = 1e300;
  int best_b = ctx->block;
  int64_t best_c = ctx->chunk;
  const bool was_tuned = ctx->tuned;
  ctx->tuned = true;                      // the trial transports must not recurse into tuning
  for (int b : blocks) {
    for (int64_t c : chunks) {
      ctx->block = b;
      ctx->chunk = c;
      double t = 1e300;
      for (int rep = 0; rep < 2; ++rep) {   // the first run also builds the graph
        const auto t0 = std::chrono::steady_clock::now();
        const int rc = pmc_transport(ctx, n_histories, seed + rep, PMC_FULL_CASCADE, nullptr);
        const auto t1 = std::chrono::steady_clock::now();
        if (rc) { ctx->tuned = was_tuned; return rc; }
        if (rep) t = std::chrono::duration<double>(t1 - t0).count();
      }
      if (t < best) { best = t; best_b = b; best_c = c; }
    }
  }
  ctx->block = best_b;
  ctx->chunk = best_c;
  if (block_out) *block_out = best_b;
  if (chunk_out) *chunk_out = best_c;
  return PMC_OK;
}

int pmc_read_dose(pmc_ctx* ctx, double* dose, double* sigma, size_t n) {
  if (!ctx) return PMC_E_INVALID;
  if (!ctx->have_run) return fail(ctx, PMC_E_INVALID, "no transport has run");
  if (n != static_cast<size_t>(ctx->n_vox)) return fail(ctx, PMC_E_INVALID, "n_voxels %zu != %lld", n, ctx->n_vox);
  cudaSetDevice(ctx->opt.device);
  if (dose) CK(cudaMemcpyAsync(dose, ctx->d_dose.p, n * 8, cudaMemcpyDeviceToHost, ctx->stream));
  if (sigma) CK(cudaMemcpyAsync(sigma, ctx->d_sigma.p, n * 8, cudaMemcpyDeviceToHost, ctx->stream));
  CK(cudaStreamSynchronize(ctx->stream));
  return PMC_OK;
}

int pmc_read_let(pmc_ctx* ctx, double* let_d, double* sigma, size_t n) {
  if (!ctx) return PMC_E_INVALID;
  if (!ctx->let_valid) return fail(ctx, PMC_E_INVALID, "no transport with LET scoring has run (pmc_enable_let)");
  if (n != static_cast<size_t>(ctx->n_vox)) return fail(ctx, PMC_E_INVALID, "n_voxels %zu != %lld", n, ctx->n_vox);
  cudaSetDevice(ctx->opt.device);
  if (let_d) CK(cudaMemcpyAsync(let_d, ctx->d_let.p, n * 8, cudaMemcpyDeviceToHost, ctx->stream));
  if (sigma) CK(cudaMemcpyAsync(sigma, ctx->d_let_sigma.p, n * 8, cudaMemcpyDeviceToHost, ctx->stream));
  CK(cudaStreamSynchronize(ctx->stream));
  return PMC_OK;
}

int pmc_read_let_tally(pmc_ctx* ctx, int64_t* num, int64_t* den, size_t n) {
  if (!ctx) return PMC_E_INVALID;
  if (!ctx->let_valid) return fail(ctx, PMC_E_INVALID, "no transport with LET scoring has run (pmc_enable_let)");
  const size_t need = static_cast<size_t>(ctx->n_vox) * ctx->opt.n_batches;
  if (n != need) return fail(ctx, PMC_E_INVALID, "LET tallies have %zu entries", need);
  cudaSetDevice(ctx->opt.device);
  if (num) CK(cudaMemcpyAsync(num, ctx->d_let_num.p, n * 8, cudaMemcpyDeviceToHost, ctx->stream));
  if (den) CK(cudaMemcpyAsync(den, ctx->d_let_den.p, n * 8, cudaMemcpyDeviceToHost, ctx->stream));
  CK(cudaStreamSynchronize(ctx->stream));
  return PMC_OK;
}

int pmc_read_tally(pmc_ctx* ctx, int64_t* tally, size_t n) {
  if (!ctx || !tally) return PMC_E_INVALID;
  if (!ctx->have_run) return fail(ctx, PMC_E_INVALID, "no transport has run");
  const size_t need = static_cast<size_t>(ctx->n_vox) * ctx->opt.n_batches;
  if (n != need) return fail(ctx, PMC_E_INVALID, "tally has %zu entries", need);
  cudaSetDevice(ctx->opt.device);
  CK(cudaMemcpyAsync(tally, ctx->d_tally.p, n * 8, cudaMemcpyDeviceToHost, ctx->stream));
  CK(cudaStreamSynchronize(ctx->stream));
  return PMC_OK;
}

int pmc_read_ledger(pmc_ctx* ctx, pmc_ledger* out) {
  if (!ctx || !out) return PMC_E_INVALID;
  *out = ctx->last;
  return PMC_OK;
}

int pmc_read_history_ledger(pmc_ctx* ctx, int64_t* out, uint64_t n) {
  if (!ctx || !out) return PMC_E_INVALID;
  if (n > ctx->hist_n) return fail(ctx, PMC_E_INVALID, "history ledger holds %llu histories", (unsigned long long)ctx->hist_n);
  cudaSetDevice(ctx->opt.device);
  CK(cudaMemcpyAsync(out, ctx->d_hist.p, n * 4 * sizeof(long long), cudaMemcpyDeviceToHost, ctx->stream));
  CK(cudaStreamSynchronize(ctx->stream));
  return PMC_OK;
}

int pmc_read_escape_record(pmc_ctx* ctx, float* out, uint64_t cap, uint64_t* n) {
  if (!ctx || !out || !n) return PMC_E_INVALID;
  cudaSetDevice(ctx->opt.device);
  Counters hc{};
  CK(cudaMemcpy(&hc, ctx->d_counters.p, sizeof(Counters), cudaMemcpyDeviceToHost));
  const uint64_t m = std::min<uint64_t>(std::min<uint64_t>(hc.esc_count, ctx->esc_cap), cap);
  if (m) CK(cudaMemcpy(out, ctx->d_esc.p, m * 8 * sizeof(float), cudaMemcpyDeviceToHost));
  *n = m;
  return PMC_OK;
}

int pmc_debug_philox(const uint32_t* ctr, const uint32_t* key, uint32_t* out, int n) {
  if (!ctr || !key || !out || n < 0) return PMC_E_INVALID;
  if (n == 0) return PMC_OK;
  void *dc = nullptr, *dout = nullptr;
  if (cudaMalloc(&dc, n * 16ull) != cudaSuccess || cudaMalloc(&dout, n * 16ull) != cudaSuccess) {
    cudaFree(dc);
    return PMC_E_OOM;
  }
  int rc = PMC_OK;
  if (cudaMemcpy(dc, ctr, n * 16ull, cudaMemcpyHostToDevice) != cudaSuccess ||
      launch_debug_philox(static_cast<const uint4*>(dc), make_uint2(key[0], key[1]), static_cast<uint4*>(dout), n,
                          nullptr) != cudaSuccess ||
      cudaMemcpy(out, dout, n * 16ull, cudaMemcpyDeviceToHost) != cudaSuccess)
    rc = PMC_E_CUDA;
  cudaFree(dc);
  cudaFree(dout);
  return rc;
}

int pmc_debug_tables(pmc_ctx* ctx, int material, const double* E, double* r_out, double* e_out, int n) {
  if (!ctx || !E || !r_out || !e_out || n < 0) return PMC_E_INVALID;
  if (!ctx->have_materials || material < 0 || material >= ctx->phys.n_mat)
    return fail(ctx, PMC_E_INVALID, "bad material");
  cudaSetDevice(ctx->opt.device);
  DevBuf b;
  int rc = dalloc(ctx, b, n * 24ull);
  if (rc) return rc;
  double* dE = static_cast<double*>(b.p);
  CK(cudaMemcpy(dE, E, n * 8ull, cudaMemcpyHostToDevice));
  CK(launch_debug_tables(static_cast<const Physics*>(ctx->d_phys.p), static_cast<const float2*>(ctx->d_rt.p),
                         static_cast<const float2*>(ctx->d_et.p), ctx->phys.mat[material].cls, dE, dE + n, dE + 2 * n,
                         n, ctx->stream));
  CK(cudaStreamSynchronize(ctx->stream));
  CK(cudaMemcpy(r_out, dE + n, n * 8ull, cudaMemcpyDeviceToHost));
  CK(cudaMemcpy(e_out, dE + 2 * n, n * 8ull, cudaMemcpyDeviceToHost));
  dfree(ctx, b);
  return PMC_OK;
}

int pmc_debug_inc(pmc_ctx* ctx, int nuclide, double E, uint64_t seed, uint64_t pid0, int n, double* summary,
                  double* products, int cap) {
  if (!ctx || !summary || !products || n < 0 || cap < 1) return PMC_E_INVALID;
  if (!ctx->have_materials || nuclide < 0 || nuclide >= ctx->phys.n_nuc || ctx->nucs[nuclide].A < 2)
    return fail(ctx, PMC_E_INVALID, "bad nuclide");
  cudaSetDevice(ctx->opt.device);
  DevBuf b;
  const size_t ns = n * 8ull, np = static_cast<size_t>(n) * cap * 5;
  int rc = dalloc(ctx, b, (ns + np) * 8);
  if (rc) return rc;
  double* d = static_cast<double*>(b.p);
  CK(cudaMemset(d, 0, (ns + np) * 8));
  CK(launch_debug_inc(static_cast<const NucleusModel*>(ctx->d_nuclei.p) + nuclide,
                      static_cast<const float*>(ctx->d_btab.p), static_cast<float>(E), seed, pid0, n, d, d + ns, cap,
                      ctx->stream));
  CK(cudaStreamSynchronize(ctx->stream));
  CK(cudaMemcpy(summary, d, ns * 8, cudaMemcpyDeviceToHost));
  CK(cudaMemcpy(products, d + ns, np * 8, cudaMemcpyDeviceToHost));
  dfree(ctx, b);
  return PMC_OK;
}

int pmc_nonelastic_events(pmc_ctx* ctx, int nuclide, double E, uint64_t n, uint64_t seed, uint64_t pid0,
                          pmc_event_yields* out) {
  if (!ctx || !out || !(E > 0.0) || !(E < 1.0e4)) return PMC_E_INVALID;
  if (!ctx->have_materials || nuclide < 0 || nuclide >= ctx->phys.n_nuc || ctx->nucs[nuclide].A < 2)
    return fail(ctx, PMC_E_INVALID, "bad nuclide (a loaded nuclide with A >= 2)");
  cudaSetDevice(ctx->opt.device);
  int rc;
  if ((rc = dalloc(ctx, ctx->d_yields, sizeof(EventYields)))) return rc;
  if (!ctx->ev_a) {
    CK(cudaEventCreate(&ctx->ev_a));
    CK(cudaEventCreate(&ctx->ev_b));
  }
  EventYields* d = static_cast<EventYields*>(ctx->d_yields.p);
  CK(cudaEventRecord(ctx->ev_a, ctx->stream));
  CK(launch_inc_yields(static_cast<const NucleusModel*>(ctx->d_nuclei.p) + nuclide,
                       static_cast<const float*>(ctx->d_btab.p), static_cast<float>(E), seed, pid0, n, d, ctx->stream));
  CK(cudaEventRecord(ctx->ev_b, ctx->stream));
  EventYields h{};
  CK(cudaMemcpyAsync(&h, d, sizeof(h), cudaMemcpyDeviceToHost, ctx->stream));
  CK(cudaStreamSynchronize(ctx->stream));
  float ms = 0.0f;
  CK(cudaEventElapsedTime(&ms, ctx->ev_a, ctx->ev_b));
  *out = pmc_event_yields{};
  out->events = h.events;
  out->transparent = h.transparent;
  out->retries = h.retries;
  for (int k = 0; k < 6; ++k) {
    out->count[k] = h.count[k];
    out->energy[k] = static_cast<double>(h.energy[k]) * (1.0 / kFixD);
  }
  out->residual_T = static_cast<double>(h.residual) * (1.0 / kFixD);
  out->excitation_left = static_cast<double>(h.excitation) * (1.0 / kFixD);
  out->binding = static_cast<double>(h.binding) * (1.0 / kFixD);
  out->ms = ms;
  return PMC_OK;
}

int pmc_debug_elastic(pmc_ctx* ctx, int nuclide, double E, const double* u, double* out, int n) {
  if (!ctx || !u || !out || n < 0) return PMC_E_INVALID;
  if (!ctx->have_materials || nuclide < 0 || nuclide >= ctx->phys.n_nuc) return fail(ctx, PMC_E_INVALID, "bad nuclide");
  cudaSetDevice(ctx->opt.device);
  DevBuf b;
  int rc = dalloc(ctx, b, n * 64ull);
  if (rc) return rc;
  double* d = static_cast<double*>(b.p);
  CK(cudaMemcpy(d, u, n * 24ull, cudaMemcpyHostToDevice));
  CK(launch_debug_elastic(static_cast<const Physics*>(ctx->d_phys.p), nuclide, static_cast<float>(E), d, d + 3 * n, n,
                          ctx->stream));
  CK(cudaStreamSynchronize(ctx->stream));
  CK(cudaMemcpy(out, d + 3 * n, n * 40ull, cudaMemcpyDeviceToHost));
  dfree(ctx, b);
  return PMC_OK;
}

int pmc_debug_event_stage(pmc_ctx* ctx, int mode, const int* nuclide, const double* E, int n, uint64_t seed,
                          float* protons, uint64_t cap, uint64_t* n_protons, double* local) {
  if (!ctx || !nuclide || !E || n <= 0 || n > (1 << 24) || !n_protons || (cap && !protons)) return PMC_E_INVALID;
  if (!ctx->have_materials) return fail(ctx, PMC_E_INVALID, "load materials first");
  if (mode != PMC_FULL_CASCADE && mode != PMC_SURROGATE) return fail(ctx, PMC_E_INVALID, "unknown mode %d", mode);
  if (mode == PMC_SURROGATE && !ctx->surr_trained) return fail(ctx, PMC_E_INVALID, "the surrogate is not trained");
  std::vector<Particle> ev(static_cast<size_t>(n));
  for (int i = 0; i < n; ++i) {
    const int k = nuclide[i];
    if (k < 0 || k >= ctx->phys.n_nuc || ctx->phys.nuc[k].A < 2)
      return fail(ctx, PMC_E_INVALID, "event %d: nuclide %d has no non-elastic channel", i, k);
    if (!(E[i] > 0.0 && E[i] <= 400.0)) return fail(ctx, PMC_E_INVALID, "event %d: energy %g MeV", i, E[i]);
    Particle& r = ev[static_cast<size_t>(i)];
    r.x = r.y = r.z = 0.0f;
    r.u = r.v = 0.0f;
    r.w = 1.0f;
    r.E = static_cast<float>(E[i]);
    r.voxel = i;
    r.pid = static_cast<unsigned long long>(i);
    r.root = static_cast<unsigned>(i);
    r.target = k;
  }
  cudaSetDevice(ctx->opt.device);
  const unsigned qcap = 32u * static_cast<unsigned>(n) + 1024u;
  DevBuf d_ev, d_out, d_cnt, d_tal, d_ctr, d_seed, d_rec;
  auto release_all = [&] {
    cudaStreamSynchronize(ctx->stream);
    for (DevBuf* b : {&d_ev, &d_out, &d_cnt, &d_tal, &d_ctr, &d_seed, &d_rec}) dfree(ctx, *b);
  };
  int rc = 0;
  if ((rc = dalloc(ctx, d_ev, ev.size() * sizeof(Particle))) || (rc = dalloc(ctx, d_out, qcap * sizeof(Particle))) ||
      (rc = dalloc(ctx, d_cnt, 4 * sizeof(unsigned))) || (rc = dalloc(ctx, d_tal, static_cast<size_t>(n) * 8)) ||
      (rc = dalloc(ctx, d_ctr, sizeof(Counters))) || (rc = dalloc(ctx, d_seed, sizeof(uint64_t))) ||
      (mode == PMC_FULL_CASCADE && (rc = dalloc(ctx, d_rec, static_cast<size_t>(n) * sizeof(EvapRecord))))) {
    release_all();
    return rc;
  }
  cudaStream_t s = ctx->stream;
  unsigned* cnt = static_cast<unsigned*>(d_cnt.p);
  const unsigned nu = static_cast<unsigned>(n);
  cudaError_t e = cudaMemcpyAsync(d_ev.p, ev.data(), ev.size() * sizeof(Particle), cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess) e = cudaMemsetAsync(cnt, 0, 4 * sizeof(unsigned), s);
  if (e == cudaSuccess) e = cudaMemcpyAsync(cnt, &nu, sizeof(unsigned), cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess) e = cudaMemsetAsync(d_tal.p, 0, static_cast<size_t>(n) * 8, s);
  if (e == cudaSuccess) e = cudaMemsetAsync(d_ctr.p, 0, sizeof(Counters), s);
  if (e == cudaSuccess) e = cudaMemcpyAsync(d_seed.p, &seed, sizeof(uint64_t), cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess) {
    if (mode == PMC_FULL_CASCADE) {
      CascadeArgs c = cascade_args(ctx);
      c.tally = static_cast<unsigned long long*>(d_tal.p);
      c.B = 1;
      c.seed = static_cast<const unsigned long long*>(d_seed.p);
      c.cnt = static_cast<Counters*>(d_ctr.p);
      c.hist = nullptr;
      c.hist_n = 0;
      c.dlog = nullptr;
      c.dlog_count = nullptr;
      c.dlog_cap = 0;
      c.qne = static_cast<const Particle*>(d_ev.p);
      c.qne_count = cnt;
      c.qne_cap = nu;
      c.qsec = static_cast<Particle*>(d_out.p);
      c.qsec_count = cnt + 1;
      c.qsec_cap = qcap;
      c.work = cnt + 2;
      c.rec = static_cast<EvapRecord*>(d_rec.p);
      c.rec_count = cnt + 3;
      c.rec_cap = nu;
      e = launch_cascade(c, s);
    } else {
      e = launch_surrogate_events(cnt, nu, static_cast<const Particle*>(d_ev.p),
                                  static_cast<const int*>(ctx->d_nuc_slot.p),
                                  static_cast<const unsigned long long*>(d_seed.p), ctx->d_swb.p,
                                  static_cast<const float*>(ctx->d_sp.p), static_cast<unsigned long long*>(d_tal.p), 1,
                                  static_cast<Particle*>(d_out.p), cnt + 1, qcap, static_cast<Counters*>(d_ctr.p),
                                  nullptr, 0, ctx->n_sm * 2, s);
    }
  }
  unsigned hc[4] = {0, 0, 0, 0};
  Counters ctr{};
  if (e == cudaSuccess) e = cudaMemcpyAsync(hc, cnt, sizeof(hc), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaMemcpyAsync(&ctr, d_ctr.p, sizeof(Counters), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  const unsigned emitted = std::min(hc[1], qcap);
  std::vector<Particle> out(emitted);
  std::vector<long long> tal(local ? static_cast<size_t>(n) : 0);
  if (e == cudaSuccess && emitted)
    e = cudaMemcpy(out.data(), d_out.p, emitted * sizeof(Particle), cudaMemcpyDeviceToHost);
  if (e == cudaSuccess && local) e = cudaMemcpy(tal.data(), d_tal.p, static_cast<size_t>(n) * 8, cudaMemcpyDeviceToHost);
  release_all();
  if (e != cudaSuccess) return fail(ctx, PMC_E_CUDA, "event stage: %s", cudaGetErrorString(e));
  if (ctr.errors) return fail(ctx, PMC_E_TIMEOUT, "event stage: %llu device waits timed out", (unsigned long long)ctr.errors);
  *n_protons = emitted;
  const uint64_t k = std::min<uint64_t>(emitted, cap);
  for (uint64_t i = 0; i < k; ++i) {
    protons[3 * i] = static_cast<float>(out[i].root);
    protons[3 * i + 1] = out[i].E;
    protons[3 * i + 2] = out[i].w;
  }
  if (local)
    for (int i = 0; i < n; ++i) local[i] = static_cast<double>(tal[static_cast<size_t>(i)]) / 16777216.0;
  if (ctr.dropped || hc[1] > qcap) return fail(ctx, PMC_E_QUEUE_OVERFLOW, "event stage: proton queue full");
  if (emitted > cap) return fail(ctx, PMC_E_QUEUE_OVERFLOW, "%u protons, room for %llu", emitted, (unsigned long long)cap);
  return PMC_OK;
}

}  // extern "C"

// ---------------------------------------------------------------------------
// Transport without device allocation.
//
// Some callers cannot allocate device memory while they run a dose
// calculation: a real-time control loop may not call cudaMalloc (it can
// synchronise the device or stall behind other work), and a caller with its
// own fixed memory budget may have handed the whole GPU to its pool.  This
// entry point runs the same kernels as pmc_transport (the full cascade) but
// keeps every piece of scratch (particle queues, counters, spot table, seed)
// in one static device array; the caller supplies the output arrays.  It
// synchronises its stream before it returns, so it cannot run inside a stream
// callback or a stream capture.
//
// The array lives in every GPU that loads this library until the process
// exits.  All calls on a device share it and it keeps the last call's
// contents: each call clears what must start at zero.  Calls from several host
// threads are serialised per device by a lock (the call is synchronous, so this
// keeps their work from overlapping on the GPU).  The array's device address
// is looked up once per device, on the first call there, with that device
// current.
// ---------------------------------------------------------------------------
namespace {

constexpr size_t kNaQueue = static_cast<size_t>(PMC_NOALLOC_CHUNK) * sizeof(Particle);
constexpr size_t kNaRec = 3 * kNaQueue;   // queues: primaries' phase space, protons for the drain, events
constexpr size_t kNaCounters = kNaRec + static_cast<size_t>(PMC_NOALLOC_CHUNK) * sizeof(EvapRecord);
constexpr size_t kNaCounts = kNaCounters + 256;
constexpr size_t kNaSeed = kNaCounts + 256;
constexpr size_t kNaDrain = kNaSeed + 256;       // the drain's control block
constexpr size_t kNaReady = kNaDrain + 1024;     // ready marks of the drain's particle and event queues
static_assert(sizeof(DrainCtl) <= 1024, "the drain's control block fits its slot");
constexpr size_t kNaSpots = kNaReady + 3ull * PMC_NOALLOC_CHUNK * sizeof(unsigned);
constexpr size_t kNaBytes = kNaSpots + static_cast<size_t>(PMC_NOALLOC_MAX_SPOTS) * sizeof(SpotDev);
static_assert(kNaBytes == PMC_NOALLOC_SCRATCH_BYTES, "scratch size stated in pmc.h");
static_assert(sizeof(Counters) <= 256, "counters fit their slot");

static __device__ __align__(256) unsigned char g_noalloc_scratch[kNaBytes];

constexpr int kNaMaxDevices = 64;
struct NoallocSlot {
  std::once_flag once;             // the address lookup, once per device
  cudaError_t status = cudaSuccess;
  unsigned char* addr = nullptr;
  std::mutex run;                  // one call at a time per device
};
NoallocSlot g_noalloc[kNaMaxDevices];

}  // namespace

extern "C" int pmc_transport_noalloc(pmc_ctx* ctx, uint64_t n_histories, uint64_t seed, int64_t* tally,
                                     double* dose_gy, double* sigma_gy, void* stream) {
  if (!ctx) return PMC_E_INVALID;
  if (!ctx->have_materials || !ctx->have_phantom) return fail(ctx, PMC_E_INVALID, "load materials and phantom first");
  if (!tally) return fail(ctx, PMC_E_INVALID, "tally output is required");
  if ((dose_gy == nullptr) != (sigma_gy == nullptr)) return fail(ctx, PMC_E_INVALID, "give both dose and sigma, or neither");
  if (ctx->spots.empty()) return fail(ctx, PMC_E_INVALID, "no spots");
  if (n_histories == 0 || n_histories > 0xFFFFFFFFull) return fail(ctx, PMC_E_INVALID, "n_histories must be in [1, 2^32)");
  const int dev = ctx->opt.device;
  if (dev < 0 || dev >= kNaMaxDevices) return fail(ctx, PMC_E_INVALID, "device ordinal beyond %d", kNaMaxDevices);
  double wsum = 0.0;
  for (const auto& sp : ctx->spots) wsum += sp.weight;
  if (!(wsum > 0.0)) return fail(ctx, PMC_E_INVALID, "spot weights sum to zero");
  try {
    // spots in work order, as in pmc_transport
    std::vector<uint64_t> cnt = split_histories(ctx->spots, n_histories);
    std::vector<uint64_t> hfirst(ctx->spots.size());
    uint64_t acc = 0;
    for (size_t i = 0; i < cnt.size(); ++i) { hfirst[i] = acc; acc += cnt[i]; }
    std::vector<size_t> order(ctx->spots.size());
    std::iota(order.begin(), order.end(), 0);
    std::stable_sort(order.begin(), order.end(), [&](size_t a, size_t b) { return ctx->spots[a].E > ctx->spots[b].E; });
    std::vector<SpotDev> sd;
    uint64_t wacc = 0;
    for (size_t k : order) {
      if (cnt[k] == 0) continue;
      const pmc_spot& p = ctx->spots[k];
      const double dn = std::sqrt(p.u * p.u + p.v * p.v + p.w * p.w);
      SpotDev d{};
      d.E = static_cast<float>(p.E); d.sE = static_cast<float>(p.sigma_E);
      d.x = static_cast<float>(p.x); d.y = static_cast<float>(p.y);
      d.sx = static_cast<float>(p.sigma_x); d.sy = static_cast<float>(p.sigma_y);
      d.u = static_cast<float>(p.u / dn); d.v = static_cast<float>(p.v / dn); d.w = static_cast<float>(p.w / dn);
      d.h_first = hfirst[k];
      d.w_first = wacc;
      wacc += cnt[k];
      sd.push_back(d);
    }
    if (sd.size() > static_cast<size_t>(PMC_NOALLOC_MAX_SPOTS))
      return fail(ctx, PMC_E_INVALID, "%zu spots with histories exceed the no-allocation limit of %d", sd.size(),
                  PMC_NOALLOC_MAX_SPOTS);
    CK(cudaSetDevice(dev));
    NoallocSlot& slot = g_noalloc[dev];
    std::call_once(slot.once, [&slot] {
      void* p = nullptr;
      slot.status = cudaGetSymbolAddress(&p, g_noalloc_scratch);   // the current device is dev
      if (slot.status == cudaSuccess) slot.addr = static_cast<unsigned char*>(p);
      else cudaGetLastError();
    });
    if (slot.status != cudaSuccess)
      return fail(ctx, PMC_E_CUDA, "address of the no-allocation scratch: %s", cudaGetErrorString(slot.status));
    std::lock_guard<std::mutex> hold(slot.run);
    unsigned char* base = slot.addr;
    cudaStream_t s = stream ? static_cast<cudaStream_t>(stream) : ctx->stream;
    Particle* q[3];
    for (int i = 0; i < 3; ++i) q[i] = reinterpret_cast<Particle*>(base + i * kNaQueue);
    Counters* counters = reinterpret_cast<Counters*>(base + kNaCounters);
    unsigned* counts = reinterpret_cast<unsigned*>(base + kNaCounts);
    unsigned long long* dseed = reinterpret_cast<unsigned long long*>(base + kNaSeed);
    SpotDev* dspots = reinterpret_cast<SpotDev*>(base + kNaSpots);
    const size_t B = ctx->opt.n_batches;
    CK(cudaMemcpyAsync(dspots, sd.data(), sd.size() * sizeof(SpotDev), cudaMemcpyHostToDevice, s));
    CK(cudaMemcpyAsync(dseed, &seed, sizeof(uint64_t), cudaMemcpyHostToDevice, s));
    CK(cudaMemsetAsync(tally, 0, static_cast<size_t>(ctx->n_vox) * B * 8, s));
    CK(cudaMemsetAsync(counters, 0, sizeof(Counters), s));
    const size_t smem = transport_smem_bytes(ctx->phys.n_cls, ctx->phys.n_mat, ctx->d_mol.p != nullptr);
    int bps = 0;
    CK(transport_occupancy(ctx->block, smem, &bps));
    if (bps < 1)
      return fail(ctx, PMC_E_CUDA, "transport kernel does not fit (block %d, smem %zu)", ctx->block, smem);
    const int grid_t = ctx->n_sm * bps;
    TransportArgs ta{};
    ta.phys = static_cast<const Physics*>(ctx->d_phys.p);
    ta.rtab = static_cast<const float2*>(ctx->d_rt.p);
    ta.etab = static_cast<const float2*>(ctx->d_et.p);
    ta.stab = static_cast<const float*>(ctx->d_st.p);
    ta.mol = static_cast<const float4*>(ctx->d_mol.p);
    ta.vav = static_cast<const float*>(ctx->d_vav.p);
    ta.g = ctx->geo;
    ta.tally = reinterpret_cast<unsigned long long*>(tally);
    ta.B = ctx->opt.n_batches;
    ta.seed = dseed;
    ta.spots = dspots;
    ta.n_spots = static_cast<int>(sd.size());
    ta.cnt = counters;
    ta.qin_cap = ta.qsec_cap = ta.qne_cap = PMC_NOALLOC_CHUNK;
    CascadeArgs ca{};
    ca.nuclei = static_cast<const NucleusModel*>(ctx->d_nuclei.p);
    ca.btab = static_cast<const float*>(ctx->d_btab.p);
    ca.n_nuc = ctx->phys.n_nuc;
    ca.g = ctx->geo;
    ca.tally = ta.tally;
    ca.B = ta.B;
    ca.seed = dseed;
    ca.cnt = counters;
    ca.qne_cap = ca.qsec_cap = PMC_NOALLOC_CHUNK;
    ca.rec = reinterpret_cast<EvapRecord*>(base + kNaRec);
    ca.rec_cap = PMC_NOALLOC_CHUNK;
    DrainArgs da{};
    da.t = ta;
    da.c = ca;
    da.pq = q[1];
    da.pq_ready = reinterpret_cast<unsigned*>(base + kNaReady);
    da.pq_cap = PMC_NOALLOC_CHUNK;
    da.pq_n0 = counts + 1;
    da.eq = q[2];
    da.eq_ready = da.pq_ready + PMC_NOALLOC_CHUNK;
    da.eq_cap = PMC_NOALLOC_CHUNK;
    da.eq_n0 = nullptr;
    da.xq = reinterpret_cast<EvapRecord*>(base + kNaRec);   // free again once the evaporation kernel has run
    da.xq_ready = da.eq_ready + PMC_NOALLOC_CHUNK;
    da.xq_cap = PMC_NOALLOC_CHUNK;
    da.ctl = reinterpret_cast<DrainCtl*>(base + kNaDrain);
    const size_t smem_d = drain_smem_bytes(ctx->phys.n_cls, ctx->phys.n_mat, ctx->d_mol.p != nullptr, ctx->phys.n_nuc);
    int bpd = 0;
    CK(drain_occupancy(ctx->block, smem_d, &bpd));
    if (bpd < 1) return fail(ctx, PMC_E_CUDA, "drain kernel does not fit (block %d, smem %zu)", ctx->block, smem_d);
    // sub-groups of PMC_NOALLOC_CHUNK primaries: the primaries (phase space, transport, the
    // cascades of their events), then the drain of everything they left (counts: [1] protons
    // queued for the drain, [2] events, [3] transport work, [4] cascade work, [5] residuals)
    for (uint64_t w0 = 0; w0 < n_histories; w0 += PMC_NOALLOC_CHUNK) {
      const uint64_t w1 = std::min<uint64_t>(n_histories, w0 + PMC_NOALLOC_CHUNK);
      CK(cudaMemsetAsync(counts, 0, 8 * sizeof(unsigned), s));
      ta.w_begin = w0;
      ta.w_end = w1;
      ta.qin = q[0];
      ta.qsec = q[1];
      ta.qsec_count = counts + 1;
      ta.qne = q[2];
      ta.qne_count = counts + 2;
      ta.work = counts + 3;
      CK(launch_transport(ta, grid_t, ctx->block, smem, s));
      ca.qne = q[2];
      ca.qne_count = counts + 2;
      ca.qsec = q[1];
      ca.qsec_count = counts + 1;
      ca.work = counts + 4;
      ca.rec_count = counts + 5;
      CK(launch_cascade(ca, s));
      da.t = ta;
      da.c = ca;
      CK(launch_drain(da, ctx->n_sm * bpd, ctx->block, smem_d, s));
    }
    if (dose_gy) {
      StatsArgs sa{};
      sa.tally = ta.tally;
      sa.B = ta.B;
      sa.n_vox = ctx->n_vox;
      sa.g = ctx->geo;
      sa.phys = ta.phys;
      sa.dose = dose_gy;
      sa.sigma = sigma_gy;
      CK(launch_stats(sa, s));
    }
    Counters hc{};
    CK(cudaMemcpyAsync(&hc, counters, sizeof(Counters), cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    CK(cudaGetLastError());
    pmc_ledger& L = ctx->last;
    L = pmc_ledger{};
    L.incident = static_cast<int64_t>(hc.incident);
    L.deposited = static_cast<int64_t>(hc.deposited);
    L.escaped = static_cast<int64_t>(hc.escaped);
    L.binding = static_cast<int64_t>(hc.binding);
    L.histories = static_cast<int64_t>(n_histories);
    L.steps = static_cast<int64_t>(hc.steps);
    L.elastic = static_cast<int64_t>(hc.elastic);
    L.inelastic = static_cast<int64_t>(hc.inelastic);
    L.secondaries = static_cast<int64_t>(hc.secondaries);
    L.transparent = static_cast<int64_t>(hc.transparent);
    L.inc_retries = static_cast<int64_t>(hc.inc_retries);
    L.dropped = static_cast<int64_t>(hc.dropped);
    L.errors = static_cast<int64_t>(hc.errors);
    if (hc.dropped) return fail(ctx, PMC_E_QUEUE_OVERFLOW, "%llu particles did not fit a queue", (unsigned long long)hc.dropped);
    if (hc.errors)
      return fail(ctx, PMC_E_TIMEOUT, "%llu particles exceeded the step limit or device waits timed out",
                  (unsigned long long)hc.errors);
    return PMC_OK;
  } catch (...) {
    return fail(ctx, PMC_E_INVALID, "exception in transport");
  }
}

// ---------------------------------------------------------------------------
// Learned stand-in of the event generator: data, training, weights, checks.
// ---------------------------------------------------------------------------
namespace {

int surrogate_ready(pmc_ctx* ctx) {
  if (!ctx->have_materials) return fail(ctx, PMC_E_INVALID, "load materials first");
  if (ctx->n_slots < 1 || ctx->n_slots > kSurrTargets)
    return fail(ctx, PMC_E_INVALID, "the network takes 1..%d target nuclides (A >= 2), got %d", kSurrTargets, ctx->n_slots);
  int rc;
  if ((rc = dalloc(ctx, ctx->d_sp, kSurrParams * sizeof(float)))) return rc;
  if ((rc = dalloc(ctx, ctx->d_sg, kSurrParams * sizeof(float)))) return rc;
  if ((rc = dalloc(ctx, ctx->d_sm, kSurrParams * sizeof(float)))) return rc;
  if ((rc = dalloc(ctx, ctx->d_sv, kSurrParams * sizeof(float)))) return rc;
  return PMC_OK;
}

// He-normal weights, zero biases, from a seeded host generator (Box-Muller on a
// 64-bit LCG: initial values only need to be reproducible, not independent of
// anything in the method).
std::vector<float> init_params(uint64_t seed) {
  std::vector<float> p(kSurrParams, 0.0f);
  uint64_t x = seed * 6364136223846793005ull + 1442695040888963407ull;
  auto uni = [&]() {
    x = x * 6364136223846793005ull + 1442695040888963407ull;
    return (static_cast<double>(x >> 11) + 0.5) * (1.0 / 9007199254740992.0);
  };
  for (int l = 0; l < kSurrLayers; ++l) {
    const double sd = std::sqrt(2.0 / kLayerIn[l]) * (l == kSurrLayers - 1 ? 0.1 : 1.0);
    for (size_t i = 0; i < static_cast<size_t>(kLayerIn[l]) * kLayerOut[l]; ++i) {
      const double r = std::sqrt(-2.0 * std::log(uni())), ph = 6.283185307179586 * uni();
      p[w_off(l) + i] = static_cast<float>(sd * r * std::cos(ph));
    }
  }
  return p;
}

}  // namespace

extern "C" {

int pmc_surrogate_dataset(pmc_ctx* ctx, uint64_t n_events, uint64_t seed, float* out) {
  if (!ctx || !out) return PMC_E_INVALID;
  int rc;
  if ((rc = surrogate_ready(ctx))) return rc;
  cudaSetDevice(ctx->opt.device);
  DevBuf b;
  if ((rc = dalloc(ctx, b, n_events * kSurrFeatures * sizeof(float)))) return rc;
  CK(launch_surrogate_dataset(static_cast<const NucleusModel*>(ctx->d_nuclei.p), static_cast<const float*>(ctx->d_btab.p),
                              static_cast<const int*>(ctx->d_slot_nuc.p), ctx->n_slots, seed, n_events,
                              static_cast<float*>(b.p), ctx->stream));
  CK(cudaStreamSynchronize(ctx->stream));
  CK(cudaMemcpy(out, b.p, n_events * kSurrFeatures * sizeof(float), cudaMemcpyDeviceToHost));
  dfree(ctx, b);
  return PMC_OK;
}

int pmc_train_surrogate(pmc_ctx* ctx, const pmc_train_opts* o, pmc_train_result* res) {
  if (!ctx || !o) return PMC_E_INVALID;
  if (o->n_events < 1024 || o->batch < 64 || o->batch > 65536 || o->epochs < 1 || !(o->lr > 0.0))
    return fail(ctx, PMC_E_INVALID, "training options out of range");
  int rc;
  if ((rc = surrogate_ready(ctx))) return rc;
  try {
    cudaSetDevice(ctx->opt.device);
    cudaStream_t s = ctx->stream;
    const uint64_t n = o->n_events;
    const int B = o->batch, rows = 2 * B;
    // 1. events from the project's own cascade + evaporation kernel
    DevBuf feat, perm, X, Y, T, M, act[kSurrLayers + 1], g0, g1, loss;
    if ((rc = dalloc(ctx, feat, n * kSurrFeatures * sizeof(float)))) return rc;
    CK(launch_surrogate_dataset(static_cast<const NucleusModel*>(ctx->d_nuclei.p), static_cast<const float*>(ctx->d_btab.p),
                                static_cast<const int*>(ctx->d_slot_nuc.p), ctx->n_slots, o->seed, n,
                                static_cast<float*>(feat.p), s));
    // 2. buffers and initial weights
    if ((rc = dalloc(ctx, perm, n * sizeof(unsigned)))) return rc;
    if ((rc = dalloc(ctx, X, static_cast<size_t>(rows) * kSurrIn * sizeof(float)))) return rc;
    for (DevBuf* b : {&Y, &T, &M})
      if ((rc = dalloc(ctx, *b, static_cast<size_t>(rows) * kSurrOut * sizeof(float)))) return rc;
    for (int l = 0; l < kSurrLayers; ++l)
      if ((rc = dalloc(ctx, act[l], static_cast<size_t>(rows) * kLayerOut[l] * sizeof(float)))) return rc;
    if ((rc = dalloc(ctx, act[kSurrLayers], static_cast<size_t>(rows) * kSurrOut * sizeof(float)))) return rc;
    if ((rc = dalloc(ctx, g0, static_cast<size_t>(rows) * kSurrHidden * sizeof(float)))) return rc;
    if ((rc = dalloc(ctx, g1, static_cast<size_t>(rows) * kSurrHidden * sizeof(float)))) return rc;
    if ((rc = dalloc(ctx, loss, 64 * sizeof(float)))) return rc;
    std::vector<float> p0 = init_params(o->seed);
    CK(cudaMemcpyAsync(ctx->d_sp.p, p0.data(), kSurrParams * sizeof(float), cudaMemcpyHostToDevice, s));
    CK(cudaMemsetAsync(ctx->d_sm.p, 0, kSurrParams * sizeof(float), s));
    CK(cudaMemsetAsync(ctx->d_sv.p, 0, kSurrParams * sizeof(float), s));
    float* P = static_cast<float*>(ctx->d_sp.p);
    float* Gp = static_cast<float*>(ctx->d_sg.p);
    float* A[kSurrLayers + 1];
    for (int l = 0; l <= kSurrLayers; ++l) A[l] = static_cast<float*>(act[l].p);
    // 3. epochs of shuffled mini-batches, AdamW
    std::vector<unsigned> order(n);
    uint64_t x = o->seed ^ 0x9e3779b97f4a7c15ull;
    const uint64_t steps_per_epoch = n / B;
    int step = 0;
    double first_loss = 0.0, last_loss = 0.0;
    float* dloss = static_cast<float*>(loss.p);
    for (int ep = 0; ep < o->epochs; ++ep) {
      std::iota(order.begin(), order.end(), 0u);
      for (uint64_t i = n - 1; i > 0; --i) {                   // Fisher-Yates with a 64-bit LCG
        x = x * 6364136223846793005ull + 1442695040888963407ull;
        std::swap(order[i], order[(x >> 33) % (i + 1)]);
      }
      CK(cudaMemcpyAsync(perm.p, order.data(), n * sizeof(unsigned), cudaMemcpyHostToDevice, s));
      CK(cudaMemsetAsync(dloss, 0, 64 * sizeof(float), s));
      for (uint64_t k = 0; k < steps_per_epoch; ++k) {
        ++step;
        CK(launch_train_rows(B, static_cast<const float*>(feat.p), static_cast<const unsigned*>(perm.p), k * B, n,
                             o->seed, static_cast<unsigned>(step), static_cast<float*>(X.p), static_cast<float*>(Y.p),
                             static_cast<float*>(T.p), static_cast<float*>(M.p), s));
        if ((rc = mlp_forward(ctx, P, rows, static_cast<float*>(X.p), A, s))) return rc;
        float* lslot = dloss + (k + 1 == steps_per_epoch ? 1 : (k == 0 ? 2 : 0));
        CK(launch_pinball(rows, A[kSurrLayers - 1], static_cast<float*>(Y.p), static_cast<float*>(T.p),
                          static_cast<float*>(M.p), A[kSurrLayers], lslot, s));
        if ((rc = mlp_backward(ctx, P, Gp, rows, static_cast<float*>(X.p), A, static_cast<float*>(g0.p),
                               static_cast<float*>(g1.p), s)))
          return rc;
        CK(launch_adamw(static_cast<int>(kSurrParams), P, Gp, static_cast<float*>(ctx->d_sm.p),
                        static_cast<float*>(ctx->d_sv.p), static_cast<float>(o->lr), 0.9f, 0.999f, 1e-8f,
                        static_cast<float>(o->weight_decay), step, s));
      }
      float h[3];
      CK(cudaMemcpyAsync(h, dloss, 3 * sizeof(float), cudaMemcpyDeviceToHost, s));
      CK(cudaStreamSynchronize(s));
      if (ep == 0) first_loss = h[2];
      last_loss = h[1];
    }
    CK(cudaStreamSynchronize(s));
    CK(cudaGetLastError());
    if ((rc = gemm_errors(ctx))) return rc;
    for (DevBuf* b : {&feat, &perm, &X, &Y, &T, &M, &g0, &g1, &loss}) dfree(ctx, *b);
    for (int l = 0; l <= kSurrLayers; ++l) dfree(ctx, act[l]);
    if ((rc = dalloc(ctx, ctx->d_swb, packed_weight_bytes()))) return rc;
    CK(launch_pack_weights(P, ctx->d_swb.p, s));
    CK(cudaStreamSynchronize(s));
    ctx->surr_trained = true;
    if (ctx->gexec) { cudaGraphExecDestroy(ctx->gexec); ctx->gexec = nullptr; ctx->gkey.clear(); }
    if (res) {
      res->first_loss = first_loss;
      res->last_loss = last_loss;
      res->steps = step;
    }
    return PMC_OK;
  } catch (...) {
    return fail(ctx, PMC_E_INVALID, "exception in training");
  }
}

int pmc_surrogate_params(pmc_ctx* ctx, float* out, size_t n) {
  if (!ctx || !out) return PMC_E_INVALID;
  if (n != kSurrParams) return fail(ctx, PMC_E_INVALID, "the network has %zu parameters", kSurrParams);
  if (!ctx->d_sp.p) return fail(ctx, PMC_E_INVALID, "no network");
  cudaSetDevice(ctx->opt.device);
  CK(cudaMemcpy(out, ctx->d_sp.p, n * sizeof(float), cudaMemcpyDeviceToHost));
  return PMC_OK;
}

int pmc_surrogate_load(pmc_ctx* ctx, const float* params, size_t n) {
  if (!ctx || !params) return PMC_E_INVALID;
  if (n != kSurrParams) return fail(ctx, PMC_E_INVALID, "the network has %zu parameters", kSurrParams);
  int rc;
  if ((rc = surrogate_ready(ctx))) return rc;
  cudaSetDevice(ctx->opt.device);
  CK(cudaMemcpy(ctx->d_sp.p, params, n * sizeof(float), cudaMemcpyHostToDevice));
  if ((rc = dalloc(ctx, ctx->d_swb, packed_weight_bytes()))) return rc;
  CK(launch_pack_weights(static_cast<const float*>(ctx->d_sp.p), ctx->d_swb.p, ctx->stream));
  CK(cudaStreamSynchronize(ctx->stream));
  ctx->surr_trained = true;
  if (ctx->gexec) { cudaGraphExecDestroy(ctx->gexec); ctx->gexec = nullptr; ctx->gkey.clear(); }
  return PMC_OK;
}

int pmc_surrogate_grad(pmc_ctx* ctx, const float* params, const float* x, const float* y, const float* tau,
                       const float* mask, int rows, float* loss, float* grad, float* yhat) {
  if (!ctx || !params || !x || !y || !tau || !mask || rows < 1 || rows > 65536) return PMC_E_INVALID;
  int rc;
  if ((rc = surrogate_ready(ctx))) return rc;
  cudaSetDevice(ctx->opt.device);
  cudaStream_t s = ctx->stream;
  DevBuf X, Y, T, M, act[kSurrLayers + 1], g0, g1, L;
  if ((rc = dalloc(ctx, X, static_cast<size_t>(rows) * kSurrIn * 4))) return rc;
  for (DevBuf* b : {&Y, &T, &M})
    if ((rc = dalloc(ctx, *b, static_cast<size_t>(rows) * kSurrOut * 4))) return rc;
  for (int l = 0; l < kSurrLayers; ++l)
    if ((rc = dalloc(ctx, act[l], static_cast<size_t>(rows) * kLayerOut[l] * 4))) return rc;
  if ((rc = dalloc(ctx, act[kSurrLayers], static_cast<size_t>(rows) * kSurrOut * 4))) return rc;
  if ((rc = dalloc(ctx, g0, static_cast<size_t>(rows) * kSurrHidden * 4))) return rc;
  if ((rc = dalloc(ctx, g1, static_cast<size_t>(rows) * kSurrHidden * 4))) return rc;
  if ((rc = dalloc(ctx, L, 64))) return rc;
  CK(cudaMemcpy(ctx->d_sp.p, params, kSurrParams * 4, cudaMemcpyHostToDevice));
  CK(cudaMemcpy(X.p, x, static_cast<size_t>(rows) * kSurrIn * 4, cudaMemcpyHostToDevice));
  CK(cudaMemcpy(Y.p, y, static_cast<size_t>(rows) * kSurrOut * 4, cudaMemcpyHostToDevice));
  CK(cudaMemcpy(T.p, tau, static_cast<size_t>(rows) * kSurrOut * 4, cudaMemcpyHostToDevice));
  CK(cudaMemcpy(M.p, mask, static_cast<size_t>(rows) * kSurrOut * 4, cudaMemcpyHostToDevice));
  CK(cudaMemset(L.p, 0, 64));
  float* A[kSurrLayers + 1];
  for (int l = 0; l <= kSurrLayers; ++l) A[l] = static_cast<float*>(act[l].p);
  const float* P = static_cast<const float*>(ctx->d_sp.p);
  if ((rc = mlp_forward(ctx, P, rows, static_cast<float*>(X.p), A, s))) return rc;
  CK(launch_pinball(rows, A[kSurrLayers - 1], static_cast<float*>(Y.p), static_cast<float*>(T.p),
                    static_cast<float*>(M.p), A[kSurrLayers], static_cast<float*>(L.p), s));
  if ((rc = mlp_backward(ctx, P, static_cast<float*>(ctx->d_sg.p), rows, static_cast<float*>(X.p), A,
                         static_cast<float*>(g0.p), static_cast<float*>(g1.p), s)))
    return rc;
  CK(cudaStreamSynchronize(s));
  if ((rc = gemm_errors(ctx))) return rc;
  if (loss) CK(cudaMemcpy(loss, L.p, 4, cudaMemcpyDeviceToHost));
  if (grad) CK(cudaMemcpy(grad, ctx->d_sg.p, kSurrParams * 4, cudaMemcpyDeviceToHost));
  if (yhat) CK(cudaMemcpy(yhat, A[kSurrLayers - 1], static_cast<size_t>(rows) * kSurrOut * 4, cudaMemcpyDeviceToHost));
  for (DevBuf* b : {&X, &Y, &T, &M, &g0, &g1, &L}) dfree(ctx, *b);
  for (int l = 0; l <= kSurrLayers; ++l) dfree(ctx, act[l]);
  return PMC_OK;
}

namespace {
int surrogate_rows(pmc_ctx* ctx, const float* x, int rows, float* y, bool check_waits) {
  if (!ctx->surr_trained || !ctx->d_swb.p) return fail(ctx, PMC_E_INVALID, "no network loaded");
  cudaSetDevice(ctx->opt.device);
  cudaStream_t s = ctx->stream;
  DevBuf X, Y, E;
  int rc;
  if ((rc = dalloc(ctx, X, static_cast<size_t>(rows) * kSurrIn * 4))) return rc;
  if ((rc = dalloc(ctx, Y, static_cast<size_t>(rows) * kSurrOut * 4))) return rc;
  if ((rc = dalloc(ctx, E, sizeof(int)))) return rc;
  CK(cudaMemcpyAsync(X.p, x, static_cast<size_t>(rows) * kSurrIn * 4, cudaMemcpyHostToDevice, s));
  CK(cudaMemsetAsync(E.p, 0, sizeof(int), s));
  CK(launch_mlp_rows(rows, static_cast<const float*>(X.p), ctx->d_swb.p, static_cast<const float*>(ctx->d_sp.p),
                     static_cast<float*>(Y.p), static_cast<int*>(E.p), ctx->n_sm, check_waits, s));
  int err = 0;
  CK(cudaMemcpyAsync(y, Y.p, static_cast<size_t>(rows) * kSurrOut * 4, cudaMemcpyDeviceToHost, s));
  CK(cudaMemcpyAsync(&err, E.p, sizeof(int), cudaMemcpyDeviceToHost, s));
  CK(cudaStreamSynchronize(s));
  for (DevBuf* b : {&X, &Y, &E}) dfree(ctx, *b);
  if (err) return fail(ctx, PMC_E_TIMEOUT, "a tensor-core wait timed out");
  return PMC_OK;
}
}  // namespace

int pmc_surrogate_infer(pmc_ctx* ctx, const float* x, int rows, float* y) {
  if (!ctx || !x || !y || rows < 1 || rows > (1 << 20)) return PMC_E_INVALID;
  return surrogate_rows(ctx, x, rows, y, false);
}

int pmc_debug_vavilov_table(float* out, size_t n) {
  const std::vector<float>& t = vavilov_table();
  if (!out || n != t.size()) return PMC_E_INVALID;
  std::memcpy(out, t.data(), n * sizeof(float));
  return PMC_OK;
}

int pmc_debug_drain_waits(pmc_ctx* ctx, uint64_t n_histories, uint64_t seed) {
  if (!ctx) return PMC_E_INVALID;
  ctx->drain_debug = true;
  const int rc = pmc_transport(ctx, n_histories, seed, PMC_FULL_CASCADE, nullptr);
  ctx->drain_debug = false;
  return rc;
}

int pmc_debug_surrogate_waits(pmc_ctx* ctx) {
  if (!ctx) return PMC_E_INVALID;
  std::vector<float> x(128 * kSurrIn, 0.0f), y(128 * kSurrOut);
  return surrogate_rows(ctx, x.data(), 128, y.data(), true);
}

}  // extern "C"

// ---- 3-D gamma index (Sec. II.D; Low et al.) --------------------------------
namespace {

bool gamma_args_ok(double dx, double dy, double dz, double dta_mm, double search_mm) {
  return dx > 0 && dy > 0 && dz > 0 && dta_mm > 0 && std::isfinite(dx) && std::isfinite(dy) && std::isfinite(dz) &&
         std::isfinite(dta_mm) && std::isfinite(search_mm);
}

// Offsets of the search sphere (voxel sizes in cm, radii in mm), sorted by their
// distance term so that a voxel's scan can stop early.
int gamma_offsets(double dx_cm, double dy_cm, double dz_cm, double dta_mm, double search_mm,
                  std::vector<GammaOffset>* out) {
  if (!gamma_args_ok(dx_cm, dy_cm, dz_cm, dta_mm, search_mm)) return PMC_E_INVALID;
  const double dx = dx_cm * 10.0, dy = dy_cm * 10.0, dz = dz_cm * 10.0;
  const double search = search_mm > 0 ? search_mm : 1.5 * dta_mm;
  const double kxm = std::floor(search / dx) + 1, kym = std::floor(search / dy) + 1, kzm = std::floor(search / dz) + 1;
  if (kxm * kym * kzm > 8.0 * PMC_GAMMA_MAX_OFFSETS) return PMC_E_INVALID;
  const int mx = static_cast<int>(kxm), my = static_cast<int>(kym), mz = static_cast<int>(kzm);
  out->clear();
  for (int kz = -mz; kz <= mz; ++kz)
    for (int ky = -my; ky <= my; ++ky)
      for (int kx = -mx; kx <= mx; ++kx) {
        const double ax = kx * dx, ay = ky * dy, az = kz * dz;
        const double r2 = ax * ax + ay * ay + az * az;
        if (r2 > search * search) continue;
        if (out->size() >= static_cast<size_t>(PMC_GAMMA_MAX_OFFSETS)) return PMC_E_INVALID;
        GammaOffset o{};
        o.kx = static_cast<int16_t>(kx);
        o.ky = static_cast<int16_t>(ky);
        o.kz = static_cast<int16_t>(kz);
        o.r_term = r2 / (dta_mm * dta_mm);
        out->push_back(o);
      }
  std::stable_sort(out->begin(), out->end(),
                   [](const GammaOffset& a, const GammaOffset& b) { return a.r_term < b.r_term; });
  return PMC_OK;
}

}  // namespace

extern "C" int pmc_gamma_plan_bytes(double dx, double dy, double dz, double dta_mm, double search_mm, size_t* bytes) {
  if (!bytes) return PMC_E_INVALID;
  std::vector<GammaOffset> off;
  const int rc = gamma_offsets(dx, dy, dz, dta_mm, search_mm, &off);
  if (rc != PMC_OK) return rc;
  *bytes = kGammaHeadBytes + off.size() * sizeof(GammaOffset);
  return PMC_OK;
}

extern "C" int pmc_gamma_plan(double dx, double dy, double dz, double dta_mm, double search_mm, void* plan,
                              size_t plan_bytes, void* stream) {
  if (!plan || (reinterpret_cast<uintptr_t>(plan) & 255u) != 0) return PMC_E_INVALID;
  std::vector<GammaOffset> off;
  const int rc = gamma_offsets(dx, dy, dz, dta_mm, search_mm, &off);
  if (rc != PMC_OK) return rc;
  const size_t bytes = kGammaHeadBytes + off.size() * sizeof(GammaOffset);
  if (plan_bytes < bytes) return PMC_E_INVALID;
  std::vector<unsigned char> host(bytes, 0);
  GammaHead head{};
  head.n_off = static_cast<int>(off.size());
  head.dx = dx * 10.0;
  head.dy = dy * 10.0;
  head.dz = dz * 10.0;
  head.dta = dta_mm;
  head.search = search_mm > 0 ? search_mm : 1.5 * dta_mm;
  std::memcpy(host.data(), &head, sizeof(head));
  std::memcpy(host.data() + kGammaHeadBytes, off.data(), off.size() * sizeof(GammaOffset));
  // pageable source: the copy is staged before the call returns, so `host` may go
  if (cudaMemcpyAsync(plan, host.data(), bytes, cudaMemcpyHostToDevice, static_cast<cudaStream_t>(stream)) != cudaSuccess)
    return PMC_E_CUDA;
  return PMC_OK;
}

extern "C" int pmc_gamma_device(void* plan, const double* ref, const double* eval, int nx, int ny, int nz,
                                double dose_pct, double threshold, float* gamma, void* stream) {
  if (!plan || !ref || !eval || nx < 1 || ny < 1 || nz < 1 || !(dose_pct > 0) || !(threshold >= 0) ||
      !std::isfinite(dose_pct) || !std::isfinite(threshold) || (reinterpret_cast<uintptr_t>(plan) & 255u) != 0 ||
      static_cast<double>(nx) * ny * nz > 9.0e18)
    return PMC_E_INVALID;
  if (launch_gamma(ref, eval, nx, ny, nz, plan, dose_pct, threshold, gamma, static_cast<cudaStream_t>(stream)) !=
      cudaSuccess)
    return PMC_E_CUDA;
  return PMC_OK;
}

extern "C" int pmc_gamma_index(const double* ref, const double* eval, int nx, int ny, int nz, double dx, double dy,
                               double dz, double dose_pct, double dta_mm, double threshold, double search_mm,
                               float* gamma, double* pass_rate) {
  if (!ref || !eval || nx < 1 || ny < 1 || nz < 1) return PMC_E_INVALID;
  size_t pb = 0;
  int rc = pmc_gamma_plan_bytes(dx, dy, dz, dta_mm, search_mm, &pb);
  if (rc != PMC_OK) return rc;
  const size_t n = static_cast<size_t>(nx) * ny * nz;
  void *dr = nullptr, *de = nullptr, *dg = nullptr, *dp = nullptr;
  if (cudaMalloc(&dr, n * 8) != cudaSuccess || cudaMalloc(&de, n * 8) != cudaSuccess ||
      (gamma && cudaMalloc(&dg, n * 4) != cudaSuccess) || cudaMalloc(&dp, pb) != cudaSuccess) {
    rc = PMC_E_OOM;
  } else if (cudaMemcpy(dr, ref, n * 8, cudaMemcpyHostToDevice) != cudaSuccess ||
             cudaMemcpy(de, eval, n * 8, cudaMemcpyHostToDevice) != cudaSuccess) {
    rc = PMC_E_CUDA;
  } else {
    rc = pmc_gamma_plan(dx, dy, dz, dta_mm, search_mm, dp, pb, nullptr);
    if (rc == PMC_OK)
      rc = pmc_gamma_device(dp, static_cast<const double*>(dr), static_cast<const double*>(de), nx, ny, nz, dose_pct,
                            threshold, static_cast<float*>(dg), nullptr);
    unsigned long long c[2] = {0, 0};
    if (rc == PMC_OK && (cudaStreamSynchronize(nullptr) != cudaSuccess ||
                         cudaMemcpy(c, dp, sizeof(c), cudaMemcpyDeviceToHost) != cudaSuccess ||
                         (gamma && cudaMemcpy(gamma, dg, n * 4, cudaMemcpyDeviceToHost) != cudaSuccess)))
      rc = PMC_E_CUDA;
    if (rc == PMC_OK && pass_rate) *pass_rate = c[0] ? static_cast<double>(c[1]) / static_cast<double>(c[0]) : NAN;
  }
  cudaFree(dr);
  cudaFree(de);
  cudaFree(dg);
  cudaFree(dp);
  return rc;
}

// ---- multi-plan stream: concurrent plans admitted by device memory ----------
// A pool of concurrency slots, each an engine context with its own streams,
// serves a list of plans in order.  A plan is admitted when its device
// footprint fits in what the budget leaves; its slot then uploads the phantom,
// transports, copies the dose out and releases the plan's buffers.  The slots'
// persistent kernels share the SMs, so the latency-bound drain of one plan
// overlaps the full-width launches of another.  All allocation is stream-ordered from
// one memory pool: a plan starting or ending never synchronises the device.
struct pmc_plan_stream {
  pmc_options opt{};
  uint64_t budget = 0;
  cudaMemPool_t pool = nullptr;
  std::vector<pmc_ctx*> slots;
  bool have_materials = false, have_surrogate = false;
  std::string err;
};

namespace {

int sfail(pmc_plan_stream* S, int code, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  std::vsnprintf(buf, sizeof(buf), fmt, ap);
  va_end(ap);
  S->err = buf;
  return code;
}

// Pool allocations are rounded to the pool's 2 MiB granularity.
uint64_t pool_round(uint64_t b) { return b == 0 ? 0 : (b + (2ull << 20) - 1) / (2ull << 20) * (2ull << 20); }

uint64_t plan_footprint(const pmc_options& opt, const pmc_plan& pl, int mode) {
  const uint64_t nv = static_cast<uint64_t>(pl.nx) * pl.ny * pl.nz;
  const uint64_t B = static_cast<uint64_t>(opt.n_batches);
  const int64_t chunk = opt.chunk > 0 ? opt.chunk : (1ll << 22);
  const uint64_t qcap = std::max<uint64_t>(std::min<uint64_t>(pl.n_histories, static_cast<uint64_t>(chunk)), 1024);
  const uint64_t n_chunks = (pl.n_histories + qcap - 1) / qcap;
  uint64_t b = 0;
  b += pl.hu ? pool_round(nv * 2) : pool_round(nv) + pool_round(nv * 4);
  b += pool_round(nv * B * 8) + 2 * pool_round(nv * 8);
  b += kQueues * pool_round(qcap * sizeof(Particle));
  b += pool_round(n_chunks * kSlots * sizeof(unsigned));
  b += pool_round(drain_buffer_bytes(qcap));
  b += pool_round(sizeof(Counters)) + pool_round(8) + pool_round(static_cast<uint64_t>(pl.n_spots) * sizeof(SpotDev));
  b += 2 * pool_round(qcap * sizeof(EvapRecord));
  return b;
}

// Frees what a plan allocated (phantom, tallies, queues); keeps the tables.
void release_plan(pmc_ctx* ctx) {
  DevBuf* bufs[] = {&ctx->d_mat, &ctx->d_rho, &ctx->d_hu, &ctx->d_tally, &ctx->d_dose, &ctx->d_sigma,
                    &ctx->d_counters, &ctx->d_counts, &ctx->d_seed, &ctx->d_spots, &ctx->d_q[0], &ctx->d_q[1],
                    &ctx->d_q[2], &ctx->d_q[3], &ctx->d_q[4], &ctx->d_q[5], &ctx->d_rec[0], &ctx->d_rec[1],
                    &ctx->d_drain};
  for (DevBuf* b : bufs) dfree(ctx, *b);
  ctx->drain_qcap = 0;
  if (ctx->gexec) { cudaGraphExecDestroy(ctx->gexec); ctx->gexec = nullptr; ctx->gkey.clear(); }
  ctx->have_phantom = false;
  ctx->have_run = false;
  ctx->n_vox = 0;
  ctx->geo = Geometry{};
}

int run_plan(pmc_ctx* ctx, const pmc_plan& pl, int mode, pmc_plan_result* r) {
  int rc = pmc_load_phantom(ctx, pl.nx, pl.ny, pl.nz, pl.dx, pl.dy, pl.dz, pl.x0, pl.y0, pl.z0, pl.hu, pl.mat, pl.rho);
  if (rc == PMC_OK) rc = pmc_clear_spots(ctx);
  if (rc == PMC_OK) rc = pmc_add_spots(ctx, pl.spots, pl.n_spots);
  if (rc == PMC_OK) rc = pmc_transport(ctx, pl.n_histories, pl.seed, mode, nullptr);
  if (rc == PMC_OK && (pl.dose_gy || pl.sigma_gy))
    rc = pmc_read_dose(ctx, pl.dose_gy, pl.sigma_gy, static_cast<size_t>(pl.nx) * pl.ny * pl.nz);
  if (rc == PMC_OK) rc = pmc_read_ledger(ctx, &r->ledger);
  release_plan(ctx);
  if (cudaStreamSynchronize(ctx->stream) != cudaSuccess && rc == PMC_OK) rc = PMC_E_CUDA;   // frees done
  return rc;
}

}  // namespace

extern "C" int pmc_plans_create(pmc_plan_stream** out, const pmc_options* opt, int n_slots, uint64_t budget) {
  if (!out || n_slots < 1 || n_slots > 64 || budget == 0) return PMC_E_INVALID;
  *out = nullptr;
  pmc_plan_stream* S = new (std::nothrow) pmc_plan_stream();
  if (!S) return PMC_E_OOM;
  if (opt) S->opt = *opt;
  if (S->opt.n_batches == 0) S->opt.n_batches = 10;
  if (S->opt.block_size <= 0) S->opt.block_size = 256;   // fixed launch shape: no per-slot autotuning
  S->opt.alloc = nullptr;
  S->opt.free = nullptr;
  S->budget = budget;
  cudaMemPoolProps props{};
  props.allocType = cudaMemAllocationTypePinned;
  props.location.type = cudaMemLocationTypeDevice;
  props.location.id = S->opt.device;
  if (cudaSetDevice(S->opt.device) != cudaSuccess || cudaMemPoolCreate(&S->pool, &props) != cudaSuccess) {
    cudaGetLastError();
    delete S;
    return PMC_E_CUDA;
  }
  uint64_t keep = ~0ull;   // keep freed memory in the pool between plans
  cudaMemPoolSetAttribute(S->pool, cudaMemPoolAttrReleaseThreshold, &keep);
  for (int i = 0; i < n_slots; ++i) {
    pmc_ctx* c = nullptr;
    const int rc = pmc_create(&c, &S->opt);
    if (rc != PMC_OK) {
      pmc_plans_destroy(S);
      return rc;
    }
    c->pool = S->pool;
    S->slots.push_back(c);
  }
  *out = S;
  return PMC_OK;
}

extern "C" void pmc_plans_destroy(pmc_plan_stream* S) {
  if (!S) return;
  for (pmc_ctx* c : S->slots) pmc_destroy(c);
  if (S->pool) {
    cudaSetDevice(S->opt.device);
    cudaMemPoolDestroy(S->pool);
  }
  delete S;
}

extern "C" const char* pmc_plans_last_error(const pmc_plan_stream* S) { return S ? S->err.c_str() : "null stream"; }

extern "C" int pmc_plans_load_materials(pmc_plan_stream* S, const pmc_nuclide* nuc, int n_nuc,
                                        const pmc_material* mat, int n_mat, const pmc_hu_bin* hu, int n_hu) {
  if (!S) return PMC_E_INVALID;
  for (pmc_ctx* c : S->slots) {
    const int rc = pmc_load_materials(c, nuc, n_nuc, mat, n_mat, hu, n_hu);
    if (rc != PMC_OK) return sfail(S, rc, "load materials: %s", c->err.c_str());
  }
  S->have_materials = true;
  S->have_surrogate = false;
  return PMC_OK;
}

extern "C" int pmc_plans_load_surrogate(pmc_plan_stream* S, const float* params, size_t n) {
  if (!S || !params) return PMC_E_INVALID;
  if (!S->have_materials) return sfail(S, PMC_E_INVALID, "load materials first");
  for (pmc_ctx* c : S->slots) {
    const int rc = pmc_surrogate_load(c, params, n);
    if (rc != PMC_OK) return sfail(S, rc, "load surrogate: %s", c->err.c_str());
  }
  S->have_surrogate = true;
  return PMC_OK;
}

extern "C" int pmc_plans_bytes(const pmc_plan_stream* S, const pmc_plan* plan, int mode, uint64_t* bytes) {
  if (!S || !plan || !bytes || plan->nx < 1 || plan->ny < 1 || plan->nz < 1) return PMC_E_INVALID;
  *bytes = plan_footprint(S->opt, *plan, mode);
  return PMC_OK;
}

extern "C" int pmc_plans_run(pmc_plan_stream* S, const pmc_plan* plans, int n, int mode, pmc_plan_result* res) {
  if (!S || n < 0 || (n > 0 && (!plans || !res))) return PMC_E_INVALID;
  if (!S->have_materials) return sfail(S, PMC_E_INVALID, "load materials first");
  if (mode != PMC_FULL_CASCADE && mode != PMC_SURROGATE) return sfail(S, PMC_E_INVALID, "unknown mode %d", mode);
  if (mode == PMC_SURROGATE && !S->have_surrogate) return sfail(S, PMC_E_INVALID, "load the surrogate first");
  std::vector<uint64_t> fp(n);
  for (int i = 0; i < n; ++i) {
    res[i] = pmc_plan_result{};
    res[i].status = PMC_E_INVALID;
    res[i].slot = -1;
    if (plans[i].nx < 1 || plans[i].ny < 1 || plans[i].nz < 1) return sfail(S, PMC_E_INVALID, "plan %d: bad grid", i);
    fp[i] = plan_footprint(S->opt, plans[i], mode);
    res[i].device_bytes = fp[i];
  }
  std::mutex m;
  std::condition_variable cv;
  int next = 0;
  uint64_t admitted = 0;
  const auto t0 = std::chrono::steady_clock::now();
  auto ms_since = [&]() {
    return std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
  };
  auto slot_main = [&](int slot) {
    pmc_ctx* ctx = S->slots[slot];
    cudaSetDevice(S->opt.device);
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    for (;;) {
      int i = -1;
      {
        std::unique_lock<std::mutex> lk(m);
        for (;;) {
          if (next >= n) break;
          if (fp[next] > S->budget) {   // can never be admitted
            res[next].status = PMC_E_OOM;
            ++next;
            continue;
          }
          if (admitted + fp[next] <= S->budget) {
            i = next++;
            admitted += fp[i];
            res[i].t_admit_ms = ms_since();
            res[i].slot = slot;
            break;
          }
          cv.wait(lk);
        }
      }
      if (i < 0) break;
      cudaEventRecord(e0, ctx->stream);
      int rc = run_plan(ctx, plans[i], mode, &res[i]);
      cudaEventRecord(e1, ctx->stream);
      float gms = 0.0f;
      if (cudaEventSynchronize(e1) == cudaSuccess && cudaEventElapsedTime(&gms, e0, e1) == cudaSuccess)
        res[i].gpu_ms = gms;
      {
        std::lock_guard<std::mutex> lk(m);
        admitted -= fp[i];
        res[i].status = rc;
        res[i].t_end_ms = ms_since();
      }
      cv.notify_all();
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
  };
  std::vector<std::thread> threads;
  for (size_t k = 0; k < S->slots.size(); ++k) threads.emplace_back(slot_main, static_cast<int>(k));
  for (auto& t : threads) t.join();
  int first_bad = PMC_OK;
  for (int i = 0; i < n; ++i)
    if (res[i].status != PMC_OK) { first_bad = res[i].status; break; }
  return first_bad;
}
