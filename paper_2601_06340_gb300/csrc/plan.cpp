// Host-side plan math in FP64 (compiled with -ffp-contract=off so that the
// operation order written here is the one executed).
//
// Per photon energy (Krzywinski & Halavanau, arXiv 2601.06340, Sec. 2):
//   lambda = hc / E, k = 2 pi / lambda, s = sin(theta_B(E)) = lambda / 2d
//   (the band centres +-k_d/2 in units of k, Eq. fov7), cos(alpha) =
//   sqrt(1 - s^2) (Eq. fov4), dz^ = k dz, dx^ = k dx (Eq. fov2), and the
//   Jacobi-Anger coefficients of Eqs. fov11-fov12 read with dz^:
//   a = J0(w) e^{i phi0}, b = i J1(w) e^{i phi0}, w = dz^ chi_h / cos(alpha),
//   phi0 = dz^ chi_0 / (2 cos(alpha)).
// Per band, the propagator exp(i dz^ sqrt(1 - (q +- s)^2)) of Eq. fov10 is
// split into the common phase g = exp(i dz^ cos(alpha)) and the mode part
// exp(i dz^ delta_+-(q)), delta_+-(q) = -q (q +- 2 s) /
// (sqrt(1 - (q +- s)^2) + cos(alpha)), which is the same quantity without
// the cancellation of sqrt(...) - cos(alpha).
#include <cmath>
#include <complex>
#include <string>
#include <vector>

#include "bpm_internal.h"

namespace bpm {

namespace {

using cd = std::complex<double>;

bool finite(double v) { return std::isfinite(v); }

// J_nu(w) by its power series sum_m (-1)^m (w/2)^(2m+nu) / (m! (m+nu)!).
// skip_first drops the m = 0 term (J0(w) - 1 without cancellation).
cd bessel(int nu, cd w, bool skip_first) {
  cd half = w / 2.0;
  cd term = (nu == 0) ? cd(1.0, 0.0) : half;
  double scale = std::max(std::abs(term), 1e-300);
  cd total = skip_first ? cd(0.0, 0.0) : term;
  for (int m = 1; m <= 200; ++m) {
    term = term * (-(half * half)) / double(m * (m + nu));
    total += term;
    if (std::abs(term) < 1e-18 * scale) break;
  }
  return total;
}

// exp(i z) - 1 for complex z without cancellation.
cd expm1_i(cd z) {
  double x = z.real(), y = z.imag();          // i z = -y + i x
  double ey = std::exp(-y), em = std::expm1(-y);
  double sh = std::sin(0.5 * x);
  double cosm1 = -2.0 * sh * sh;               // cos x - 1
  return cd(em * std::cos(x) + cosm1, ey * std::sin(x));
}

double fftfreq_q(int k, int n, double dxh) {
  int kk = (k < n / 2) ? k : k - n;
  return kTwoPi * (double(kk) * (1.0 / (double(n) * dxh)));
}

// delta_+-(q) in the cancellation-free form (sign = +1 for psi_+).
double delta_q(double q, double s, double c, int sign) {
  double t = q + sign * s;
  double root = std::sqrt(1.0 - t * t);
  return -q * (q + sign * 2.0 * s) / (root + c);
}

}  // namespace

static void unit_root(int m, int n, double* cr, double* ci);

int validate_problem(const bpm_problem* p, std::string* why) {
  auto bad = [&](const std::string& m) { *why = m; return BPM_ERR_INVALID; };
  if (!p) return bad("problem is NULL");
  if (p->nx < 8 || p->nx > (1 << kMaxLogN) || (p->nx & (p->nx - 1)))
    return bad("nx must be a power of two in [8, " +
               std::to_string(1 << kMaxLogN) + "]");
  if (p->nz < 1) return bad("nz must be >= 1");
  if (!(p->dx_um > 0) || !finite(p->dx_um)) return bad("dx_um must be > 0");
  if (!(p->dz_um > 0) || !finite(p->dz_um)) return bad("dz_um must be > 0");
  if (!finite(p->x0_um)) return bad("x0_um must be finite");
  if (p->n_energy < 1 || !p->energy_ev) return bad("need n_energy >= 1 energies");
  if (p->n_energy > (1 << 20)) return bad("n_energy too large");
  if (!(p->e_ref_ev > 0) || !finite(p->e_ref_ev)) return bad("e_ref_ev must be > 0");
  if (!(p->theta_b_ref_rad > 0) || !(p->theta_b_ref_rad < 1.5707963267948966))
    return bad("theta_b_ref_rad must be in (0, pi/2)");
  if (!finite(p->chi0_re) || !finite(p->chi0_im) || !finite(p->chih_re) ||
      !finite(p->chih_im))
    return bad("chi values must be finite");
  if (p->record_every < 0) return bad("record_every must be >= 0");
  if (p->precision != BPM_FP64_PLAIN && p->precision != BPM_FP32_FUSED)
    return bad("precision must be BPM_FP64_PLAIN or BPM_FP32_FUSED");
  for (int j = 0; j < p->n_energy; ++j) {
    double e = p->energy_ev[j];
    if (!(e > 0) || !finite(e)) return bad("energies must be > 0");
    double s = std::sin(p->theta_b_ref_rad) * (p->e_ref_ev / e);
    if (!(s < 1.0)) return bad("no Bragg angle at energy " + std::to_string(e));
    double lam = kHcEvAngstrom / e * 1e-4;
    double k = kTwoPi / lam;
    double qmax = M_PI / (k * p->dx_um);
    if (!((qmax + s) * (qmax + s) < 1.0))
      return bad("evanescent modes: 1 - (q_max + s)^2 <= 0, refine the grid");
    // Eqs. fov11-fov12 expand the step's coupling in powers of
    // w = dz^ chi_h / cos(alpha); the series is summed in FP64, which stays
    // accurate for |w| <= 1 (steps far shorter than the extinction length)
    const double c = std::sqrt((1.0 - s) * (1.0 + s));
    const double w = k * p->dz_um * std::hypot(p->chih_re, p->chih_im) / c;
    const double phi_im = k * p->dz_um * std::fabs(p->chi0_im) / (2.0 * c);
    if (!(w <= 1.0))
      return bad("dz too long for the coupling expansion: |dz^ chi_h / cos(alpha)| = " +
                 std::to_string(w) + " > 1");
    if (!(phi_im <= 700.0)) return bad("dz too long: the per-step absorption underflows");
  }
  return BPM_OK;
}

int validate_problem3d(const bpm_problem* p, int ny, double dy_um, double y0_um,
                       std::string* why) {
  auto bad = [&](const std::string& m) { *why = m; return BPM_ERR_INVALID; };
  int rc = validate_problem(p, why);
  if (rc != BPM_OK) return rc;
  if (p->precision != BPM_FP32_FUSED) return bad("3D plans run in BPM_FP32_FUSED");
  if (p->nx < 256 || p->nx > 4096) return bad("3D plans need nx in [256, 4096]");
  if (ny < 256 || ny > 1024 || (ny & (ny - 1)))
    return bad("ny must be a power of two in [256, 1024]");
  if (!(dy_um > 0) || !finite(dy_um)) return bad("dy_um must be > 0");
  if (!finite(y0_um)) return bad("y0_um must be finite");
  for (int j = 0; j < p->n_energy; ++j) {
    double e = p->energy_ev[j];
    double s = std::sin(p->theta_b_ref_rad) * (p->e_ref_ev / e);
    double k = kTwoPi / (kHcEvAngstrom / e * 1e-4);
    double qx = M_PI / (k * p->dx_um), qy = M_PI / (k * dy_um);
    if (!((qx + s) * (qx + s) + qy * qy < 1.0))
      return bad("evanescent modes: 1 - (qx_max + s)^2 - qy_max^2 <= 0, refine the grid");
  }
  return BPM_OK;
}

void compute_energy_consts(bpm_plan_s* plan) {
  plan->ec.clear();
  for (double e : plan->energies) {
    EnergyConsts c{};
    c.e_ev = e;
    double lam_a = kHcEvAngstrom / e;
    double lam_um = lam_a * 1e-4;
    c.k_um = kTwoPi / lam_um;
    c.s = std::sin(plan->theta_b_ref) * (plan->e_ref_ev / e);
    c.c = std::sqrt((1.0 - c.s) * (1.0 + c.s));
    c.dzh = c.k_um * plan->dz_um;
    c.dxh = c.k_um * plan->dx_um;
    c.w = c.dzh * plan->chih / c.c;
    c.phi0 = c.dzh * plan->chi0 / (2.0 * c.c);
    cd ephi = std::exp(cd(0.0, 1.0) * c.phi0);
    cd j0m1 = bessel(0, c.w, true);
    cd j1 = bessel(1, c.w, false);
    c.a = (1.0 + j0m1) * ephi;
    c.b = cd(0.0, 1.0) * j1 * ephi;
    c.am1 = j0m1 * ephi + expm1_i(c.phi0);
    c.gphase = std::fmod(c.dzh * c.c, kTwoPi);
    plan->ec.push_back(c);
  }
}

// Radices of the fused kernel's passes: radix 16 while at least 16 remain,
// then one pass with the remaining power of two.
static std::vector<int> fused_radices(int logn) {
  std::vector<int> r;
  int left = logn;
  while (left > 4) { r.push_back(16); left -= 4; }
  r.push_back(1 << left);
  return r;
}

std::vector<int> fft_output_order(int logn) {
  int n = 1 << logn;
  std::vector<int> rad = fused_radices(logn);
  std::vector<int> out(n);
  for (int pos = 0; pos < n; ++pos) {
    int rem = pos, len = n, freq = 0, mult = 1;
    for (int r : rad) {
      int stride = len / r;
      int d = rem / stride;
      rem %= stride;
      freq += d * mult;
      mult *= r;
      len = stride;
    }
    out[pos] = freq;
  }
  return out;
}

// Split bands (N = M P), per band and local position pos of the local
// M-point transform's digit-reversed output, with spectral index k and
// D = (P(q) - 1)/N:
//   P = 2: [band][D(k) | D(k + M)][pos] -- the kernel forms
//          X_r = F_0 + (-1)^r W_N^k F_1 and D(k + M r) X_r itself, so each
//          table value is rounded relative to itself;
//   P = 4: [band][h][delta][pos] of E_delta[k] W_N^{s k}, s = h' - h for the
//          sender h' = (h + delta) mod 4, E_delta[k] = sum_r W_4^{delta r}
//          D[k + M r], as double-float pairs (hi, lo): float4 (hi.re,
//          hi.im, lo.re, lo.im).  Part h forms sum_delta of these times the
//          senders' local spectra F_h'.  E mixes D values of very different
//          size, so a single float would round the small ones far beyond
//          their own size, and that error repeats every step; hi + lo keeps
//          it at FP64 level.
void split_prop_table(const bpm_plan_s* plan, int row, int logm, std::vector<float2>* out) {
  split_prop_table_frac(plan, row, logm, 1.0, out);
}

void split_prop_table_frac(const bpm_plan_s* plan, int row, int logm, double frac,
                           std::vector<float2>* out) {
  const EnergyConsts& c = plan->ec[row];
  const int n = plan->nx, m = 1 << logm, parts = n / m;
  std::vector<int> local = fft_output_order(logm);
  out->assign(size_t(split_table_stride(plan, logm)), float2{0.f, 0.f});
  std::vector<cd> dk(parts), w(parts);
  for (int r = 0; r < parts; ++r) {
    double cr, ci;
    unit_root(r, parts, &cr, &ci);
    w[r] = cd(cr, ci);
  }
  for (int band = 0; band < 2; ++band) {
    int sign = band == 0 ? +1 : -1;
    for (int pos = 0; pos < m; ++pos) {
      for (int r = 0; r < parts; ++r) {
        double q = fftfreq_q(local[pos] + m * r, n, c.dxh);
        dk[r] = expm1_i(cd(frac * c.dzh * delta_q(q, c.s, c.c, sign), 0.0)) * (1.0 / double(n));
      }
      if (parts == 2) {
        for (int r = 0; r < 2; ++r)
          (*out)[(size_t(band) * 2 + r) * m + pos] =
              float2{float(dk[r].real()), float(dk[r].imag())};
        continue;
      }
      for (int dl = 0; dl < parts; ++dl) {
        cd e(0.0, 0.0);
        for (int r = 0; r < parts; ++r) e += w[(dl * r) % parts] * dk[r];
        for (int h = 0; h < parts; ++h) {
          const int sh = h + dl < parts ? dl : dl - parts;     // h' - h
          double wr, wi;
          unit_root(((sh * local[pos]) % n + n) % n, n, &wr, &wi);   // W_N^{sh k}
          const cd f = e * cd(wr, wi);
          const float fr = float(f.real()), fi = float(f.imag());
          const size_t at = 2 * (((size_t(band) * parts + h) * parts + dl) * m + pos);
          (*out)[at] = float2{fr, fi};
          (*out)[at + 1] = float2{float(f.real() - double(fr)), float(f.imag() - double(fi))};
        }
      }
    }
  }
}

int split_table_stride(const bpm_plan_s* plan, int logm) {
  const int parts = plan->nx >> logm;
  return parts == 2 ? 2 * parts * (1 << logm) : 2 * parts * parts * (1 << logm) * 2;
}

void fused_prop_table(const bpm_plan_s* plan, int row, std::vector<float2>* out) {
  const EnergyConsts& c = plan->ec[row];
  int n = plan->nx;
  if (plan->logn >= kSplitLogN) {   // N = 4096 P, P = 2 or 4
    split_prop_table(plan, row, 12, out);
    return;
  }
  std::vector<int> order = fft_output_order(plan->logn);
  out->assign(2 * size_t(n), float2{0.f, 0.f});
  double inv_n = 1.0 / double(n);
  for (int band = 0; band < 2; ++band) {
    int sign = band == 0 ? +1 : -1;
    for (int pos = 0; pos < n; ++pos) {
      double q = fftfreq_q(order[pos], n, c.dxh);
      double ph = c.dzh * delta_q(q, c.s, c.c, sign);
      cd d = expm1_i(cd(ph, 0.0)) * inv_n;
      (*out)[size_t(band) * n + pos] = float2{float(d.real()), float(d.imag())};
    }
  }
}

void fused_prop_table_frac(const bpm_plan_s* plan, int row, double frac,
                           std::vector<float2>* out) {
  const EnergyConsts& c = plan->ec[row];
  const int n = plan->nx;
  std::vector<int> order = fft_output_order(plan->logn);
  out->assign(2 * size_t(n), float2{0.f, 0.f});
  const double inv_n = 1.0 / double(n);
  for (int band = 0; band < 2; ++band) {
    const int sign = band == 0 ? +1 : -1;
    for (int pos = 0; pos < n; ++pos) {
      const double q = fftfreq_q(order[pos], n, c.dxh);
      const double ph = frac * c.dzh * delta_q(q, c.s, c.c, sign);
      const cd d = expm1_i(cd(ph, 0.0)) * inv_n;
      (*out)[size_t(band) * n + pos] = float2{float(d.real()), float(d.imag())};
    }
  }
}

void vol_prop_table(const bpm_plan_s* plan, int row, std::vector<float2>* out) {
  // delta_+-(qx, qy) = sqrt(1 - (qx +- s)^2 - qy^2) - cos(alpha)
  //                  = -(qx (qx +- 2 s) + qy^2) / (sqrt(...) + cos(alpha))
  const EnergyConsts& c = plan->ec[row];
  const int nx = plan->nx, ny = plan->ny;
  const double dyh = c.k_um * plan->dy_um;
  std::vector<int> ox = fft_output_order(plan->logn), oy = fft_output_order(plan->logny);
  const double inv = 1.0 / (double(nx) * double(ny));
  out->assign(2 * size_t(nx) * ny, float2{0.f, 0.f});
  for (int band = 0; band < 2; ++band) {
    const double sign = band == 0 ? 1.0 : -1.0;
    for (int py = 0; py < ny; ++py) {
      const double qy = fftfreq_q(oy[py], ny, dyh);
      for (int px = 0; px < nx; ++px) {
        const double qx = fftfreq_q(ox[px], nx, c.dxh);
        const double t = qx + sign * c.s;
        const double root = std::sqrt(1.0 - t * t - qy * qy);
        const double delta = -(qx * (qx + sign * 2.0 * c.s) + qy * qy) / (root + c.c);
        const cd d = expm1_i(cd(c.dzh * delta, 0.0)) * inv;
        (*out)[(size_t(band) * ny + py) * nx + px] = float2{float(d.real()), float(d.imag())};
      }
    }
  }
}

std::vector<std::pair<double, double>> split_stages(int method) {
  if (method == BPM_SPLIT_VERLET) return {{0.0, 0.5}, {1.0, 0.5}};
  if (method == BPM_SPLIT_FOREST_RUTH) {
    const double t = 1.0 / (2.0 - std::cbrt(2.0));
    return {{0.0, t / 2.0}, {t, (1.0 - t) / 2.0}, {1.0 - 2.0 * t, (1.0 - t) / 2.0}, {t, t / 2.0}};
  }
  return {{1.0, 1.0}};
}

void coupling_frac(const bpm_plan_s* plan, int row, double frac, cd* a, cd* b) {
  const EnergyConsts& c = plan->ec[row];
  const cd w = frac * c.w, phi0 = frac * c.phi0;
  const cd ephi = std::exp(cd(0.0, 1.0) * phi0);
  *a = (1.0 + bessel(0, w, true)) * ephi;
  *b = cd(0.0, 1.0) * bessel(1, w, false) * ephi;
}

void plain_prop_table_frac(const bpm_plan_s* plan, int row, double frac,
                           std::vector<double2>* out) {
  const EnergyConsts& c = plan->ec[row];
  int n = plan->nx;
  out->assign(2 * size_t(n), double2{0.0, 0.0});
  double inv_n = 1.0 / double(n);
  for (int band = 0; band < 2; ++band) {
    int sign = band == 0 ? +1 : -1;
    for (int m = 0; m < n; ++m) {
      double q = fftfreq_q(m, n, c.dxh);
      double ph = frac * c.dzh * delta_q(q, c.s, c.c, sign);
      (*out)[size_t(band) * n + m] = double2{std::cos(ph) * inv_n, std::sin(ph) * inv_n};
    }
  }
}

void plain_prop_table(const bpm_plan_s* plan, int row, std::vector<double2>* out) {
  const EnergyConsts& c = plan->ec[row];
  int n = plan->nx;
  out->assign(2 * size_t(n), double2{0.0, 0.0});
  double inv_n = 1.0 / double(n);
  for (int band = 0; band < 2; ++band) {
    int sign = band == 0 ? +1 : -1;
    for (int m = 0; m < n; ++m) {
      double q = fftfreq_q(m, n, c.dxh);
      double ph = c.dzh * delta_q(q, c.s, c.c, sign);
      (*out)[size_t(band) * n + m] = double2{std::cos(ph) * inv_n, std::sin(ph) * inv_n};
    }
  }
}

static void unit_root(int m, int n, double* cr, double* ci) {
  // exp(-2 pi i m / n) with exact zeros on the axes.
  double ang = kTwoPi * (double(m) / double(n));
  double c = std::cos(ang), s = -std::sin(ang);
  if ((4 * m) % n == 0) {
    int q = (4 * m) / n;
    const double cs[4][2] = {{1, 0}, {0, -1}, {-1, 0}, {0, 1}};
    c = cs[q & 3][0];
    s = cs[q & 3][1];
  }
  *cr = c;
  *ci = s;
}

void twiddle_table_f32(int n, std::vector<float4>* out) {
  out->resize(n);
  for (int m = 0; m < n; ++m) {
    double c, s;
    unit_root(m, n, &c, &s);
    float ch = float(c), sh = float(s);
    float cl = float(c - double(ch)), sl = float(s - double(sh));
    (*out)[m] = float4{ch, sh, cl, sl};
  }
}

void twiddle_table_f64(int n, std::vector<double2>* out) {
  out->resize(n);
  for (int m = 0; m < n; ++m) {
    double c, s;
    unit_root(m, n, &c, &s);
    (*out)[m] = double2{c, s};
  }
}

}  // namespace bpm
