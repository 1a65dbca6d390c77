// Two-term Boltzmann transport of a uniform-field electron swarm (host, FP64):
// the tabulated closure of the fluid model (Sec. IV.A, eqs. 6-9).
//
// EEDF F(eps) with int eps^(1/2) F = 1, rates per gas density N, gamma =
// (2e/m)^(1/2).  Steady state: dG/deps = S, with the energy-space flux
//   G = -A dF/deps - B F,  A = (gamma/3)(E/N)^2 eps/sigma_m,  B = gamma (2m/M) eps^2 sigma_el
// (field heating, elastic recoil cooling with the gas at rest) and S the
// inelastic redistribution (excitation: eps -> eps - u_k; ionization: the
// scattered electron uniform on [0, eps - u_iz], no new electron).
//
// Discretisation: uniform energy cells; the face flux by the exponential
// (Scharfetter-Gummel) scheme, exact for constant A and B across a face, so
// it stays monotone where elastic cooling dominates; electrons moved by an
// inelastic process are put back conservatively (linear weights for a shift,
// exact overlaps for the uniform interval).  Because redistribution only
// moves electrons downward, the matrix has a single subdiagonal: with the
// first balance row replaced by the normalisation it is upper Hessenberg and
// is solved by O(n^2) elimination with adjacent-row pivoting.
#include <cmath>
#include <cstdlib>
#include <cstring>
#include <vector>

#include "pic.h"

namespace {

constexpr double kQe = 1.602176634e-19;
constexpr double kMe = 9.1093837015e-31;
constexpr double kAmu = 1.66053906660e-27;
constexpr double kTd = 1e-21;

double sigma_lin(const pic_xsec &x, double eps) {
  if (x.kind != PIC_ELASTIC && eps < x.threshold_eV) return 0.0;
  const double *E = x.energy_eV, *S = x.sigma_m2;
  const int n = x.n;
  if (eps <= E[0]) return S[0];
  if (eps >= E[n - 1]) return S[n - 1];
  int lo = 0, hi = n - 1;
  while (hi - lo > 1) {
    const int mid = (lo + hi) >> 1;
    if (E[mid] <= eps) lo = mid; else hi = mid;
  }
  return S[lo] + (eps - E[lo]) / (E[lo + 1] - E[lo]) * (S[lo + 1] - S[lo]);
}

// Bernoulli function z / (e^z - 1)
double bern(double z) {
  if (std::fabs(z) < 1e-4) return 1.0 - 0.5 * z + z * z / 12.0;
  return z / std::expm1(z);
}

struct Solver {
  int n;
  double d;
  std::vector<double> ec, ef;          // cell centres, interior faces
  std::vector<double> sm_c, sm_f, sel_f, sel_c;
  std::vector<std::vector<double>> sig_c;  // per electron process
  std::vector<int> kind;
  std::vector<double> thr;
  std::vector<double> M;               // dense n x n, row-major
  std::vector<double> F;
};

int solve_one(Solver &S, double EN_Td, double mratio, pic_transport *o) {
  const int n = S.n;
  const double d = S.d, g = std::sqrt(2.0 * kQe / kMe), EN = EN_Td * kTd;
  std::vector<double> &M = S.M;
  std::fill(M.begin(), M.end(), 0.0);
  auto at = [&](int r, int c) -> double & { return M[(size_t)r * n + c]; };
  // face fluxes G_{i+1/2} = (A/d) [bern(z) F_i - bern(-z) F_{i+1}], z = B d / A
  for (int i = 0; i + 1 < n; ++i) {
    const double A = g / 3.0 * EN * EN * S.ef[i] / S.sm_f[i];
    const double B = g * mratio * S.ef[i] * S.ef[i] * S.sel_f[i];
    const double z = B * d / A;
    const double ci = A / d * bern(z), cj = -A / d * bern(-z);
    at(i, i) += ci;
    at(i, i + 1) += cj;
    at(i + 1, i) -= ci;
    at(i + 1, i + 1) -= cj;
  }
  // inelastic sinks and the redistributed electrons
  for (size_t k = 0; k < S.kind.size(); ++k) {
    if (S.kind[k] == PIC_ELASTIC) continue;
    const std::vector<double> &s = S.sig_c[k];
    for (int j = 0; j < n; ++j) {
      if (s[j] <= 0.0) continue;
      const double R = d * g * S.ec[j] * s[j];
      at(j, j) += R;
      const double top = S.ec[j] - S.thr[k];
      if (top < 0.0) continue;
      if (S.kind[k] == PIC_EXCITATION) {
        const double pos = top / d - 0.5;
        const int c = (int)std::floor(pos);
        if (c < 0) {
          at(0, j) -= R;
        } else {
          const double fr = pos - c;
          at(c, j) -= R * (1.0 - fr);
          at(c + 1 < n ? c + 1 : n - 1, j) -= R * fr;
        }
      } else {
        if (top == 0.0) { at(0, j) -= R; continue; }
        const int cmax = std::min(n - 1, (int)(top / d));
        for (int c = 0; c <= cmax; ++c) {
          const double ov = std::min((c + 1) * d, top) - c * d;
          if (ov > 0.0) at(c, j) -= R * ov / top;
        }
      }
    }
  }
  // row 0 -> normalisation; row equilibration
  std::vector<double> rhs(n, 0.0);
  for (int c = 0; c < n; ++c) at(0, c) = std::sqrt(S.ec[c]) * d;
  rhs[0] = 1.0;
  for (int r = 0; r < n; ++r) {
    double mx = 0.0;
    for (int c = (r > 0 ? r - 1 : 0); c < n; ++c) mx = std::max(mx, std::fabs(at(r, c)));
    if (!(mx > 0.0)) return PIC_EINVAL;
    const double s = 1.0 / mx;
    for (int c = (r > 0 ? r - 1 : 0); c < n; ++c) at(r, c) *= s;
    rhs[r] *= s;
  }
  // upper Hessenberg elimination: only row k+1 has an entry below the diagonal in column k
  for (int k = 0; k + 1 < n; ++k) {
    if (std::fabs(at(k + 1, k)) > std::fabs(at(k, k))) {
      for (int c = k; c < n; ++c) std::swap(at(k, c), at(k + 1, c));
      std::swap(rhs[k], rhs[k + 1]);
    }
    const double p = at(k, k);
    if (p == 0.0) return PIC_EINVAL;
    const double l = at(k + 1, k) / p;
    if (l != 0.0) {
      for (int c = k; c < n; ++c) at(k + 1, c) -= l * at(k, c);
      rhs[k + 1] -= l * rhs[k];
    }
  }
  std::vector<double> &F = S.F;
  for (int r = n - 1; r >= 0; --r) {
    double acc = rhs[r];
    for (int c = r + 1; c < n; ++c) acc -= at(r, c) * F[c];
    F[r] = acc / at(r, r);
  }
  // transport integrals
  double ebar = 0.0, DN = 0.0, De = 0.0, mu = 0.0, mue = 0.0, lel = 0.0;
  for (int i = 0; i < n; ++i) {
    const double e = S.ec[i];
    ebar += e * std::sqrt(e) * F[i] * d;
    DN += e / S.sm_c[i] * F[i] * d;
    De += e * e / S.sm_c[i] * F[i] * d;
    lel += e * e * S.sel_c[i] * F[i] * d;
  }
  for (int i = 0; i + 1 < n; ++i) {
    mu += S.ef[i] / S.sm_f[i] * (F[i + 1] - F[i]);
    mue += S.ef[i] * S.ef[i] / S.sm_f[i] * (F[i + 1] - F[i]);
  }
  double nu_iz = 0.0, linel = 0.0;
  for (size_t k = 0; k < S.kind.size(); ++k) {
    if (S.kind[k] == PIC_ELASTIC) continue;
    double nu = 0.0;
    for (int i = 0; i < n; ++i) nu += S.ec[i] * S.sig_c[k][i] * F[i] * d;
    nu *= g;
    linel += S.thr[k] * nu;
    if (S.kind[k] == PIC_IONIZATION) nu_iz += nu;
  }
  o->EN_Td = EN_Td;
  o->mean_eps_eV = ebar;
  o->muN = -g / 3.0 * mu;
  o->DN = g / 3.0 * DN;
  o->mueN = -g / (3.0 * ebar) * mue;
  o->DeN = g / (3.0 * ebar) * De;
  o->nu_izN = nu_iz;
  o->lossN = g * mratio * lel + linel;
  o->powerN = o->muN * EN * EN;
  const double w = o->muN * EN;
  o->alphaN = w > 0.0 ? nu_iz / w : 0.0;
  if (!std::isfinite(ebar) || !std::isfinite(o->muN)) return PIC_EINVAL;
  return 0;
}

}  // namespace

extern "C" int pic_two_term(const pic_xsec *xs, int n_xsec, double gas_mass_amu, const double *EN_Td, int n_EN,
                            double eps_max_eV, int n_grid, pic_transport *out) {
  if (!xs || n_xsec <= 0 || !EN_Td || n_EN <= 0 || !out || !(gas_mass_amu > 0.0) || !(eps_max_eV > 0.0) ||
      n_grid < 64 || n_grid > 8192)
    return PIC_EINVAL;
  Solver S;
  S.n = n_grid;
  S.d = eps_max_eV / n_grid;
  const int n = n_grid;
  S.ec.resize(n);
  S.ef.resize(n - 1);
  for (int i = 0; i < n; ++i) S.ec[i] = (i + 0.5) * S.d;
  for (int i = 0; i + 1 < n; ++i) S.ef[i] = (i + 1) * S.d;
  S.sm_c.assign(n, 0.0);
  S.sel_c.assign(n, 0.0);
  S.sm_f.assign(n - 1, 0.0);
  S.sel_f.assign(n - 1, 0.0);
  for (int k = 0; k < n_xsec; ++k) {
    const pic_xsec &x = xs[k];
    if (x.kind > PIC_IONIZATION) continue;
    if (x.n < 1 || !x.energy_eV || !x.sigma_m2) return PIC_EINVAL;
    std::vector<double> sc(n);
    for (int i = 0; i < n; ++i) {
      sc[i] = sigma_lin(x, S.ec[i]);
      S.sm_c[i] += sc[i];
      if (x.kind == PIC_ELASTIC) S.sel_c[i] += sc[i];
    }
    for (int i = 0; i + 1 < n; ++i) {
      const double sf = sigma_lin(x, S.ef[i]);
      S.sm_f[i] += sf;
      if (x.kind == PIC_ELASTIC) S.sel_f[i] += sf;
    }
    S.sig_c.push_back(std::move(sc));
    S.kind.push_back(x.kind);
    S.thr.push_back(x.kind == PIC_ELASTIC ? 0.0 : x.threshold_eV);
  }
  for (int i = 0; i < n; ++i)
    if (!(S.sm_c[i] > 0.0)) return PIC_EINVAL;
  for (int i = 0; i + 1 < n; ++i)
    if (!(S.sm_f[i] > 0.0)) return PIC_EINVAL;
  try {
    S.M.assign((size_t)n * n, 0.0);
    S.F.assign(n, 0.0);
  } catch (...) {
    return PIC_ENOMEM;
  }
  const double mratio = 2.0 * kMe / (gas_mass_amu * kAmu);
  for (int q = 0; q < n_EN; ++q) {
    if (!(EN_Td[q] > 0.0)) return PIC_EINVAL;
    const int rc = solve_one(S, EN_Td[q], mratio, &out[q]);
    if (rc) return rc;
  }
  return 0;
}

namespace {

constexpr double kKb = 1.380649e-23;
constexpr double kTorr = 133.32236842105263;
constexpr double kPi = 3.14159265358979323846;

}  // namespace

extern "C" int pic_drive_ri(const pic_params *p, double out[4]) {
  if (!p || !out || !(p->R_m > 0.0) || !(p->I_A > 0.0) || !(p->pressure_torr > 0.0) || !(p->T_gas_K > 0.0) ||
      !(p->gas_mass_amu > 0.0) || !(p->eps_max_e_eV > 0.0) || p->n_xsec <= 0 || !p->xsec)
    return PIC_EINVAL;
  const double N = p->pressure_torr * kTorr / (kKb * p->T_gas_K);
  const double M = p->gas_mass_amu * kAmu;
  // ion mobility: momentum-transfer cross section at the mean thermal relative energy
  const double eps_th = 8.0 * kKb * p->T_gas_K / (kPi * kQe);
  double omega = 0.0;
  for (int k = 0; k < p->n_xsec; ++k) {
    const pic_xsec &x = p->xsec[k];
    if (x.n < 1 || !x.energy_eV || !x.sigma_m2) return PIC_EINVAL;
    if (x.kind == PIC_ION_CX) omega += 2.0 * sigma_lin(x, eps_th);
    if (x.kind == PIC_ION_ISO) omega += sigma_lin(x, eps_th);
  }
  if (!(omega > 0.0)) return PIC_EINVAL;
  const double mu_i = 3.0 * kQe / (16.0 * N * omega) * std::sqrt(2.0 * kPi / (0.5 * M * kKb * p->T_gas_K));
  const double g2 = (2.405 / p->R_m) * (2.405 / p->R_m);
  pic_transport tr;
  // balance f(E/N) = N nu_izN - (mu_i N / N)(DN / muN)(2.405/R)^2: negative below, positive above
  auto f = [&](double EN, int &rc) {
    rc = pic_two_term(p->xsec, p->n_xsec, p->gas_mass_amu, &EN, 1, p->eps_max_e_eV, 800, &tr);
    return N * tr.nu_izN - mu_i * (tr.DN / tr.muN) * g2;
  };
  int rc = 0;
  double lo = std::log(1.0), hi = std::log(2000.0);
  const double flo = f(std::exp(lo), rc);
  if (rc) return rc;
  const double fhi = f(std::exp(hi), rc);
  if (rc) return rc;
  if (!(flo < 0.0 && fhi > 0.0)) return PIC_EINVAL;
  for (int it = 0; it < 40; ++it) {
    const double mid = 0.5 * (lo + hi);
    const double fm = f(std::exp(mid), rc);
    if (rc) return rc;
    if (fm < 0.0) lo = mid; else hi = mid;
  }
  const double EN = std::exp(0.5 * (lo + hi));
  f(EN, rc);
  if (rc) return rc;
  const double E0 = EN * kTd * N;
  const double mu_e = tr.muN / N;
  const double J = p->I_A / (kPi * p->R_m * p->R_m);
  out[0] = E0;
  out[1] = J / (kQe * (mu_e + mu_i) * E0);
  out[2] = 2.0 / 3.0 * tr.mean_eps_eV;
  out[3] = mu_i * N;
  return 0;
}
