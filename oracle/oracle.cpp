// FP64 CPU oracle for the iterative galactic-binary subtraction
// (arXiv 2602.18560, Appendix D "Subtraction algorithm", Sec. III.A).
//
// TEST INFRASTRUCTURE ONLY.  This file is the slow, plain, single-threaded
// reference that the CUDA path is checked against.  Only the test suite, the
// smoke check and the CPU-baseline leg of the benchmark may load it; the
// library itself never calls into it and shares no code, header, table or
// constant with it.
//
// Everything here follows the paper's statement of the method, in its order:
//   tables    : S_instr (App. C, SciRDv1 A channel, TDI-2 factor), R (App. B)
//   grid      : DFT bins k / T_obs inside [f_min, f_max] (Sec. III.B, Eq. SNR inner product band)
//   sources   : averaged incoherent power of a linear chirp (Eqs. GB waveform,
//               phase Taylor expansion) deposited over the bins it sweeps
//   SNR       : Eqs. SNR inner product / inner product, discretised on the bins
//   estimators: running mean (Eq. running mean), running median with the
//               chi^2_2 bias constant (Eq. running median), and median-then-mean
//   loop      : Algorithm of App. D: pre-filter rho >= kappa rho_th, then repeat
//               {estimate S_n, SNR, remove rho > rho_th} until none is removed.
//
// Readings of points the paper leaves open are listed in the design notes
// (window offsets, band edges, even-count median, normalisation K = 1/5, ...).
// Compiled with -ffp-contract=off so that no multiply-add is fused.

#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <vector>

namespace {

// Physical constants used by the oracle (App. B/C; L from Sec. III.A).
const double kC = 299792458.0;    // speed of light, m/s
const double kArm = 2.5e9;        // LISA arm length, m ("2.5 x 10^6 km")
const double kPi = 3.14159265358979323846;

// f* = c / (2 pi L)  (App. C, below the TDI PSDs).
double fstar() { return kC / (2.0 * kPi * kArm); }

// P_OMS(f), App. C: P^2 pm^2/Hz [1 + (2 mHz / f)^4] (2 pi f / c)^2 with P = 15.
double p_oms(double f) {
  double pm = 15.0e-12;
  double r = 2.0e-3 / f;
  double w = 2.0 * kPi * f / kC;
  return pm * pm * (1.0 + r * r * r * r) * w * w;
}

// P_TM(f), App. C: A^2 fm^2/s^4/Hz [1 + (0.4 mHz / f)^2][1 + (f / 8 mHz)^4]
// (2 pi f)^-4 (2 pi f / c)^2 with A = 3.  The printed bracket "(f/8 mHz^4)" is
// read as (f / 8 mHz)^4.
double p_tm(double f) {
  double fm = 3.0e-15;
  double r1 = 0.4e-3 / f;
  double r2 = f / 8.0e-3;
  double om = 2.0 * kPi * f;
  double w = om / kC;
  return fm * fm * (1.0 + r1 * r1) * (1.0 + r2 * r2 * r2 * r2) / (om * om * om * om) * w * w;
}

// S_instr^AA(f), App. C, times the TDI-2.0 factor 4 sin^2(2 f / f*) when tdi2.
double s_instr(double f, int tdi2) {
  double x = f / fstar();
  double s = std::sin(x);
  double c = std::cos(x);
  double v = 8.0 * s * s * (4.0 * (1.0 + c + c * c) * p_tm(f) + (2.0 + c) * p_oms(f));
  if (tdi2) {
    double s2 = std::sin(2.0 * x);
    v *= 4.0 * s2 * s2;
  }
  return v;
}

// R_AA(f) = 16 sin^2(f/f*) (f/f*)^2 (9/20) / (1 + 0.7 (f/f*)^2), App. B; the
// TDI-2.0 factor multiplies the signal response exactly as it multiplies the
// noise, so it is applied here too when tdi2.
double response(double f, int tdi2) {
  double x = f / fstar();
  double s = std::sin(x);
  double v = 16.0 * s * s * x * x * (9.0 / 20.0) / (1.0 + 0.7 * x * x);
  if (tdi2) {
    double s2 = std::sin(2.0 * x);
    v *= 4.0 * s2 * s2;
  }
  return v;
}

// Bias constant of the running median, C = (1 - 2/(9 nu))^-3 with nu = 2.
double median_bias() {
  double nu = 2.0;
  double b = 1.0 - 2.0 / (9.0 * nu);
  return 1.0 / (b * b * b);
}

struct Piece {
  int64_t j;   // local bin index (k - k_lo)
  double w;    // fraction of the sweep that falls inside the bin
};

// Bins swept by a source and the weight of each.  The instantaneous frequency of
// the chirp phi = phi0 + 2 pi f t + pi fdot t^2 runs linearly from f to
// f + fdot T over the observation, so it spends equal time per unit frequency:
// in bin units the sweep is [u0, u1] = [f T, f T + fdot T^2] and the weight of
// bin k is |[min, max] n [k - 1/2, k + 1/2)| / |u1 - u0|.  A sweep of zero
// length puts all its weight in the cell that holds it, bin floor(u0 + 1/2).
// Weight outside the band [k_lo, k_lo + n) is dropped.
void source_pieces(double T, int64_t k_lo, int64_t n, double f, double fdot,
                   std::vector<Piece>& out) {
  out.clear();
  double T2 = T * T;
  double u0 = f * T;
  double du = fdot * T2;
  double u1 = u0 + du;
  double lo = std::min(u0, u1);
  double hi = std::max(u0, u1);
  if (hi == lo) {
    int64_t k = (int64_t)std::floor(lo + 0.5);
    if (k >= k_lo && k < k_lo + n) out.push_back(Piece{k - k_lo, 1.0});
    return;
  }
  double len = hi - lo;
  int64_t ka = (int64_t)std::floor(lo + 0.5);
  int64_t kb = (int64_t)std::floor(hi + 0.5);
  for (int64_t k = ka; k <= kb; ++k) {
    double a = std::max(lo, (double)k - 0.5);
    double b = std::min(hi, (double)k + 0.5);
    if (!(b > a)) continue;
    if (k < k_lo || k >= k_lo + n) continue;
    out.push_back(Piece{k - k_lo, (b - a) / len});
  }
}

// Window of output bin j: [j - floor(W/2), j - floor(W/2) + W - 1] cut to the band.
void window_bounds(int64_t j, int64_t W, int64_t n, int64_t* a, int64_t* b) {
  int64_t s = j - W / 2;
  int64_t e = s + W - 1;
  if (s < 0) s = 0;
  if (e > n - 1) e = n - 1;
  *a = s;
  *b = e;
}

double window_mean(const double* x, int64_t a, int64_t b) {
  double s = 0.0;
  for (int64_t i = a; i <= b; ++i) s += x[i];
  return s / (double)(b - a + 1);
}

// Median of x[a..b]; an even count gives the mean of the two middle values.
double window_median(const double* x, int64_t a, int64_t b, std::vector<double>& tmp) {
  int64_t c = b - a + 1;
  tmp.assign(x + a, x + b + 1);
  int64_t m = c / 2;
  std::nth_element(tmp.begin(), tmp.begin() + m, tmp.end());
  double hi = tmp[m];
  if (c % 2 == 1) return hi;
  double lo = *std::max_element(tmp.begin(), tmp.begin() + m);
  return (lo + hi) * 0.5;
}

}  // namespace

extern "C" {

enum { ORC_MEAN = 0, ORC_MEDIAN = 1, ORC_MEDIAN_MEAN = 2 };

struct orc_params {
  double T_obs;
  double f_min;
  double f_max;
  int32_t window;
  int32_t estimator;
  double rho_th;
  double kappa;
  int32_t max_iter;
  int32_t tdi2;
  double conv_rtol;
};

struct orc_stats {
  int32_t iterations;
  int32_t converged;
  int64_t n_candidates;
  int64_t n_resolved;
};

double orc_fstar() { return fstar(); }
double orc_median_bias() { return median_bias(); }
double orc_p_oms(double f) { return p_oms(f); }
double orc_p_tm(double f) { return p_tm(f); }
double orc_s_instr(double f, int tdi2) { return s_instr(f, tdi2); }
double orc_response(double f, int tdi2) { return response(f, tdi2); }

// Frequency grid: bins k with f_k = k / T_obs, k_lo = ceil(f_min T), k_hi = floor(f_max T).
int orc_grid(double T, double f_min, double f_max, int64_t* k_lo, int64_t* n) {
  if (!(T > 0.0) || !(f_max > f_min) || !(f_min > 0.0)) return -1;
  int64_t a = (int64_t)std::ceil(f_min * T);
  int64_t b = (int64_t)std::floor(f_max * T);
  *k_lo = a;
  *n = b - a + 1;
  return *n > 0 ? 0 : -1;
}

// Per-bin tables S_instr(f_k) and R(f_k), f_k = k / T.
void orc_tables(double T, int64_t k_lo, int64_t n, int tdi2, double* S, double* R) {
  for (int64_t j = 0; j < n; ++j) {
    double f = (double)(k_lo + j) / T;
    S[j] = s_instr(f, tdi2);
    R[j] = response(f, tdi2);
  }
}

// Pieces of one source: returns their count (at most cap are written).
int64_t orc_source_pieces(double T, int64_t k_lo, int64_t n, double f, double fdot,
                          int64_t* j_out, double* w_out, int64_t cap) {
  std::vector<Piece> p;
  source_pieces(T, k_lo, n, f, fdot, p);
  for (size_t i = 0; i < p.size() && (int64_t)i < cap; ++i) {
    j_out[i] = p[i].j;
    w_out[i] = p[i].w;
  }
  return (int64_t)p.size();
}

// Running estimator over the whole band (Eqs. running mean / running median).
// The median output includes the bias constant C; median-then-mean applies the
// mean to the median output.
void orc_smooth(int est, int64_t W, const double* P, int64_t n, double* out) {
  std::vector<double> tmp;
  if (est == ORC_MEAN) {
    for (int64_t j = 0; j < n; ++j) {
      int64_t a, b;
      window_bounds(j, W, n, &a, &b);
      out[j] = window_mean(P, a, b);
    }
    return;
  }
  double C = median_bias();
  std::vector<double> med(n);
  for (int64_t j = 0; j < n; ++j) {
    int64_t a, b;
    window_bounds(j, W, n, &a, &b);
    med[j] = C * window_median(P, a, b, tmp);
  }
  if (est == ORC_MEDIAN) {
    for (int64_t j = 0; j < n; ++j) out[j] = med[j];
    return;
  }
  for (int64_t j = 0; j < n; ++j) {
    int64_t a, b;
    window_bounds(j, W, n, &a, &b);
    out[j] = window_mean(med.data(), a, b);
  }
}

// The same estimator evaluated only at the listed output bins (for spot checks
// at sizes where the whole band is too slow).
void orc_smooth_at(int est, int64_t W, const double* P, int64_t n, const int64_t* idx,
                   int64_t m, double* out) {
  std::vector<double> tmp;
  double C = median_bias();
  for (int64_t q = 0; q < m; ++q) {
    int64_t j = idx[q];
    int64_t a, b;
    window_bounds(j, W, n, &a, &b);
    if (est == ORC_MEAN) {
      out[q] = window_mean(P, a, b);
    } else if (est == ORC_MEDIAN) {
      out[q] = C * window_median(P, a, b, tmp);
    } else {
      double s = 0.0;
      for (int64_t i = a; i <= b; ++i) {
        int64_t a2, b2;
        window_bounds(i, W, n, &a2, &b2);
        s += C * window_median(P, a2, b2, tmp);
      }
      out[q] = s / (double)(b - a + 1);
    }
  }
}

// D_k = sum over sources not excluded of A_s^2 w_sk, summed in ascending s.
// exclude may be null (no source excluded); a nonzero byte excludes the source.
void orc_deposit(double T, int64_t k_lo, int64_t n, const double* A, const double* f,
                 const double* fdot, int64_t nsrc, const uint8_t* exclude, double* D) {
  std::vector<Piece> p;
  for (int64_t j = 0; j < n; ++j) D[j] = 0.0;
  for (int64_t s = 0; s < nsrc; ++s) {
    if (exclude && exclude[s]) continue;
    source_pieces(T, k_lo, n, f[s], fdot[s], p);
    double a2 = A[s] * A[s];
    for (const Piece& q : p) D[q.j] += a2 * q.w;
  }
}

// Channel power P_k = (T/5) R_k D_k: the inclination/polarisation average of
// h+^2 + hx^2 is (2/5) A^2, the A-channel response is R times half of it, and
// the one-sided periodogram of a tone observed for T is T times its mean square.
void orc_power(double T, const double* R, const double* D, int64_t n, double* P) {
  double t5 = T / 5.0;
  for (int64_t j = 0; j < n; ++j) P[j] = t5 * R[j] * D[j];
}

// rho^2 of each listed source against S_n = S_instr + S_gal (S_gal may be null
// for S_gal = 0): rho^2 = sum over A and E of 4 sum_k P_sk / S_n,k
// = 4 (T/5) A^2 sum_k w_k R_k / S_n,k  (Eqs. SNR inner product / inner product;
// T is insensitive and dropped, A and E are identical under the average).
void orc_snr2(double T, int64_t k_lo, int64_t n, const double* S_instr, const double* R,
              const double* S_gal, const double* A, const double* f, const double* fdot,
              int64_t nsrc, double* rho2) {
  std::vector<Piece> p;
  double t5 = T / 5.0;
  for (int64_t s = 0; s < nsrc; ++s) {
    source_pieces(T, k_lo, n, f[s], fdot[s], p);
    double a2 = A[s] * A[s];
    double acc = 0.0;
    for (const Piece& q : p) {
      double Sn = S_instr[q.j] + (S_gal ? S_gal[q.j] : 0.0);
      double Psk = t5 * R[q.j] * a2 * q.w;
      acc += Psk / Sn;
    }
    rho2[s] = 2.0 * 2.0 * acc;
  }
}

// The subtraction algorithm of App. D.
//   1. rho_0 of every source against S_instr; candidates C = {rho_0 >= kappa rho_th}.
//   2. repeat: D from all sources not resolved; S_gal = est_W((T/5) R D);
//      rho of every unresolved candidate against S_instr + S_gal;
//      New = {rho > rho_th}; stop if New is empty; else resolve all of New.
//   3. if max_iter runs out, S_gal is re-estimated from the final resolved set
//      and the run reports "not converged".
//   An optional relative tolerance on S_n (conv_rtol > 0) also stops the loop.
// S_gal (n values) and resolved (nsrc bytes) are written; trace, if not null,
// receives the S_gal of every iteration (trace_cap iterations at most).
int orc_run(const orc_params* prm, const double* A, const double* f, const double* fdot,
            int64_t nsrc, double* S_gal, uint8_t* resolved, orc_stats* st, double* trace,
            int64_t trace_cap) {
  int64_t k_lo, n;
  if (orc_grid(prm->T_obs, prm->f_min, prm->f_max, &k_lo, &n) != 0) return -1;
  if (prm->window < 1 || prm->max_iter < 1) return -1;
  double T = prm->T_obs;
  std::vector<double> S(n), R(n), D(n), P(n), Sg(n), Sprev(n);
  orc_tables(T, k_lo, n, prm->tdi2, S.data(), R.data());

  std::vector<double> rho2(nsrc);
  orc_snr2(T, k_lo, n, S.data(), R.data(), nullptr, A, f, fdot, nsrc, rho2.data());
  double pre = prm->kappa * prm->rho_th;
  std::vector<int64_t> cand;
  for (int64_t s = 0; s < nsrc; ++s)
    if (rho2[s] >= pre * pre) cand.push_back(s);

  std::vector<uint8_t> res(nsrc, 0);
  double th2 = prm->rho_th * prm->rho_th;
  int iters = 0;
  int converged = 0;
  std::vector<double> one(1);
  for (int it = 1; it <= prm->max_iter; ++it) {
    iters = it;
    orc_deposit(T, k_lo, n, A, f, fdot, nsrc, res.data(), D.data());
    orc_power(T, R.data(), D.data(), n, P.data());
    orc_smooth(prm->estimator, prm->window, P.data(), n, Sg.data());
    if (trace && it <= trace_cap) std::memcpy(trace + (int64_t)(it - 1) * n, Sg.data(), n * sizeof(double));
    if (prm->conv_rtol > 0.0 && it > 1) {
      double worst = 0.0;
      for (int64_t j = 0; j < n; ++j) {
        double a = S[j] + Sg[j], b = S[j] + Sprev[j];
        double r = std::fabs(a - b) / a;
        if (r > worst) worst = r;
      }
      if (worst <= prm->conv_rtol) {
        converged = 1;
        break;
      }
    }
    Sprev = Sg;
    std::vector<int64_t> fresh;
    for (int64_t s : cand) {
      if (res[s]) continue;
      double r2;
      orc_snr2(T, k_lo, n, S.data(), R.data(), Sg.data(), A + s, f + s, fdot + s, 1, &r2);
      if (r2 > th2) fresh.push_back(s);
    }
    if (fresh.empty()) {
      converged = 1;
      break;
    }
    for (int64_t s : fresh) res[s] = 1;
    if (it == prm->max_iter) {
      orc_deposit(T, k_lo, n, A, f, fdot, nsrc, res.data(), D.data());
      orc_power(T, R.data(), D.data(), n, P.data());
      orc_smooth(prm->estimator, prm->window, P.data(), n, Sg.data());
    }
  }
  int64_t nres = 0;
  for (int64_t s = 0; s < nsrc; ++s) nres += res[s];
  for (int64_t j = 0; j < n; ++j) S_gal[j] = Sg[j];
  std::memcpy(resolved, res.data(), nsrc);
  st->iterations = iters;
  st->converged = converged;
  st->n_candidates = (int64_t)cand.size();
  st->n_resolved = nres;
  return converged ? 0 : 1;
}

// Coarse-graining (Sec. "Coarse-graining of the data": the bin averages of the spectrum
// and of the frequencies).  The band [f_min, f_max] is split into nb logarithmically spaced
// bins with edges e_k = 10^(log10 f_min + k (log10 f_max - log10 f_min) / nb).  Reading:
// bin k holds the grid frequencies f_i = (k_lo + i) / T with e_k <= f_i < e_{k+1}; the
// first bin also takes the grid frequencies below e_1, the last those from e_{nb-1} on.
// Each bin averages x and f over its frequencies; an empty bin gets NaN and a zero count.
void orc_coarse_grain(double T, double f_min, double f_max, int64_t k_lo, int64_t n,
                      const double* x, int32_t nb, double* S_out, double* f_out, int64_t* cnt) {
  const double l0 = std::log10(f_min), l1 = std::log10(f_max);
  std::vector<double> edge(nb + 1);
  for (int32_t k = 0; k <= nb; ++k) edge[k] = std::pow(10.0, l0 + (double)k * (l1 - l0) / (double)nb);
  std::vector<double> sx(nb, 0.0), sf(nb, 0.0);
  std::vector<int64_t> c(nb, 0);
  for (int64_t i = 0; i < n; ++i) {
    const double f = (double)(k_lo + i) / T;
    int32_t k = 0;
    while (k + 1 < nb && f >= edge[k + 1]) ++k;  // the highest bin whose lower edge is <= f
    sx[k] += x[i];
    sf[k] += f;
    c[k] += 1;
  }
  for (int32_t k = 0; k < nb; ++k) {
    cnt[k] = c[k];
    S_out[k] = c[k] ? sx[k] / (double)c[k] : std::nan("");
    f_out[k] = c[k] ? sf[k] / (double)c[k] : std::nan("");
  }
}

}  // extern "C"
