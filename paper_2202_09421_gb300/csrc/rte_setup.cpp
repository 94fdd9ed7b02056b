// FP64 host set-up: FC derivative operators, phase matrix, Fresnel and
// boundary tables.  See rte_setup.h.
#include "rte_setup.h"

#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstdlib>
#include <cstring>

#include "fcgram_table.h"

namespace rte_setup {

int smooth5(int n) {
  for (int m = n;; ++m) {
    int r = m;
    for (int p : {2, 3, 5})
      while (r % p == 0) r /= p;
    if (r == 1) return m;
  }
}

// Filter sigma_k = exp(-alpha |2k/N_p|^(2 beta)) of eq. (FFilter).
static double filter(int k, int Np, double alpha, double beta) {
  double x = std::fabs(2.0 * k / Np);
  return std::exp(-alpha * std::pow(x, 2.0 * beta));
}

void fc_derivative_matrix(int n, double h, double alpha, double beta,
                          std::vector<double>& D) {
  const int d = FC_D, C = FC_C;
  const int Np = smooth5(n + C);
  const int kmax = (Np - 1) / 2;  // the Nyquist mode of an even N_p is dropped
  // Kernel of the filtered periodic derivative: derivative of the periodic
  // N_p-vector G is dG[p] = sum_q ker[(p - q) mod N_p] G[q], with
  // ker[r] = (1/N_p) sum_k (2 pi i k / (N_p h)) sigma_k e^{2 pi i k r / N_p}
  //        = -(4 pi / (N_p^2 h)) sum_{k=1}^{kmax} k sigma_k sin(2 pi k r / N_p).
  std::vector<double> ker(Np, 0.0), sig(kmax + 1);
  for (int k = 1; k <= kmax; ++k) sig[k] = filter(k, Np, alpha, beta);
  for (int r = 0; r < Np; ++r) {
    double s = 0.0;
    for (int k = 1; k <= kmax; ++k) {
      long long kr = (static_cast<long long>(k) * r) % Np;
      s += k * sig[k] * std::sin(2.0 * kPi * static_cast<double>(kr) / Np);
    }
    ker[r] = -4.0 * kPi / (static_cast<double>(Np) * Np * h) * s;
  }
  auto K = [&](int p) { int r = p % Np; if (r < 0) r += Np; return ker[r]; };
  D.assign(static_cast<size_t>(n) * n, 0.0);
  for (int i = 0; i < n; ++i)
    for (int j = 0; j < n; ++j) D[static_cast<size_t>(i) * n + j] = K(i - j);
  // Continuation rows p = n .. N_p-1 of the extension (steps 1-4 of the
  // continuation procedure): the right continuation starts right after
  // g[n-1] and uses g[n-d..n-1]; the left one ends right before g[0]
  // (periodically) and uses g[0..d-1] mirrored.
  for (int r = 0; r < C; ++r) {
    const int p_right = n + r;         // distance r + 1 past g[n-1]
    const int p_left = Np - 1 - r;     // distance r + 1 before g[0]
    for (int t = 0; t < d; ++t) {
      const double a = FC_CONT[r][t];
      const int j_right = n - d + t;   // z = t on the right end
      const int j_left = d - 1 - t;    // z = t mirrored on the left end
      for (int i = 0; i < n; ++i) {
        D[static_cast<size_t>(i) * n + j_right] += K(i - p_right) * a;
        D[static_cast<size_t>(i) * n + j_left] += K(i - p_left) * a;
      }
    }
  }
}

namespace {
constexpr int kFringe = 2;   // fringe points on each interior side (Sec. 4.4)

}  // namespace

void part_range(int n, int parts, int k, int& lo, int& hi, int& slo, int& shi) {
  lo = static_cast<int>(static_cast<long long>(k) * n / parts);
  hi = static_cast<int>(static_cast<long long>(k + 1) * n / parts);
  slo = k > 0 ? lo - kFringe : lo;
  shi = k < parts - 1 ? hi + kFringe : hi;
}

bool fc_derivative_matrix_parts(int n, double h, double alpha, double beta, int parts,
                                std::vector<double>& D) {
  if (parts <= 1) {
    fc_derivative_matrix(n, h, alpha, beta, D);
    return true;
  }
  D.assign(static_cast<size_t>(n) * n, 0.0);
  std::vector<double> Ds;
  for (int k = 0; k < parts; ++k) {
    int lo, hi, slo, shi;
    part_range(n, parts, k, lo, hi, slo, shi);
    const int ns = shi - slo;
    if (ns < 16) return false;
    fc_derivative_matrix(ns, h, alpha, beta, Ds);
    for (int i = lo; i < hi; ++i)
      for (int j = 0; j < ns; ++j)
        D[static_cast<size_t>(i) * n + slo + j] = Ds[static_cast<size_t>(i - slo) * ns + j];
  }
  return true;
}

double fc_spectral_radius_parts(int n, double h, double alpha, double beta, int parts) {
  if (parts <= 1) return fc_spectral_radius(n, h, alpha, beta);
  double best = 0.0;
  for (int k = 0; k < parts; ++k) {
    int lo, hi, slo, shi;
    part_range(n, parts, k, lo, hi, slo, shi);
    best = std::max(best, fc_spectral_radius(shi - slo, h, alpha, beta));
  }
  return best;
}

// Round an FP32 value to tf32 (10-bit mantissa), nearest with ties away
// from zero: add half of the dropped range to the magnitude and truncate.
static float tf32_round(float x) {
  uint32_t b;
  std::memcpy(&b, &x, 4);
  if ((b & 0x7f800000u) == 0x7f800000u) return x;
  b = (b + 0x1000u) & ~0x1fffu;
  float r;
  std::memcpy(&r, &b, 4);
  return r;
}

void tc_operator_image(const std::vector<double>& D, int n, std::vector<float>& img) {
  const int n_rows = (n + 127) / 128 * 128, n_kc = (n + 31) / 32;
  img.assign(static_cast<size_t>(n_kc) * 2 * n_rows * 32, 0.f);
  for (int q = 0; q < n_kc; ++q)
    for (int i = 0; i < n; ++i)
      for (int kk = 0; kk < 32; ++kk) {
        const int k = q * 32 + kk;
        if (k >= n) continue;
        const double v = D[static_cast<size_t>(i) * n + k];
        const float hi = tf32_round(static_cast<float>(v));
        const float lo = tf32_round(static_cast<float>(v - static_cast<double>(hi)));
        const size_t pos = static_cast<size_t>(i) * 32 + (((kk >> 2) ^ (i & 7)) << 2) + (kk & 3);
        const size_t base = static_cast<size_t>(q) * 2 * n_rows * 32;
        img[base + pos] = hi;
        img[base + static_cast<size_t>(n_rows) * 32 + pos] = lo;
      }
}

// Round an FP32 value to bf16 (8-bit significand), nearest with ties to
// even, returned as its upper 16 bits.
static unsigned short bf16_round(float x) {
  uint32_t b;
  std::memcpy(&b, &x, 4);
  if ((b & 0x7f800000u) != 0x7f800000u) b += 0x7fffu + ((b >> 16) & 1u);
  return static_cast<unsigned short>(b >> 16);
}

static double bf16_value(unsigned short h) {
  const uint32_t b = static_cast<uint32_t>(h) << 16;
  float f;
  std::memcpy(&f, &b, 4);
  return f;
}

void tc_operator_image_bf16(const std::vector<double>& D, int n, std::vector<unsigned short>& img) {
  const int n_rows = (n + 127) / 128 * 128, n_kc = (n + 63) / 64;
  img.assign(static_cast<size_t>(n_kc) * 2 * n_rows * 64, 0);
  for (int q = 0; q < n_kc; ++q)
    for (int i = 0; i < n; ++i)
      for (int kk = 0; kk < 64; ++kk) {
        const int k = q * 64 + kk;
        if (k >= n) continue;
        const double v = D[static_cast<size_t>(i) * n + k];
        const unsigned short hi = bf16_round(static_cast<float>(v));
        const unsigned short lo = bf16_round(static_cast<float>(v - bf16_value(hi)));
        const size_t pos = static_cast<size_t>(i) * 64 + (((kk >> 3) ^ (i & 7)) << 3) + (kk & 7);
        const size_t base = static_cast<size_t>(q) * 2 * n_rows * 64;
        img[base + pos] = hi;
        img[base + static_cast<size_t>(n_rows) * 64 + pos] = lo;
      }
}

void tc_phase_image(const std::vector<double>& P, int M, std::vector<float>& img) {
  img.assign(2 * 32 * 32, 0.f);
  for (int m = 0; m < M; ++m)
    for (int q = 0; q < M; ++q) {
      const double v = P[static_cast<size_t>(m) * M + q];
      const float hi = tf32_round(static_cast<float>(v));
      const float lo = tf32_round(static_cast<float>(v - static_cast<double>(hi)));
      const size_t pos = static_cast<size_t>(m) * 32 + (((q >> 2) ^ (m & 7)) << 2) + (q & 3);
      img[pos] = hi;
      img[32 * 32 + pos] = lo;
    }
}

void tc_segment_image(const std::vector<double>& D, int n, int lo, int hi, int slo, int shi, float* img) {
  std::fill(img, img + 2 * 16 * 32, 0.f);
  const int off = slo - lo + 2;
  for (int i = 0; i < hi - lo && i < 16; ++i)
    for (int s = 0; s < shi - slo; ++s) {
      const int p = s + off;
      if (p < 0 || p >= 32) continue;
      const double v = D[static_cast<size_t>(lo + i) * n + slo + s];
      const float h = tf32_round(static_cast<float>(v));
      const float l = tf32_round(static_cast<float>(v - static_cast<double>(h)));
      const size_t pos = static_cast<size_t>(i) * 32 + (((p >> 2) ^ (i & 7)) << 2) + (p & 3);
      img[pos] = h;
      img[16 * 32 + pos] = l;
    }
}

double fc_spectral_radius(int n, double h, double alpha, double beta) {
  const int Np = smooth5(n + FC_C);
  const int kmax = (Np - 1) / 2;
  double best = 0.0;
  for (int k = 1; k <= kmax; ++k) {
    double v = 2.0 * kPi * k / (Np * h) * filter(k, Np, alpha, beta);
    if (v > best) best = v;
  }
  return best;
}

void phase_matrix(int M, double g, double exponent, std::vector<double>& P) {
  const double w = 2.0 * kPi / M;
  P.assign(static_cast<size_t>(M) * M, 0.0);
  for (int m = 0; m < M; ++m) {
    double row = 0.0;
    for (int q = 0; q < M; ++q) {
      double c = std::cos(2.0 * kPi * (m - q) / M);
      double p = (1.0 - g * g) / (2.0 * kPi * std::pow(1.0 + g * g - 2.0 * g * c, exponent));
      P[static_cast<size_t>(m) * M + q] = p;
      row += w * p;
    }
    for (int q = 0; q < M; ++q) P[static_cast<size_t>(m) * M + q] *= w / row;
  }
}

double fresnel(double cos_i, double n_in, double n_out) {
  double ci = std::fabs(cos_i);
  double si = std::sqrt(std::fmax(0.0, 1.0 - ci * ci));
  double st = n_in / n_out * si;
  if (st >= 1.0) return 1.0;
  double ct = std::sqrt(1.0 - st * st);
  double rs = (n_in * ci - n_out * ct) / (n_in * ci + n_out * ct);
  double rp = (n_out * ci - n_in * ct) / (n_out * ci + n_in * ct);
  return 0.5 * (rs * rs + rp * rp);
}

double window(double v) {
  v = std::fabs(v);
  if (v == 0.0) return 1.0;
  if (v >= 1.0) return 0.0;
  return std::exp(2.0 * std::exp(-1.0 / v) / (v - 1.0));
}

void boundary_tables(int M, double n_in, double n_out, BoundaryTables& bt) {
  const double nu[4][2] = {{-1, 0}, {1, 0}, {0, -1}, {0, 1}};
  std::vector<double> fc(4 * M);
  bt.face_refl.assign(4 * M, 0);
  bt.face_f.assign(4 * M, 0.0);
  bt.face_act.assign(4 * M, 0);
  bt.wexit.assign(4 * M, 0.0);
  const double w = 2.0 * kPi / M;
  for (int F = 0; F < 4; ++F)
    for (int m = 0; m < M; ++m) {
      double th = 2.0 * kPi * m / M;
      double c = nu[F][0] * std::cos(th) + nu[F][1] * std::sin(th);
      fc[F * M + m] = c;
      // theta_r = 2 theta_nu - theta + pi: pi - theta on x-faces, -theta on y-faces
      bt.face_refl[F * M + m] = F < 2 ? ((M / 2 - m) % M + M) % M : (M - m) % M;
      bt.face_f[F * M + m] = fresnel(c, n_in, n_out);
      bt.face_act[F * M + m] = c < -kTieTol;
      if (c > kTieTol) bt.wexit[F * M + m] = w * (1.0 - fresnel(c, n_in, n_out)) * c;
    }
  const int cx[4] = {0, 1, 0, 1}, cy[4] = {2, 2, 3, 3};
  bt.corner_refl.assign(4 * M, 0);
  bt.corner_f.assign(4 * M, 0.0);
  bt.corner_act.assign(4 * M, 0);
  for (int c = 0; c < 4; ++c)
    for (int m = 0; m < M; ++m) {
      int Fx = cx[c], Fy = cy[c], F = -1;
      bool inx = bt.face_act[Fx * M + m], iny = bt.face_act[Fy * M + m];
      if (inx && iny) {
        // both faces incoming: the larger |theta . nu| governs, y-face on a tie
        F = std::fabs(fc[Fx * M + m]) > std::fabs(fc[Fy * M + m]) + kTieTol ? Fx : Fy;
      } else if (inx) {
        F = Fx;
      } else if (iny) {
        F = Fy;
      }
      if (F >= 0) {
        bt.corner_act[c * M + m] = 1;
        bt.corner_refl[c * M + m] = bt.face_refl[F * M + m];
        bt.corner_f[c * M + m] = bt.face_f[F * M + m];
      }
    }
}

bool bc_transpose_tables(const BoundaryTables& bt, int M, std::vector<int>& src, std::vector<double>& f) {
  src.assign(static_cast<size_t>(8) * M * 4, 0);
  f.assign(static_cast<size_t>(8) * M * 4, 0.0);
  for (int tb = 0; tb < 8; ++tb) {
    const bool face = tb < 4;
    const int base = (face ? tb : tb - 4) * M;
    const std::vector<int>& refl = face ? bt.face_refl : bt.corner_refl;
    const std::vector<double>& fc = face ? bt.face_f : bt.corner_f;
    const std::vector<unsigned char>& act = face ? bt.face_act : bt.corner_act;
    for (int k = 0; k < M; ++k) {
      const size_t e = (static_cast<size_t>(tb) * M + k) * 4;
      for (int q = 0; q < 4; ++q) src[e + q] = k;
      f[e] = act[base + k] ? 0.0 : 1.0;
      int used = 1;
      for (int m = 0; m < M; ++m) {
        if (!act[base + m] || refl[base + m] != k) continue;
        if (used == 4) return false;
        src[e + used] = m;
        f[e + used] = fc[base + m];
        ++used;
      }
    }
  }
  return true;
}

void ring_geometry(int nx, int ny, double xmin, double xmax, double ymin, double ymax,
                   std::vector<double>& px, std::vector<double>& py,
                   std::vector<double>& weight) {
  const double dx = (xmax - xmin) / (nx - 1), dy = (ymax - ymin) / (ny - 1);
  px.clear();
  py.clear();
  weight.clear();
  for (int F = 0; F < 4; ++F) {
    const int cnt = F < 2 ? ny : nx;
    for (int k = 0; k < cnt; ++k) {
      double x, y, wgt;
      if (F < 2) {
        x = F == 0 ? xmin : xmax;
        y = ymin + k * dy;
        wgt = dy;
      } else {
        x = xmin + k * dx;
        y = F == 2 ? ymin : ymax;
        wgt = dx;
      }
      if (k == 0 || k == cnt - 1) wgt *= 0.5;
      px.push_back(x);
      py.push_back(y);
      weight.push_back(wgt);
    }
  }
}

}  // namespace rte_setup
