// params.cpp -- host construction of the SRFT realization (Section 3).
//
// The paper fixes distributions, not a generator: d, zeta, zeta~ i.i.d. uniform
// on the unit circle; Pi, Pi~ uniform random permutations; theta, theta~ i.i.d.
// uniform on [0, 2 pi]; the l rows of F drawn without replacement (as the
// paper's own implementation does, which keeps the rows of T orthonormal).
// Random bits come from SplitMix64 (Steele, Lea & Flood, OOPSLA 2014) used as
// one counter-based stream per parameter kind; bounded integers from Lemire's
// multiply-shift rejection method (ACM TOMS 45(1), 2019); permutations from the
// Durstenfeld form of the Fisher-Yates shuffle. The sample is sorted, which
// only reorders the rows of the sketch and leaves R unchanged.
#include "params.h"

#include <algorithm>
#include <cmath>

namespace mn {

namespace {

constexpr uint64_t kGamma = 0x9E3779B97F4A7C15ULL;

inline uint64_t splitmix_finalize(uint64_t z) {
  z ^= z >> 30;
  z *= 0xBF58476D1CE4E5B9ULL;
  z ^= z >> 27;
  z *= 0x94D049BB133111EBULL;
  z ^= z >> 31;
  return z;
}

class Stream {
 public:
  Stream(uint64_t seed, uint64_t kind) : base_(seed + kGamma * (kind << 40)), count_(0) {}
  uint64_t next() { return splitmix_finalize(base_ + kGamma * (++count_)); }
  // [0, 1) with 53 random bits
  double unit() { return static_cast<double>(next() >> 11) * 0x1.0p-53; }
  // uniform in [0, bound), unbiased
  uint64_t below(uint64_t bound) {
    unsigned __int128 wide = static_cast<unsigned __int128>(next()) * bound;
    uint64_t low = static_cast<uint64_t>(wide);
    if (low < bound) {
      const uint64_t reject_below = (0 - bound) % bound;
      while (low < reject_below) {
        wide = static_cast<unsigned __int128>(next()) * bound;
        low = static_cast<uint64_t>(wide);
      }
    }
    return static_cast<uint64_t>(wide >> 64);
  }

 private:
  uint64_t base_, count_;
};

constexpr double kTwoPi = 6.283185307179586476925286766559;

void unit_circle(Stream &st, int64_t n, std::vector<std::complex<double>> &out) {
  out.resize(n);
  for (int64_t j = 0; j < n; ++j) {
    const double a = kTwoPi * st.unit();
    out[j] = std::complex<double>(std::cos(a), std::sin(a));
  }
}

void angles(Stream &st, int64_t count, std::vector<double> &out) {
  out.resize(count);
  for (int64_t k = 0; k < count; ++k) out[k] = kTwoPi * st.unit();
}

void shuffle(Stream &st, int64_t n, std::vector<int64_t> &p) {
  p.resize(n);
  for (int64_t j = 0; j < n; ++j) p[j] = j;
  for (int64_t i = n - 1; i >= 1; --i) {
    const int64_t j = static_cast<int64_t>(st.below(static_cast<uint64_t>(i) + 1));
    std::swap(p[i], p[j]);
  }
}

void sample(Stream &st, int64_t n, int64_t l, std::vector<int64_t> &s) {
  std::vector<int64_t> pool(n);
  for (int64_t j = 0; j < n; ++j) pool[j] = j;
  for (int64_t i = 0; i < l; ++i) {
    const int64_t j = i + static_cast<int64_t>(st.below(static_cast<uint64_t>(n - i)));
    std::swap(pool[i], pool[j]);
  }
  s.assign(pool.begin(), pool.begin() + l);
  std::sort(s.begin(), s.end());
}

}  // namespace

void draw_srft_params(uint64_t seed, int64_t n, int64_t l, SrftParams &P) {
  P.n = n;
  P.l = l;
  { Stream st(seed, 0); unit_circle(st, n, P.zeta_t); }
  { Stream st(seed, 1); shuffle(st, n, P.pi_t); }
  { Stream st(seed, 2); angles(st, n - 1, P.theta_t); }
  { Stream st(seed, 3); unit_circle(st, n, P.zeta); }
  { Stream st(seed, 4); shuffle(st, n, P.pi); }
  { Stream st(seed, 5); angles(st, n - 1, P.theta); }
  { Stream st(seed, 6); unit_circle(st, n, P.d); }
  { Stream st(seed, 7); sample(st, n, l, P.s); }
}

bool validate_srft_params(const SrftParams &P) {
  const int64_t n = P.n, l = P.l;
  if (n < 2 || l < 1 || l > n) return false;
  if ((int64_t)P.zeta_t.size() != n || (int64_t)P.zeta.size() != n || (int64_t)P.d.size() != n) return false;
  if ((int64_t)P.theta_t.size() != n - 1 || (int64_t)P.theta.size() != n - 1) return false;
  if ((int64_t)P.s.size() != l) return false;
  for (const auto *perm : {&P.pi_t, &P.pi}) {
    if ((int64_t)perm->size() != n) return false;
    std::vector<char> seen(n, 0);
    for (int64_t v : *perm) {
      if (v < 0 || v >= n || seen[v]) return false;
      seen[v] = 1;
    }
  }
  for (int64_t t = 0; t < l; ++t) {
    if (P.s[t] < 0 || P.s[t] >= n) return false;
    if (t > 0 && P.s[t] <= P.s[t - 1]) return false;
  }
  for (const auto *v : {&P.zeta_t, &P.zeta, &P.d})
    for (const auto &z : *v)
      if (!std::isfinite(z.real()) || !std::isfinite(z.imag())) return false;
  for (const auto *v : {&P.theta_t, &P.theta})
    for (double t : *v)
      if (!std::isfinite(t)) return false;
  return true;
}

// Chain Theta = G_0 ... G_{n-2} applied with G_{n-2} first is the reverse
// recurrence C_k = cos(t_k) v_k + sin(t_k) C_{k+1} (C_{n-1} = v_{n-1}). A
// segment whose outputs need C_j for j < e is computed exactly up to a term
// prod_{k=e-1}^{E-1} sin(t_k) * C_E when the recurrence is started at E with
// C_E = 0. The halo is the smallest E - e making that product <= tol (or E = n,
// where the start is exact).
std::vector<int32_t> chain_halos(const std::vector<double> &theta, int64_t n, int seg, double tol,
                                 int *hmax) {
  const int64_t nseg = (n + seg - 1) / seg;
  std::vector<int32_t> h(nseg, 0);
  int mx = 0;
  for (int64_t g = 0; g < nseg; ++g) {
    const int64_t e = std::min<int64_t>((g + 1) * seg, n);  // one past the segment's outputs
    if (e >= n) { h[g] = 0; continue; }
    double prod = std::fabs(std::sin(theta[e - 1]));
    int64_t E = e;
    while (prod > tol && E < n) {
      prod *= (E <= n - 2) ? std::fabs(std::sin(theta[E])) : 0.0;
      ++E;
    }
    h[g] = static_cast<int32_t>(E - e);
    mx = std::max(mx, h[g]);
  }
  *hmax = mx;
  return h;
}

// in-place radix-2 FFT, forward (e^{-2 pi i jk/L}), natural order in and out
static void host_fft_pow2(std::vector<std::complex<double>> &a) {
  const int64_t L = (int64_t)a.size();
  for (int64_t i = 1, j = 0; i < L; ++i) {
    int64_t bit = L >> 1;
    for (; j & bit; bit >>= 1) j ^= bit;
    j ^= bit;
    if (i < j) std::swap(a[i], a[j]);
  }
  const double two_pi = 6.283185307179586476925286766559;
  for (int64_t h = 1; h < L; h <<= 1) {
    for (int64_t k = 0; k < h; ++k) {
      const double ang = -two_pi * (double)k / (double)(2 * h);
      const std::complex<double> w(std::cos(ang), std::sin(ang));
      for (int64_t s0 = 0; s0 < L; s0 += 2 * h) {
        const std::complex<double> u = a[s0 + k], v = a[s0 + k + h] * w;
        a[s0 + k] = u + v;
        a[s0 + k + h] = u - v;
      }
    }
  }
}

void bluestein_tables(int64_t n, int64_t L, std::vector<std::complex<double>> &chirp,
                      std::vector<std::complex<double>> &bh) {
  const double pi = 3.14159265358979323846264338327950;
  chirp.resize(n);
  for (int64_t j = 0; j < n; ++j) {
    const int64_t q = (int64_t)(((uint64_t)j * (uint64_t)j) % (uint64_t)(2 * n));  // j < 2^31
    const double ang = -pi * (double)q / (double)n;
    chirp[j] = std::complex<double>(std::cos(ang), std::sin(ang));
  }
  std::vector<std::complex<double>> b(L, std::complex<double>(0.0, 0.0));
  for (int64_t t = 0; t < n; ++t) {
    b[t] = std::conj(chirp[t]);
    if (t > 0) b[L - t] = std::conj(chirp[t]);
  }
  host_fft_pow2(b);
  bh.resize(L);
  for (int64_t k = 0; k < L; ++k) bh[k] = b[k] / (double)L;
}

}  // namespace mn
