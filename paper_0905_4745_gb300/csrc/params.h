// params.h -- host-side construction of one SRFT realization (Section 3 of the
// paper) and of the tables the sketch kernels read.
#pragma once

#include <complex>
#include <cstdint>
#include <vector>

namespace mn {

// The random parameters, in the paper's notation (0-based):
//   T = S F D Theta Pi Z Theta~ Pi~ Z~   (Eqs. SRFT, SRFT2, Rokhlin_trans, big_def)
struct SrftParams {
  int64_t n = 0, l = 0;
  std::vector<std::complex<double>> zeta_t, zeta, d;  // unit-modulus diagonals Z~, Z, D
  std::vector<int64_t> pi_t, pi;                      // permutations, (Pi v)[j] = v[pi[j]]
  std::vector<double> theta_t, theta;                 // n-1 Givens angles each
  std::vector<int64_t> s;                             // l sampled rows of F, strictly increasing
};

// Draw from SplitMix64 counter streams: kind k (0..7 = zeta~, pi~, theta~, zeta,
// pi, theta, d, s), j-th draw = mix64(seed + G*(k*2^40 + j + 1)).
void draw_srft_params(uint64_t seed, int64_t n, int64_t l, SrftParams &P);

// Checks ranges (permutations, strictly increasing samples, finite values).
bool validate_srft_params(const SrftParams &P);

// Right halo of a Givens-chain segment: the number of elements past the
// segment end whose carry is still above `tol` (see sketch.cu). Returns, per
// segment of length `seg`, the halo length, and the maximum through hmax.
std::vector<int32_t> chain_halos(const std::vector<double> &theta, int64_t n, int seg, double tol,
                                 int *hmax);

// Tables of the DFT of a length n that is not a power of two, computed by
// Bluestein's identity j k = (j^2 + k^2 - (k - j)^2) / 2 as a circular
// convolution of power-of-two length L >= 2n - 1:
//   X_k = c_k sum_j (x_j c_j) conj(c_{k-j}),   c_j = exp(-pi i j^2 / n).
// chirp: c_j for j < n; bh: FFT_L(b) / L with b_t = conj(c_t) for |t| < n
// (indices mod L) and 0 elsewhere. Both in FP64 (the angle uses j^2 mod 2n).
void bluestein_tables(int64_t n, int64_t L, std::vector<std::complex<double>> &chirp,
                      std::vector<std::complex<double>> &bh);

}  // namespace mn
