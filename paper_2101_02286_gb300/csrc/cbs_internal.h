// cbs_internal.h -- types shared by the host plan builder and the kernels.
#pragma once
#include <cstdint>
#include <string>
#include <vector>

#include "../../include/cbs.h"

namespace cbs {

constexpr int kMaxR = 3;            // half bandwidth (heptadiagonal)
constexpr int kMaxLanes = 32;       // partitions per line in the on-chip kernel
constexpr int kMaxStages = 16;      // >= 2 (popcount(p)-1) + floor(log2 p) + 1 for p <= 32
constexpr int kMaxRhsTerms = 3;

enum StageType { kDetach = 0, kPcr = 1, kFinal = 2, kReattach = 3 };

struct Stage {
  int type, s, na;
};

// Interface schedule of Algorithm 1 (cyclic) or classic block PCR (acyclic).
std::vector<Stage> build_schedule(int p, bool cyclic);

// Per-line matrix description used by the host factorisation: Toeplitz band
// value for offset t in [-r, r].
struct Bands {
  int r;
  double v[2 * kMaxR + 1];  // v[t + r]
  double at(int t) const { return (t < -r || t > r) ? 0.0 : v[t + r]; }
};

// Everything the on-chip kernel needs that does not depend on the RHS.
struct LineTables {
  int n = 0, r = 1, p = 1;
  bool cyclic = true;
  int rows_big = 0, rows_small = 0, count_big = 0;  // partition sizes
  int nmax = 0;                                      // max bulk rows (rows_big - r)
  std::vector<int> start, size;                      // per partition
  // Bulk LU factors of D_i (identical for all partitions of a Toeplitz
  // matrix because elimination runs from the top): per bulk row j,
  // fac[j*(2r+1) + q-1] = l_q (q=1..r), fac[j*(2r+1) + r] = 1/pivot,
  // fac[j*(2r+1) + r + q] = u_q / pivot (q=1..r).
  std::vector<double> fac;
  // S_i = D_i^{-1} L_i and R_i = D_i^{-1} U_i for a partition of rows_big
  // (srB) and of rows_small (srS) rows, layout [j * 2r + c], c < r: S column
  // c, c >= r: R column c - r (cyclic; an acyclic system's last partition has
  // R = 0, which the kernels apply themselves).
  std::vector<double> srB, srS;
  // b-hat assembly blocks (Eq. 21): Lt[q][e] multiplies y_{i-1}[N_{i-1}-r+e],
  // Ut[q][e] multiplies y_i[e]; identical for all partitions (Toeplitz).
  double Lt[kMaxR][kMaxR] = {}, Ut[kMaxR][kMaxR] = {};
  // Interface stages: per stage, per lane i: C, KM, KP (r x r each) and the
  // source lanes; layout coef[((stage * 3 + m) * r*r + e) * P + i],
  // src[(stage * 2 + k) * P + i].
  std::vector<Stage> stages;
  std::vector<double> coef;
  std::vector<int> src;
  std::vector<int> stage_has_c;  // 1 when C != I for some lane
  // bit 0 (FP64) / bit 1 (FP32): the stage's coupling blocks KM, KP exceed
  // rounding in that precision, so the stage needs the neighbours' values;
  // otherwise it reduces to x~ <- C x~ (or nothing when C = I).
  std::vector<int> stage_msg;
  // schedule counts (Sec. 4)
  int pcr_steps = 0, detach_steps = 0, detached_rows = 0;
  // Reduced system blocks before PCR (for introspection/tests): W = D-hat,
  // L-hat, U-hat per partition, r x r row-major.
  std::vector<double> Dhat, Lhat, Uhat;
};

// Build the tables. Returns "" on success or an error message; *singular is
// set when a pivot or interface block is zero / non-finite.
// sizes (optional): {count_big, rows_big, rows_small} instead of the default
// rule (first n mod p partitions get ceil(n / p) rows, the rest floor).
std::string build_line_tables(LineTables& T, int n, const Bands& A, int p, bool cyclic,
                              bool* singular, int max_lanes, const int* sizes = nullptr);

// Rows q < nrows of D^{-1} for the bulk block of N rows of plan tables T
// (forward/backward elimination with T.fac), row-major nrows x N.
std::vector<double> bulk_inverse_rows(const LineTables& T, int N, int nrows);

// Tables passed by value to the on-chip kernel (they live in the constant
// bank, so uniform reads cost no load instruction).
constexpr int kMaxBulk = 32;  // max bulk rows per partition (rows_big - r)
struct DevLineTables {
  double fac[kMaxBulk * (2 * kMaxR + 1)];  // bulk LU factors, [j*(2r+1) + c]
  double srB[kMaxBulk * 2 * kMaxR];        // S|R of a big partition, [j*2r + c]
  double srS[kMaxBulk * 2 * kMaxR];        // S|R of a small partition
  float facF[kMaxBulk * (2 * kMaxR + 1)];  // FP32 copies for the FP32 bulk
  float srBF[kMaxBulk * 2 * kMaxR];
  float srSF[kMaxBulk * 2 * kMaxR];
  double Lt[kMaxR][kMaxR], Ut[kMaxR][kMaxR];  // b-hat assembly (Eq. 21)
  double band[2 * kMaxR + 1];              // A's band values (t = -r..r)
  float bandHi[2 * kMaxR + 1], bandLo[2 * kMaxR + 1];  // split into two floats
  const double* coef;                      // interface stage coefficients
  const float* coefF;                      // FP32 copy (interface inside FP32 solves)
  const int* src;                          // interface stage source lanes
  // Uniform interface (every lane has the same blocks in every stage, which
  // holds for Toeplitz bands and p a power of two): per-stage C, KM, KP blocks
  // and the PCR stride; sources are (i -+ s) mod p.
  int uniform;
  int ustage_s[kMaxStages];
  double ucoef[kMaxStages][3 * kMaxR * kMaxR];
  float ucoefF[kMaxStages][3 * kMaxR * kMaxR];
  float LtF[kMaxR][kMaxR], UtF[kMaxR][kMaxR];
  int n, r, p, pw;                         // pw: lanes per line group (pow2 >= p)
  int rows_big, rows_small, count_big;
  int nstage, cyclic;
  int stage_has_c[kMaxStages];
  int stage_msg[kMaxStages];   // see LineTables::stage_msg
  // shared-memory tile: line slot S[l*lsz + k*sp + i] holds row k of partition i
  int lsz, sp, bound;          // bound = count_big * rows_big
  unsigned mag_b, mag_s;       // ceil(2^32 / rows_big), ceil(2^32 / rows_small)
  unsigned mag_n;              // ceil(2^32 / n)
  int rows_lg;                 // log2(rows_big) when all partitions equal and a power of two, else -1
};

}  // namespace cbs
