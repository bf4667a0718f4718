// Stage plan of the line FFT (sn_fft.cuh), shared by the device transform and
// the host code that builds its twiddle tables.
//
// A line of N points is transformed by radix-R0, R1 (and R2) Stockham stages
// with every radix at most E, the elements a thread holds:
//   N <= 16          one stage, E = N;
//   32 .. 256        two stages, E = 16, R0 = N / 16 (2, 4, 8, 16), R1 = 16;
//   512, 1024        three stages, E = 16, R0 = R1 = 16, R2 = 2 or 4.
// Sixteen elements per thread keep a whole transform of any length in about
// 80 registers, so the long lines run at the occupancy of the short ones.
//
// Twiddle table (TWN entries of exp(-2 pi i x) in FP64 on the host):
//   two stages:   [r R0 + j] = exp(-2 pi i j r / N), r < R1, j < R0, for the
//                 forward transform, then [N + r R1 + j] = exp(+2 pi i j r / N),
//                 r < R0, j < R1, for the inverse (whose stages run R1, R0);
//                 TWN = 2N.
//   three stages: both directions run R0, R1, R2 and the inverse uses the
//                 conjugates: [r R0 + j] = exp(-2 pi i j r / (R0 R1)),
//                 r < R1, j < R0 (second stage), then
//                 [R0 R1 + r R0 R1 + j] = exp(-2 pi i j r / N), r < R2,
//                 j < R0 R1 (third stage); TWN = R0 R1 + N.
#pragma once

#include <cuda_runtime.h>

#include <cmath>

namespace snfft {

constexpr int plan_e(int N) { return N <= 16 ? N : 16; }
constexpr int plan_r0(int N) {
  return N <= 16 ? N : (N == 32 ? 2 : N == 64 ? 4 : N == 128 ? 8 : 16);
}
constexpr int plan_r1(int N) { return N <= 16 ? 1 : (N <= 256 ? N / plan_r0(N) : 16); }
constexpr int plan_r2(int N) { return N / (plan_r0(N) * plan_r1(N)); }
constexpr int plan_stages(int N) { return plan_r1(N) == 1 ? 1 : (plan_r2(N) == 1 ? 2 : 3); }
constexpr int plan_twn(int N) {
  return plan_stages(N) == 1 ? 0 : (plan_stages(N) == 2 ? 2 * N : plan_r0(N) * plan_r1(N) + N);
}

// Host: write the plan_twn(N) twiddles of length N to tw; returns plan_twn(N).
inline int plan_twiddles(int N, double2* tw) {
  constexpr double kTwoPi = 6.28318530717958647692;
  const int R0 = plan_r0(N), R1 = plan_r1(N);
  auto unit = [](double turns) {  // exp(2 pi i turns)
    return make_double2(std::cos(kTwoPi * turns), std::sin(kTwoPi * turns));
  };
  switch (plan_stages(N)) {
    case 2:
      for (int r = 0; r < R1; ++r)
        for (int j = 0; j < R0; ++j) tw[r * R0 + j] = unit(-(double)((long long)j * r % N) / N);
      for (int r = 0; r < R0; ++r)
        for (int j = 0; j < R1; ++j) tw[N + r * R1 + j] = unit((double)((long long)j * r % N) / N);
      break;
    case 3: {
      const int NB = R0 * R1, R2 = plan_r2(N);
      for (int r = 0; r < R1; ++r)
        for (int j = 0; j < R0; ++j) tw[r * R0 + j] = unit(-(double)((long long)j * r % NB) / NB);
      for (int r = 0; r < R2; ++r)
        for (int j = 0; j < NB; ++j) tw[NB + r * NB + j] = unit(-(double)((long long)j * r % N) / N);
      break;
    }
    default:
      break;
  }
  return plan_twn(N);
}

}  // namespace snfft
