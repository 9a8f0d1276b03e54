// Host-side check of the in-register DFT used by every FFT pass: for each
// length 1..32 and both directions, compares reg_dft against the direct
// definition sum_j x_j exp(-+2 pi i j k / n) evaluated in double precision,
// and the output-pruned form (only k < K and k >= n - K wanted) on those
// outputs, and the few-input DFT of the pruned window transform (inputs
// m >= NZ zero). Prints "max_rel_err_<type> <value>" and returns 0.
#include <math.h>
#include <stdio.h>

#include <random>

#include "../../paper_1705_03464_gb300/csrc/pg_fft_kernels.cuh"

using namespace pg::fft;

template <typename C, int RL, bool INV, int K = RL>
double check_one(std::mt19937& rng) {
  std::uniform_real_distribution<double> U(-1.0, 1.0);
  C a[RL];
  double xr[RL], xi[RL];
  for (int j = 0; j < RL; ++j) {
    xr[j] = U(rng);
    xi[j] = U(rng);
    a[j].x = (decltype(a[j].x))xr[j];
    a[j].y = (decltype(a[j].y))xi[j];
    xr[j] = a[j].x;
    xi[j] = a[j].y;
  }
  reg_dft<C, RL, INV, K>(a);
  double worst = 0.0, norm = 0.0;
  for (int k = 0; k < RL; ++k) {
    if (!(2 * K >= RL || k < K || k >= RL - K)) continue;
    double sr = 0.0, si = 0.0;
    for (int j = 0; j < RL; ++j) {
      double ang = (INV ? 2.0 : -2.0) * M_PI * (double)((j * k) % RL) / RL;
      sr += xr[j] * cos(ang) - xi[j] * sin(ang);
      si += xr[j] * sin(ang) + xi[j] * cos(ang);
    }
    norm = fmax(norm, sqrt(sr * sr + si * si));
    worst = fmax(worst, hypot(a[k].x - sr, a[k].y - si));
  }
  return worst / fmax(norm, 1e-300);
}

// The few-input forward DFT (inputs m >= NZ zero) against the definition.
template <typename C, int RL, int NZ>
double check_few(std::mt19937& rng) {
  std::uniform_real_distribution<double> U(-1.0, 1.0);
  C b[NZ], y[RL];
  double xr[NZ], xi[NZ];
  for (int m = 0; m < NZ; ++m) {
    b[m].x = (decltype(b[m].x))U(rng);
    b[m].y = (decltype(b[m].y))U(rng);
    xr[m] = b[m].x;
    xi[m] = b[m].y;
  }
  dft_few_inputs<C, RL, NZ>(b, y);
  double worst = 0.0, norm = 0.0;
  for (int k = 0; k < RL; ++k) {
    double sr = 0.0, si = 0.0;
    for (int m = 0; m < NZ; ++m) {
      double ang = -2.0 * M_PI * (double)((m * k) % RL) / RL;
      sr += xr[m] * cos(ang) - xi[m] * sin(ang);
      si += xr[m] * sin(ang) + xi[m] * cos(ang);
    }
    norm = fmax(norm, sqrt(sr * sr + si * si));
    worst = fmax(worst, hypot(y[k].x - sr, y[k].y - si));
  }
  return worst / fmax(norm, 1e-300);
}

template <typename C, bool INV>
double check_all(std::mt19937& rng) {
  double e = 0.0;
  for (int rep = 0; rep < 20; ++rep) {
    e = fmax(e, check_one<C, 1, INV>(rng));
    e = fmax(e, check_one<C, 2, INV>(rng));
    e = fmax(e, check_one<C, 4, INV>(rng));
    e = fmax(e, check_one<C, 8, INV>(rng));
    e = fmax(e, check_one<C, 16, INV>(rng));
    e = fmax(e, check_one<C, 32, INV>(rng));
    e = fmax(e, check_one<C, 32, INV, 1>(rng));
    e = fmax(e, check_one<C, 32, INV, 2>(rng));
    e = fmax(e, check_one<C, 32, INV, 3>(rng));
    e = fmax(e, check_one<C, 32, INV, 4>(rng));
    e = fmax(e, check_one<C, 32, INV, 8>(rng));
    e = fmax(e, check_one<C, 16, INV, 2>(rng));
    e = fmax(e, check_one<C, 16, INV, 4>(rng));
    e = fmax(e, check_one<C, 8, INV, 1>(rng));
    if (!INV) {
      e = fmax(e, check_few<C, 32, 2>(rng));
      e = fmax(e, check_few<C, 32, 4>(rng));
      e = fmax(e, check_few<C, 32, 8>(rng));
      e = fmax(e, check_few<C, 16, 4>(rng));
      e = fmax(e, check_few<C, 8, 2>(rng));
    }
  }
  return e;
}

int main() {
  std::mt19937 rng(7);
  double ef = fmax(check_all<float2, false>(rng), check_all<float2, true>(rng));
  double ed = fmax(check_all<double2, false>(rng), check_all<double2, true>(rng));
  printf("max_rel_err_f32 %.3e\nmax_rel_err_f64 %.3e\n", ef, ed);
  return 0;
}
