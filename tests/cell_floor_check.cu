// Host check of the fixed-point cell floor the FP64 streaming kernels use for a power-of-two
// cell size a: wherever cell_floor_fx decides, it must give floor(fl(x - s) / a), the FP64
// definition (the subtraction rounded once, the power-of-two scale exact).  Positions are
// uniform in the box, a few ulps either side of the faces of the shifted grid, within 2^-30
// cells of them, tiny, and zero; shifts are multiples of 2^-53 a in [-a/2, a/2) (and in
// [0, a), the walls case).  Prints the counts and exits 1 on any disagreement.
#include <cmath>
#include <cstdio>
#include <random>

#include "cellmath.cuh"

int main() {
  std::mt19937_64 rng(12345);
  std::uniform_real_distribution<double> U(0.0, 1.0);
  long total = 0, undecided = 0, undecided_uniform = 0, bad = 0;
  for (int log2a : {0, 1, -1, 3, -2}) {
    const double a = std::ldexp(1.0, log2a);
    for (int L : {16, 128, 1000, 1 << 20}) {
      const double B = L * a;
      for (long it = 0; it < 200000; ++it) {
        double s = (std::floor(U(rng) * 9007199254740992.0) / 9007199254740992.0 - 0.5) * a;
        if (it % 7 == 0 && s < 0.0) s += a;
        const int kind = static_cast<int>(it % 4);
        double x;
        if (kind == 0) {
          x = U(rng) * B;
        } else {
          const double face = s + std::floor(U(rng) * L) * a;
          const int steps = static_cast<int>(U(rng) * 41) - 20;
          x = face;
          for (int q = 0; q < std::abs(steps); ++q) x = std::nextafter(x, steps > 0 ? INFINITY : -INFINITY);
          if (kind == 3) x = face + (U(rng) * 2 - 1) * std::ldexp(a, -30);
          if (x < 0.0 || x >= B) continue;
        }
        if (it % 50 == 1) x = std::ldexp(U(rng), -static_cast<int>(U(rng) * 80));
        if (it % 97 == 2) x = 0.0;
        ++total;
        long long S;
        int c;
        if (!(mpcd::fx32_trunc(s, log2a, S) && mpcd::cell_floor_fx(x, S, log2a, c))) {
          ++undecided;
          if (kind == 0 && it % 50 != 1 && it % 97 != 2) ++undecided_uniform;
          continue;
        }
        const double ref = std::floor(std::ldexp(x - s, -log2a));
        if (static_cast<double>(c) != ref) {
          if (bad < 10) std::printf("x=%a s=%a log2a=%d: %d, FP64 %g\n", x, s, log2a, c, ref);
          ++bad;
        }
      }
    }
  }
  std::printf("total %ld undecided %ld undecided_uniform %ld bad %ld\n", total, undecided, undecided_uniform, bad);
  return bad ? 1 : 0;
}
