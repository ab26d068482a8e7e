// Host check of the library's Fourier mode selection (rom.cuh: ModeSel with
// its integer |k| threshold and integer bin edges), the code the GPU runs per
// mode: prints, for each (n, box) pair given on the command line, the number
// of matched real values (2 per selected mode) in each of the 100 bins.
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <vector>

#include "../paper_2604_26823_gb300/csrc/rom.cuh"

int main(int argc, char **argv) {
  for (int a = 1; a + 1 < argc; a += 2) {
    pm::rom::ModeSel m;
    m.n = std::atoi(argv[a]);
    m.h = m.n / 2 + 1;
    m.nbins = 100;
    m.kf = 2.0 * M_PI / std::atof(argv[a + 1]);
    m.kmin = 0.1;
    m.init_threshold();
    std::vector<long long> c(100, 0);
    for (int ix = 0; ix < m.n; ++ix)
      for (int iy = 0; iy < m.n; ++iy)
        for (int iz = 0; iz < m.h; ++iz) {
          const int b = m.bin_of(ix, iy, iz);
          if (b >= 0) c[b] += 2;
        }
    for (int b = 0; b < 100; ++b) std::printf("%lld%c", c[b], b == 99 ? '\n' : ' ');
  }
  return 0;
}
