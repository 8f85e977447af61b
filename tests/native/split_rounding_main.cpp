// Host driver for the bf16 term split used by the split-precision staging kernels: reads
// doubles from argv[1] and writes, for each value, ten unsigned 16-bit integers to argv[2]:
// its 3-term split (a_0, a_1, a_2 bf16 bit patterns) and 2-term split (a_0, a_1) by the
// scalar split, then the same five by the paired split (values taken two at a time, an odd
// last value paired with 0).
#include <stdio.h>
#include <stdlib.h>

#include <vector>

#include "../../paper_1509_00309_gb300/csrc/split_bf16.cuh"

int main(int argc, char** argv) {
  if (argc != 3) return 2;
  FILE* f = fopen(argv[1], "rb");
  if (!f) return 3;
  std::vector<double> x;
  double v;
  while (fread(&v, sizeof v, 1, f) == 1) x.push_back(v);
  fclose(f);
  const size_t n = x.size();
  std::vector<unsigned short> out(n * 10);
  for (size_t i = 0; i < n; ++i) {
    unsigned short t3[3], t2[2];
    clr::split::split_bf16<3>(x[i], t3);
    clr::split::split_bf16<2>(x[i], t2);
    unsigned short* o = &out[i * 10];
    o[0] = t3[0], o[1] = t3[1], o[2] = t3[2], o[3] = t2[0], o[4] = t2[1];
  }
  for (size_t i = 0; i < n; i += 2) {
    const double a = x[i], b = i + 1 < n ? x[i + 1] : 0.0;
    unsigned p3[3], p2[2];
    clr::split::split_bf16_pair<3>(a, b, p3);
    clr::split::split_bf16_pair<2>(a, b, p2);
    for (int e = 0; e < 2 && i + e < n; ++e) {
      unsigned short* o = &out[(i + e) * 10 + 5];
      const int sh = 16 * e;
      o[0] = (unsigned short)(p3[0] >> sh), o[1] = (unsigned short)(p3[1] >> sh);
      o[2] = (unsigned short)(p3[2] >> sh);
      o[3] = (unsigned short)(p2[0] >> sh), o[4] = (unsigned short)(p2[1] >> sh);
    }
  }
  FILE* g = fopen(argv[2], "wb");
  if (!g) return 4;
  const size_t w = fwrite(out.data(), sizeof(unsigned short), out.size(), g);
  fclose(g);
  return w == out.size() ? 0 : 5;
}
