// Host build of the fixed-point sine / cosine of the voltage update
// (csrc/fixtrig.h) with its table, and of its FP64 -> FP32 truncation, for
// the CPU tests.
#include <cmath>
#include <vector>

#include "../paper_1711_10579_gb300/csrc/fixtrig.h"

static std::vector<long long> g_tab;

extern "C" {

void fx_init() {
  g_tab.resize(2 * (2 * pf::fx::kHalf + 1));
  for (int j = -pf::fx::kHalf; j <= pf::fx::kHalf; ++j) {
    const long double a = (long double)j / 128.0L;
    g_tab[2 * (j + pf::fx::kHalf)] = llroundl(cosl(a) * 4611686018427387904.0L);
    g_tab[2 * (j + pf::fx::kHalf) + 1] = llroundl(sinl(a) * 4611686018427387904.0L);
  }
}

int fx_sincos(int n, const double* a, double* s, double* c) {
  int ok = 0;
  for (int k = 0; k < n; ++k) ok += pf::fx::sincos_q(g_tab.data(), a[k], s + k, c + k) ? 1 : 0;
  return ok;
}

int fx_to_q60(double a, long long* q) {
  int64_t v = 0;
  const bool ok = pf::fx::to_q60(a, &v);
  *q = v;
  return ok;
}

double fx_from_q60(long long q) { return pf::fx::from_q60(q); }

void fx_to_f32(int n, const double* v, float* out) {
  for (int k = 0; k < n; ++k) out[k] = pf::fx::to_f32_trunc(v[k]);
}
}
