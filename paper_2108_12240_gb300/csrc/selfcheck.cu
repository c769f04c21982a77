// Test utilities: bhac_check_bit_ops (the integer-pipe compares and
// conversions of bhac_device.cuh against the hardware instructions they
// replace, and its FP64 reciprocal and square roots against the IEEE ones) and bhac_get_prims_ghosted (the ghosted primitive state, to check
// ghost fills cell by cell).
#include <math.h>

#include "ctx.h"
#include "bhac_device.cuh"

namespace bhac {
namespace {

constexpr int kChecks = 11;

// splitmix64 (Steele, Lea and Flood 2014): counter-based 64-bit generator
__device__ __forceinline__ unsigned long long mix64(unsigned long long z) {
  z += 0x9E3779B97F4A7C15ULL;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
  return z ^ (z >> 31);
}

__device__ double special_double(unsigned k) {
  switch (k % 16u) {
    case 0: return 0.0;
    case 1: return -0.0;
    case 2: return __longlong_as_double(0x7FF0000000000000LL);   // +inf
    case 3: return __longlong_as_double((long long)0xFFF0000000000000ULL);  // -inf
    case 4: return __longlong_as_double(0x7FF8000000000000LL);   // NaN
    case 5: return __longlong_as_double((long long)0xFFF8000000000001ULL);  // negative NaN
    case 6: return 3.4028234663852886e38;                        // FLT_MAX
    case 7: return 3.4028235677973366e38;                        // just past the last float tie
    case 8: return 1.1754943508222875e-38;                       // FLT_MIN
    case 9: return 1.401298464324817e-45;                        // smallest float subnormal
    case 10: return __longlong_as_double(1LL);                   // smallest double subnormal
    case 11: return 1.0;
    case 12: return -1.0;
    case 13: return 1.0 + 1.0 / 16777216.0;                      // exact tie above 1 (round to even: 1)
    case 14: return 1.0 + 3.0 / 16777216.0;                      // exact tie (round to even: up)
    default: return -2.5;
  }
}

// operand k of pair i: a mix of families
__device__ double operand(unsigned long long seed, long long i, int which) {
  const unsigned long long h = mix64(seed * 0x100000001B3ULL + (unsigned long long)i * 2ULL + (unsigned long long)which);
  const unsigned fam = (unsigned)(mix64(h) % 8ULL);
  if (fam == 0) return __longlong_as_double((long long)h);                   // any bit pattern
  if (fam == 1) return special_double((unsigned)(h >> 7));
  // a double in and around the float range: exponent 880..1170, sign random
  const unsigned long long E = 880ULL + (h >> 52) % 291ULL;
  unsigned long long m = h & 0x000FFFFFFFFFFFFFULL;
  if (fam == 3) m = (m & ~0x1FFFFFFFULL) | 0x10000000ULL;                    // exact tie for narrowing
  if (fam == 4) m &= ~0x1FFFFFFFULL;                                         // exactly a float
  const unsigned long long bits = ((h >> 11) & 0x8000000000000000ULL) | (E << 52) | m;
  return __longlong_as_double((long long)bits);
}

// Distance in units of the last place between two doubles of the same sign;
// any sign disagreement or NaN counts as far apart (unless both are NaN).
__device__ long long ulp_dist(double x, double y) {
  if (isnan(x) && isnan(y)) return 0;
  if (isnan(x) || isnan(y)) return 1LL << 62;
  const long long a = __double_as_longlong(x), b = __double_as_longlong(y);
  if ((a ^ b) < 0) return (x == y) ? 0 : (1LL << 62);  // +0 and -0 are equal
  return a > b ? a - b : b - a;
}

__global__ void check_kernel(long long n, unsigned long long seed, unsigned long long* bad) {
  unsigned long long loc[kChecks] = {0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0};
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    const double a = operand(seed, i, 0);
    double b = operand(seed, i, 1);
    const unsigned long long hb = mix64(seed ^ (unsigned long long)i);
    if ((hb & 7ULL) == 0ULL) b = a;                                          // equal
    if ((hb & 7ULL) == 1ULL) b = __longlong_as_double(__double_as_longlong(a) + 1LL);  // one ulp away
    if ((hb & 7ULL) == 2ULL) b = -a;
    if (lt_t(a, b) != (a < b)) ++loc[0];
    if (gt0_t(a) != (a > 0.0)) ++loc[1];
    if (le0_t(a) != (a <= 0.0)) ++loc[2];
    if (lt_abs_t(a, b) != (fabs(a) < fabs(b))) ++loc[3];
    if (le_x(a, b) != (a <= b) || lt0_x(a) != (a < 0.0)) ++loc[4];
    if (finite_t(a) != (bool)isfinite(a)) ++loc[5];
    const float f1 = narrow_f64(a), f0 = __double2float_rn(a);
    if (!(isnan(f1) && isnan(f0)) && __float_as_uint(f1) != __float_as_uint(f0)) ++loc[6];
    const float g = __uint_as_float((unsigned)(hb >> 32));
    const double w1 = widen_f32(g), w0 = (double)g;
    if (!(isnan(w1) && isnan(w0)) && __double_as_longlong(w1) != __double_as_longlong(w0)) ++loc[7];
    // the FP64 unit's reciprocal and square roots against the IEEE operations
    if (ulp_dist(rcp_t(a), __drcp_rn(a)) > 1) ++loc[8];
    if (ulp_dist(rsqrt_t(a), rsqrt(a)) > 2) ++loc[9];
    if (ulp_dist(sqrt_t(a), __dsqrt_rn(a)) > 2) ++loc[10];
  }
  for (int k = 0; k < kChecks; ++k)
    if (loc[k]) atomicAdd(bad + k, loc[k]);
}

// disagreement counters (file scope: the library allocates no device memory)
static __device__ unsigned long long g_bad[kChecks];

}  // namespace
}  // namespace bhac

using namespace bhac;

extern "C" bhac_status bhac_check_bit_ops(long long n, unsigned seed, long long out[11]) {
  if (!out || n < 1 || n > (1LL << 26)) return BHAC_ERR_ARG;
  unsigned long long h[kChecks] = {0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0};
  unsigned long long* d = nullptr;
  cudaError_t e = cudaGetSymbolAddress((void**)&d, g_bad);
  if (e == cudaSuccess) e = cudaMemcpy(d, h, sizeof(h), cudaMemcpyHostToDevice);
  if (e == cudaSuccess) {
    check_kernel<<<1024, 256>>>(n, (unsigned long long)seed, d);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaMemcpy(h, d, sizeof(h), cudaMemcpyDeviceToHost);
  if (e != cudaSuccess) return BHAC_ERR_CUDA;
  for (int k = 0; k < kChecks; ++k) out[k] = (long long)h[k];
  return BHAC_OK;
}

extern "C" bhac_status bhac_get_prims_ghosted(bhac_ctx* c, double* out, int on_device) {
  if (!c || !out) return BHAC_ERR_ARG;
  if (!c->prims_ok || c->mixed) return BHAC_ERR_STATE;
  const size_t bytes = sizeof(double) * NV * (size_t)c->nb * c->ncell;
  cudaError_t e = cudaMemcpyAsync(out, c->P[c->cur], bytes, on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost,
                                  c->st);
  if (e == cudaSuccess && !on_device) e = cudaStreamSynchronize(c->st);
  return e == cudaSuccess ? BHAC_OK : BHAC_ERR_CUDA;
}
