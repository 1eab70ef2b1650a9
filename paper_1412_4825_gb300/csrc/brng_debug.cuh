// brng_debug.cuh -- protocol checks of the checked build (-DBRNG_DEBUG).
//
// The rings are caches of a fixed sequence, so a read of an element that was
// never generated, a read pointer moved past the generated ones, or a table
// lookup outside its range gives a wrong value rather than a fault.  The
// checked build tests those conditions where they matter (after each refill,
// at each consumption, at each job lookup) and counts the ones that fail in a
// device word per translation unit, read on the host through
// brng_debug_violations (include/brng.h).  Nothing traps: a failed check only
// counts.  In the normal build BRNG_CHECK compiles to nothing.
#pragma once

#include <cuda_runtime.h>

#include <cstdint>

namespace brng {

#ifdef BRNG_DEBUG
// Registers a reader of one translation unit's count (brng_api.cu).
void register_debug_reader(unsigned long long (*read)(bool reset));

namespace {
__device__ unsigned long long g_violations;  // this translation unit's failed checks

unsigned long long read_violations(bool reset) {
  unsigned long long v = 0;
  cudaMemcpyFromSymbol(&v, g_violations, sizeof v);
  if (reset) {
    const unsigned long long zero = 0;
    cudaMemcpyToSymbol(g_violations, &zero, sizeof zero);
  }
  return v;
}

struct DebugRegistration {
  DebugRegistration() { register_debug_reader(&read_violations); }
};
const DebugRegistration g_debug_registration;
}  // namespace

#define BRNG_CHECK(cond)                                           \
  do {                                                             \
    if (!(cond)) atomicAdd(&::brng::g_violations, 1ull);           \
  } while (0)
#else
#define BRNG_CHECK(cond) \
  do {                   \
  } while (0)
#endif

}  // namespace brng
