// wait.cuh -- bounded device-side waits.  Every spin in this library's
// kernels is limited by elapsed time read from the %globaltimer register
// (nanoseconds), never by an unbounded loop: a wait that runs out records a
// status word that the host reads (ht_device_status returns HT_ETIMEOUT) and
// the kernel returns.
#pragma once
#include <stdint.h>

namespace htgb {

__device__ __forceinline__ uint64_t globaltimer_ns() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// Longest time one device-side wait of a library kernel may take before it
// gives up: 200 ms (the waits it bounds normally end within microseconds).
constexpr int64_t kWaitLimitNs = 200ll * 1000 * 1000;

}  // namespace htgb
