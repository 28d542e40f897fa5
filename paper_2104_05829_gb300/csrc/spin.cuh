// Bounded spin-wait shared by the one-launch coarse solves.
#pragma once

namespace sem {

// Wait until *v >= target, at most about a second of SM clock (2^31 cycles); then
// raise the error flag. The flag is re-read every 64 polls, so a wait that another
// block has given up on ends too.
__device__ __forceinline__ void wait_at_least(const unsigned* v, unsigned target, int* err) {
  const long long t0 = clock64();
  unsigned polls = 0;
  while (*(const volatile unsigned*)v < target) {
    if ((++polls & 63u) == 0) {
      if (*(volatile int*)err != 0) return;
      if (clock64() - t0 > (1ll << 31)) {
        atomicExch(err, 1);
        return;
      }
    }
  }
}

}  // namespace sem
