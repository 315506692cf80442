// Bounded device-side waits.
//
// Every spin of the library's kernels -- on a release flag, an epoch-tagged
// word or an mbarrier -- is limited in wall-clock time, read from the
// %globaltimer nanosecond clock.  A wait that runs out records
// GBEM_ERR_TIMEOUT in a status word that the host reads, and its kernel
// returns, so a dependency that never arrives leaves the context usable
// instead of hanging the GPU.
//
// Two limits:
//   kDependencyNs  results of other CTAs (flags, tagged words): 1 s, far
//                  beyond any legitimate wait (microseconds);
//   kOwnAsyncNs    the CTA's own bulk copies and tensor-core operations,
//                  which complete by themselves: 2 s.  A CTA gives up on
//                  those only if the device itself is broken, so that a
//                  give-up path never releases shared or tensor memory under
//                  an operation that is still in flight.
#pragma once

#include <cstdint>

namespace bw {

constexpr uint64_t kDependencyNs = 1000000000ull;
constexpr uint64_t kOwnAsyncNs = 2000000000ull;

__device__ __forceinline__ uint64_t now_ns()
{
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// A wall-clock budget for one wait.  expired() reads the clock on every 32nd
// call only (the first reading starts the budget), so a fast poll loop pays
// almost nothing for it.
struct Deadline {
    uint64_t limit;
    uint64_t t0 = 0;
    unsigned calls = 0;
    __device__ __forceinline__ explicit Deadline(uint64_t limit_ns) : limit(limit_ns) {}
    __device__ __forceinline__ bool expired()
    {
        if ((++calls & 31u) != 0) return false;
        const uint64_t t = now_ns();
        if (t0 == 0) {
            t0 = t;
            return false;
        }
        return t - t0 > limit;
    }
};

}  // namespace bw
