// ptf_grid.h -- grid sizing of the persistent (refill) kernels, host only.
//
// A persistent kernel launches as many 128-thread blocks as fit on the device
// at once: the SM count of the device times the kernel's resident blocks per
// SM.  The latter is looked up once per kernel and device (it depends on the
// kernel's registers and shared memory and on the device), and the grid is
// formed on every call from the SM count of the device the call runs on.
#pragma once
#include <atomic>

namespace ptf {

constexpr int kGridMaxDevices = 64;

// Per-device cache of one kernel's resident blocks per SM (K: the kernel, so
// that kernels of the same signature keep separate entries).  `lookup`
// returns the count on the current device; devices outside [0, kGridMaxDevices)
// are looked up every time.
template <auto K>
struct BlocksPerSM {
    static std::atomic<int> cached[kGridMaxDevices];

    template <class F>
    static int get(int dev, F&& lookup) {
        if (dev < 0 || dev >= kGridMaxDevices) return clamp(lookup());
        int b = cached[dev].load(std::memory_order_relaxed);
        if (b <= 0) {
            b = clamp(lookup());
            cached[dev].store(b, std::memory_order_relaxed);  // racing callers store the same value
        }
        return b;
    }
    static int clamp(int b) { return b > 0 ? b : 1; }
};
template <auto K>
std::atomic<int> BlocksPerSM<K>::cached[kGridMaxDevices];

// Blocks of a persistent launch on a device with `sms` SMs.
inline int persistent_blocks(int sms, int per_sm) { return (sms > 0 ? sms : 1) * (per_sm > 0 ? per_sm : 1); }

}  // namespace ptf
