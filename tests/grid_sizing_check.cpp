// Host-only check of the persistent-grid sizing (csrc/ptf_grid.h): the
// resident blocks per SM are cached per kernel and per device, and the grid
// is formed per call from the calling device's SM count.  Built and run by
// tests/test_grid_sizing.py with the host compiler (no GPU).
#include <cstdio>
#include "ptf_grid.h"

static void kernel_a() {}
static void kernel_b() {}

static int fails = 0;
#define CHECK(c)                                              \
    do {                                                      \
        if (!(c)) {                                           \
            std::printf("FAIL line %d: %s\n", __LINE__, #c);  \
            fails++;                                          \
        }                                                     \
    } while (0)

int main() {
    using ptf::BlocksPerSM;
    using ptf::persistent_blocks;
    int lookups = 0;
    // device 0 fits 3 blocks per SM of kernel_a, device 1 only 2
    auto occ = [&](int v) { return [&lookups, v] { lookups++; return v; }; };
    CHECK(BlocksPerSM<&kernel_a>::get(0, occ(3)) == 3);
    CHECK(BlocksPerSM<&kernel_a>::get(1, occ(2)) == 2);
    // cached: a later lookup on either device is not made again
    CHECK(BlocksPerSM<&kernel_a>::get(0, occ(7)) == 3);
    CHECK(BlocksPerSM<&kernel_a>::get(1, occ(7)) == 2);
    CHECK(lookups == 2);
    // another kernel of the same signature keeps its own entry
    CHECK(BlocksPerSM<&kernel_b>::get(0, occ(4)) == 4);
    CHECK(BlocksPerSM<&kernel_a>::get(0, occ(7)) == 3);
    // a failed lookup (0) counts as one block per SM; out-of-range devices are not cached
    CHECK(BlocksPerSM<&kernel_b>::get(5, occ(0)) == 1);
    CHECK(BlocksPerSM<&kernel_b>::get(-1, occ(6)) == 6);
    CHECK(BlocksPerSM<&kernel_b>::get(-1, occ(5)) == 5);
    CHECK(BlocksPerSM<&kernel_b>::get(ptf::kGridMaxDevices, occ(2)) == 2);
    // grids follow the SM count of each call
    CHECK(persistent_blocks(152, 3) == 456);
    CHECK(persistent_blocks(148, 3) == 444);
    CHECK(persistent_blocks(152, BlocksPerSM<&kernel_a>::get(1, occ(9))) == 304);
    CHECK(persistent_blocks(0, 0) == 1);
    if (fails == 0) std::printf("grid sizing ok\n");
    return fails == 0 ? 0 : 1;
}
