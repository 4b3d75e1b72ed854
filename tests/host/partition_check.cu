// Host-side checks of the binning partition (common.cuh): every launch covers
// its vortices, stays within the histogram rows it was sized for, switches to
// the 1024-thread blocks exactly at BIN_WIDE_MIN, and a captured launch sized
// for a capacity still covers every smaller device count with the span the
// device computes from that count (bin_count).  Runs on the CPU only.
#include <cstdio>
#include <cstdint>

#include "common.cuh"

static int failures = 0;
#define CHECK(cond, ...)                                   \
    do {                                                   \
        if (!(cond)) {                                     \
            ++failures;                                    \
            if (failures < 20) {                           \
                std::printf("FAIL %s: ", #cond);           \
                std::printf(__VA_ARGS__);                  \
                std::printf("\n");                         \
            }                                              \
        }                                                  \
    } while (0)

// the device-side span of bin_count for a count read on the device
static int64_t device_span(int64_t n, int min_span, int max_blocks) {
    const int64_t s = (n + max_blocks - 1) / max_blocks;
    return s < min_span ? min_span : s;
}

int main() {
    const int spans[] = {256, 512, 1024, 2048, 4096};
    const int64_t counts[] = {1, 2, 255, 256, 257, 1023, 1024, 1025, 4096, 65536, 100000, 622591, 622592, 622593,
                              1000000, 4000000, (int64_t)1 << 29};
    for (int ms : spans)
        for (int64_t nv : counts) {
            const int mb = bin_max_blocks(nv);
            const int nb = bin_blocks(nv, ms);
            const int64_t span = bin_span(nv, ms);
            CHECK(mb == (nv >= BIN_WIDE_MIN ? BIN_WIDE_BLOCKS : BIN_MAX_BLOCKS), "nv %lld", (long long)nv);
            CHECK(nb >= 1 && nb <= mb, "nv %lld ms %d nb %d", (long long)nv, ms, nb);
            CHECK(span >= ms, "nv %lld ms %d span %lld", (long long)nv, ms, (long long)span);
            CHECK((int64_t)nb * span >= nv && (int64_t)(nb - 1) * span < nv, "nv %lld ms %d", (long long)nv, ms);
            // a launch sized for capacity nv, replayed at any count n <= nv
            for (int64_t n : {(int64_t)1, nv / 3 + 1, nv / 2 + 1, nv - 1 > 0 ? nv - 1 : 1, nv}) {
                const int64_t ds = device_span(n, ms, mb);
                CHECK((n + ds - 1) / ds <= nb, "capacity %lld count %lld ms %d", (long long)nv, (long long)n, ms);
            }
        }
    CHECK(bin_blocks(0) == 0, "empty set");
    CHECK(BIN_WIDE_BLOCKS * 4 == BIN_MAX_BLOCKS, "one 1024-thread block for four 256-thread ones");
    if (failures) {
        std::printf("%d failures\n", failures);
        return 1;
    }
    std::printf("OK\n");
    return 0;
}
