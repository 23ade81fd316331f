// Host-side check of the run-major shared-memory layout of the slab
// (slab.cuh): for every cells-per-thread CPT and CTA size, with the run
// stride P that slab_run_stride returns, cell i sits at slot
// k * P + r, r = (i + RO*CPT) / CPT, k = (i + RO*CPT) mod CPT, and
//  1. every cell from -RO*CPT to (threads + 2)*CPT - 1 (the left ghost runs,
//     the threads' runs and the two spare runs on the right that the window
//     passes may touch) has its own slot inside the extent CPT * P that
//     slab_smem_bytes sizes (three arrays of it plus the reduction words);
//  2. the interleaved writes of one warp, 32 consecutive cells starting at a
//     multiple of 32, hit 32 distinct banks (FP32, one word per bank), or,
//     for FP64, the 16 cells of each half-warp hit 16 distinct bank pairs;
//  3. lane t reading element m of its own run touches slot base + t: the
//     window reads of consecutive lanes are consecutive words.
// Prints one line per failure and exits 1 if there is any.
#include <cstdio>
#include <set>

#include "../paper_2104_09404_gb300/csrc/slab.cuh"

using namespace mgrit;

static int failures = 0;

template <typename R>
static void check(int cpt, int threads)
{
    const int P = sizeof(R) == 4 ? slab_run_stride<float>(cpt, 512) : slab_run_stride<double>(cpt, threads);
    const int RO = cpt >= 4 ? 1 : 2;
    const long long extent = (long long)cpt * P;
    auto slot = [&](long long i) {
        const long long v = i + RO * cpt;
        return (v % cpt) * P + v / cpt;
    };
    const char *name = sizeof(R) == 4 ? "fp32" : "fp64";
    // 1. distinct slots inside the extent, and the byte count
    std::set<long long> seen;
    for (long long i = -RO * cpt; i < (long long)(threads + 2) * cpt; ++i) {
        const long long s = slot(i);
        if (s < 0 || s >= extent || !seen.insert(s).second) {
            std::printf("%s cpt %d threads %d: cell %lld -> slot %lld (extent %lld)\n", name, cpt, threads, i,
                        s, extent);
            ++failures;
            return;
        }
    }
    const size_t bytes = slab_smem_bytes<R>(threads * cpt, cpt, threads);
    if (bytes != sizeof(R) * (3 * (size_t)extent + NWARP_MAX)) {
        std::printf("%s cpt %d threads %d: slab_smem_bytes %zu\n", name, cpt, threads, bytes);
        ++failures;
    }
    // 2. banks of a warp's interleaved writes (cells t + c*threads)
    for (int c = 0; c < cpt; ++c)
        for (int w = 0; w < threads / 32; ++w) {
            const long long i0 = (long long)c * threads + 32 * w;
            if (sizeof(R) == 4) {
                std::set<long long> banks;
                for (int l = 0; l < 32; ++l) banks.insert(slot(i0 + l) % 32);
                if (banks.size() != 32) {
                    std::printf("fp32 cpt %d threads %d: cells %lld..%lld on %zu banks\n", cpt, threads, i0,
                                i0 + 31, banks.size());
                    ++failures;
                    return;
                }
            } else {
                for (int h = 0; h < 2; ++h) {
                    std::set<long long> pairs;
                    for (int l = 16 * h; l < 16 * h + 16; ++l) pairs.insert(slot(i0 + l) % 16);
                    if (pairs.size() != 16) {
                        std::printf("fp64 cpt %d threads %d: cells %lld.. on %zu bank pairs\n", cpt, threads,
                                    i0 + 16 * h, pairs.size());
                        ++failures;
                        return;
                    }
                }
            }
        }
    // 3. element m of the runs of consecutive lanes: consecutive slots
    for (int m = -RO * cpt; m < 2 * cpt; ++m)
        for (int t = 0; t + 1 < threads; ++t)
            if (slot((long long)(t + 1) * cpt + m) != slot((long long)t * cpt + m) + 1) {
                std::printf("%s cpt %d threads %d: element %d of runs %d, %d not adjacent\n", name, cpt, threads,
                            m, t, t + 1);
                ++failures;
                return;
            }
}

int main()
{
    int configs = 0;
    for (int cpt = 2; cpt <= 32; cpt *= 2)
        for (int threads = 32; threads <= 512; threads += 32) {
            check<float>(cpt, threads);
            if (cpt <= 16) check<double>(cpt, threads);   // FP64 slabs hold at most 16 cells per thread
            ++configs;
        }
    std::printf("%d configurations, %d failures\n", configs, failures);
    return failures ? 1 : 0;
}
