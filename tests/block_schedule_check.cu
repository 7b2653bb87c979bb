// Host-side check of the block kernel's phase-1 schedule (built and run by
// test_block_schedule.py; no GPU needed).  For every storage type, window
// radius and tile shape (KS = radius + 16 shape, + 32 for the persistent
// kernel's thread count) it walks the phase-1 loop pixel by pixel, in the row order
// the kernel uses, and checks that
//   * each pixel reads staged rows inside the staged box, and only rows of
//     TMA bands the loop has waited for by then (the waits happen before the
//     iterations first_iter_of_band / first_iter_of_band_up name);
//   * the chosen row order leaves no more shared-memory bank conflicts on
//     the staged taps (zero flow) than the other order would.
// Prints one line per case and "FAIL" on any violation.
#include <cstdio>
#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include "k_block.cuh"

using namespace ofv;

// Extra shared-memory wavefronts of one warp-wide load of the staged tap at
// product pixel (ry, rx), summed over the warps of the loop.
template <typename T, int KS>
static long tap_conflicts(bool up)
{
    using BS = BlockShape<KS>;
    constexpr int NT = BS::NT, RW = BS::RW, SP = StageShape<T, KS>::SP;
    long extra = 0;
    for (int base = 0; base < RW * RW; base += 32) {
        long word[32];
        int n = 0;
        for (int l = 0; l < 32 && base + l < RW * RW; ++l) {
            const int idx = base + l;
            const int ry = up ? RW - 1 - idx / RW : idx / RW, rx = idx % RW;
            word[n++] = ((long)ry * SP + rx) * (long)sizeof(T) / 4;
        }
        int worst = 1;
        for (int b = 0; b < 32; ++b) {
            long seen[32];
            int k = 0;
            for (int l = 0; l < n; ++l) {
                if (word[l] % 32 != b) continue;
                bool dup = false;
                for (int m = 0; m < k; ++m) dup |= seen[m] == word[l];
                if (!dup) seen[k++] = word[l];
            }
            if (k > worst) worst = k;
        }
        extra += worst - 1;
    }
    (void)NT;
    return extra;
}

template <typename T, int KS>
static int check(const char *tname)
{
    using BS = BlockShape<KS>;
    using SS = StageShape<T, KS>;
    using RO = RowOrder<T, KS>;
    constexpr int NT = BS::NT, RW = BS::RW, SHB = SS::SHB, SLACK = RO::slack;
    constexpr bool UP = RO::bottom_up;
    constexpr int I1 = first_iter_of_band<KS, SHB>(1), I2 = first_iter_of_band<KS, SHB>(2);
    constexpr int J1 = first_iter_of_band_up<KS, SHB, SLACK>(1), J0 = first_iter_of_band_up<KS, SHB, SLACK>(0);
    int bad = 0;
    for (int idx = 0; idx < RW * RW; ++idx) {
        const int i = idx / NT;  // loop iteration of the pixel
        bool landed[3];
        if (UP) {
            landed[2] = true;
            landed[1] = i >= J1;
            landed[0] = i >= J0;
        } else {
            landed[0] = true;
            landed[1] = i >= I1;
            landed[2] = i >= I2;
        }
        const int ry = UP ? RW - 1 - idx / RW : idx / RW;
        // product row ry reads staged rows ry + SLACK .. ry + SLACK + 2 REACH + 3
        const int lo = ry + SLACK, hi = ry + SLACK + 2 * kBlockReach + 3;
        if (lo < 0 || hi >= SS::SHT) ++bad;
        for (int r = lo; r <= hi && r >= 0 && r < SS::SHT; ++r)
            if (!landed[r / SHB]) ++bad;
    }
    const long mine = tap_conflicts<T, KS>(UP), other = tap_conflicts<T, KS>(!UP);
    const bool order_ok = mine <= other;
    printf("%s KR %2d edge %2d NT %4d SP %3d order %s slack %d unlanded/out-of-box reads %d conflicts %ld (other "
           "order %ld)%s\n",
           tname, BS::R, BS::TS, NT, SS::SP, UP ? "up  " : "down", SLACK, bad, mine, other,
           bad || !order_ok ? " FAIL" : "");
    return bad || !order_ok;
}

template <typename T>
static int all(const char *n)
{
    return check<T, 1>(n) + check<T, 2>(n) + check<T, 3>(n) + check<T, 4>(n) + check<T, 5>(n) + check<T, 6>(n) +
           check<T, 7>(n) + check<T, 8>(n) + check<T, 9>(n) + check<T, 10>(n) + check<T, 17>(n) +
           check<T, 18>(n) + check<T, 19>(n) + check<T, 20>(n) + check<T, 21>(n) + check<T, 22>(n) +
           check<T, 23>(n) + check<T, 24>(n) + check<T, 25>(n) + check<T, 26>(n) +
           // the persistent kernel's forms of the 48-px tiles (512 threads)
           check<T, 33>(n) + check<T, 34>(n) + check<T, 35>(n) + check<T, 36>(n) + check<T, 37>(n);
}

int main()
{
    const int fails = all<float>("f32 ") + all<__half>("f16 ") + all<__nv_bfloat16>("bf16");
    printf("%d failing cases\n", fails);
    return fails != 0;
}
