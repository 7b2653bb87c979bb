// Block-tiled fused Gauss-Newton iteration (Sec. 2 step 3, Eq. 2), the
// kernel behind OFV_PATH_FUSED for window radii 1..10.
//
// One CTA owns a TS x TS tile of output pixels (by default 48 px for
// KR <= 5 and 64 for KR 6..10; see block_tile_edge) and works
// entirely on chip in five phases:
//   0. stage the two level images over the tile, its KR window halo, a
//      REACH px warp margin and the gradient stencil into shared memory:
//      a tile whose staged box lies inside the image takes TMA tensor
//      copies (cp.async.bulk.tensor) in three row bands, each completing on
//      its own mbarrier, when the launch carries tensor maps -- phase 1
//      waits for a band only when it reaches rows that need it; otherwise
//      16-byte cp.async rows, with clamp-to-edge applied element by element
//      at the image border;
//   1. the five products of every pixel of tile + halo (bilinear value and
//      central-difference gradient of both frames at k -/+ V0/2) into
//      shared memory; pixels whose warp reaches farther than REACH px are
//      recomputed from global memory after the loop, which keeps the loop
//      free of branches;
//   2. horizontal window sums, in place, one (row, channel) per thread;
//   3. vertical window sums, in place, one (column, channel) per thread;
//   4. the guarded 2x2 solve per output pixel and the store of V.
// Window sums use the van Herk / Gil-Werman block decomposition (suffix sums
// of one block of 2KR+1 values plus prefix sums of the next), so every sum
// is formed by additions only -- no running subtraction that would cancel
// digits the ill-conditioned solves need -- at three additions per output.
// Products of pixels outside the image are zero, which truncates the
// windows at the border.
#pragma once
#include <cuda.h>  // CUtensorMap (the type only; maps are encoded on the host)

#include "iter_math.cuh"

namespace ofv {

constexpr int kBlockReach = 4;  // |warp offset| served from the staged tile (px)
constexpr int kBlockMaxKR = 10;
constexpr int kBlockMaxBatch = kMaxPairsPerLaunch;

struct BlockParams {
    IterArgs a[kBlockMaxBatch];  // one per pair (blockIdx.z)
    int mode;                    // V0Mode, uniform per launch
    int use_tma;                 // 1: tm[k] maps the two level images of pair k
    int *err;                    // error word (set to 1 when a TMA wait expires), or null
    int by0;                     // first tile row of the launch (blockIdx.y + by0)
    CUtensorMap tm[kBlockMaxBatch][2];
};

// The block kernels' templates take KS = KR + 16 V + 32 Q: the window radius
// KR (1 .. 10), the tile shape V (0: the default shape of the radius, 1: its
// alternative, which the batched autotuner tries and ofv_params.tile_edge
// selects) and Q = 1 for the persistent batched kernel, which runs 48-px
// tiles with 512 threads instead of 576 (its queue state leaves fewer
// registers: 576 threads spill there, +3.2 % with 512).  Each output pixel
// is computed by the same tile with the same arithmetic whatever the thread
// count, so the two kernels give the same fields.
__host__ __device__ constexpr int ks_radius(int ks) { return ks & 15; }
__host__ __device__ constexpr int ks_shape(int ks) { return (ks >> 4) & 1; }
__host__ __device__ constexpr int ks_queue(int ks) { return ks >> 5; }

// Output tile edge of shape v for radius kr.  Default shapes, measured per
// radius (1 Mp stream, fields/s): KR <= 5: 48-px tiles of 576 threads, two
// CTAs per SM, 56 registers (512 threads: -2 %; 640: no gain, 48 registers
// and spills; 64-px tiles at one CTA per SM: -15..-18 %); KR 6..10: 64-px
// tiles, one CTA of 1024 threads per SM (less halo work: +21..26 % against
// 32 or 48 px at KR 7..10, +13.5 % against 32 px at KR 6; 1024 threads
// instead of 512: +13 % at KR 10).  Alternative: 32-px tiles of 256 threads.
__host__ __device__ constexpr int block_tile_edge(int kr, int v)
{
    return v == 0 ? (kr <= 5 ? 48 : 64) : 32;
}

template <int KS> struct BlockShape {
    static constexpr int R = ks_radius(KS);                // window radius
    static constexpr int TS = block_tile_edge(R, ks_shape(KS));  // output tile edge
    static constexpr int NT = TS == 32 ? 256 : TS == 48 ? (ks_queue(KS) ? 512 : 576) : 1024;  // threads
    // resident CTAs per SM (shared memory)
    static constexpr int MINB = TS == 32 ? (R <= 5 ? 3 : 2) : TS == 48 ? 2 : 1;
    static constexpr int RW = TS + 2 * R;                 // product region edge
    static constexpr int RWP = RW | 1;                    // odd row pitch of the product planes
    static constexpr int SH = RW + 2 * kBlockReach + 3;   // staged rows
};

// Rows of one TMA band: at least a third of the staged rows, and a whole
// number of 128-byte units so that every band starts 128-byte aligned.
__host__ __device__ constexpr int band_rows(int rows, int row_bytes)
{
    int b = (rows + 2) / 3;
    while ((b * row_bytes) % 128 != 0) ++b;
    return b;
}

// Phase 1 gives consecutive lanes consecutive pixels of a product row; a
// warp that runs past the end of a row goes on in the next row it visits.
// Against a run of consecutive addresses its staged taps then jump by
// SP - RW elements (rows visited top down) or by -(SP + RW) (bottom up).
// The warp's loads stay on distinct banks when the jump is a whole number
// of 32-bit words whose residue modulo the 32 banks keeps the two runs
// apart (32 elements cover 8 sizeof(T) words).
template <typename T>
__host__ __device__ constexpr bool bank_clean_jump(int shift)
{
    return (shift * (int)sizeof(T)) % 4 == 0 &&
           (((shift * (int)sizeof(T) / 4) % 32 + 32) % 32) <= 32 - 8 * (int)sizeof(T);
}

template <typename T, int KR> struct StageShape {
    static constexpr int VEC = 16 / (int)sizeof(T);
    static constexpr int SW = BlockShape<KR>::RW + 2 * kBlockReach + 3 + VEC - 1;  // incl. alignment slack
    static constexpr int NV = (SW + VEC - 1) / VEC;                               // 16-byte vectors per row
    static constexpr int SP = NV * VEC;                                           // staged row pitch
    // staged rows: three bands of SHB rows, at least the SH rows the tile needs
    static constexpr int NBAND = 3;
    static constexpr int SHB = band_rows(BlockShape<KR>::SH, SP * (int)sizeof(T));
    static constexpr int SHT = NBAND * SHB;
    // elements per staged frame, rounded so the second frame starts 128-byte aligned
    static constexpr int STG = (SHT * SP * (int)sizeof(T) + 127) / 128 * 128 / (int)sizeof(T);
};

// Order of the product rows in phase 1: bottom up where only that order
// keeps the row jumps bank-clean (FP32 staging at KR 4: SP 72, RW 56).
// Bottom up, the staged box starts `slack` rows higher (the rows by which
// the three bands exceed the SH rows the tile reads), so that the last band
// is full and the first iterations need it alone.
template <typename T, int KR> struct RowOrder {
    static constexpr int SP = StageShape<T, KR>::SP, RW = BlockShape<KR>::RW;
    static constexpr bool bottom_up = !bank_clean_jump<T>(SP - RW) && bank_clean_jump<T>(-(SP + RW));
    static constexpr int slack = bottom_up ? StageShape<T, KR>::SHT - BlockShape<KR>::SH : 0;
};

// floats of the five product planes, rounded up so the staged images that
// follow start 128-byte aligned (TMA destinations)
template <int KR> struct ProdFloats {
    static constexpr int v = (5 * BlockShape<KR>::RW * BlockShape<KR>::RWP + 31) / 32 * 32;
};

template <typename T, int KR>
constexpr size_t block_smem_bytes()
{
    return sizeof(float) * ProdFloats<KR>::v + sizeof(T) * 2 * StageShape<T, KR>::STG;
}

__device__ __forceinline__ void cp_async16(void *smem, const void *gmem)
{
    const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(s), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_wait_all()
{
    asm volatile("cp.async.commit_group;\ncp.async.wait_group 0;\n" ::: "memory");
}

__device__ __forceinline__ long long global_ns()
{
    long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// mbarrier and TMA (bulk tensor copy) primitives, CTA scope.
__device__ __forceinline__ unsigned smem_u32(const void *p) { return (unsigned)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint64_t *bar, unsigned count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t *bar, unsigned bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes) : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, unsigned parity)
{
    unsigned ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}

// 2-D tiled copy of the box at element (x, y) of the tensor map into shared
// memory; x * sizeof(element) must be a multiple of 16 bytes.
__device__ __forceinline__ void tma_load_2d(void *dst, const CUtensorMap *tm, int x, int y, uint64_t *bar)
{
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];"
        ::"r"(smem_u32(dst)), "l"(reinterpret_cast<uint64_t>(tm)), "r"(x), "r"(y), "r"(smem_u32(bar))
        : "memory");
}

// Wait for phase `parity` of the barrier, at most ~timeout_ns.
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t *bar, unsigned parity, long long timeout_ns)
{
    if (mbar_try_wait(bar, parity)) return true;
    const long long t0 = global_ns();
    for (int i = 0; i < (1 << 22); ++i) {
        if (mbar_try_wait(bar, parity)) return true;
        if ((i & 63) == 63 && global_ns() - t0 > timeout_ns) return false;
    }
    return false;
}

// Field load: through the read-only cache, or -- when the field was written
// earlier in the same launch by other CTAs (persistent batched kernel) --
// from L2 only, so no stale L1 line is read.
template <bool COH>
__device__ __forceinline__ float2 ld_field(const float2 *p)
{
    return COH ? __ldcg(p) : __ldg(p);
}

// V0 at (x, y) with the mode chosen at run time (uniform per launch):
// zero, the same-level field, or 2 * bilinear(coarse field, x/2, y/2).
template <bool COH>
__device__ __forceinline__ float2 fetch_v0_rt(const IterArgs &a, int mode, int x, int y)
{
    if (mode == V0_SAME) return ld_field<COH>(a.V0 + (int64_t)y * a.vpitch + x);
    if (mode == V0_UP) {
        const int cx = x >> 1, cy = y >> 1;
        const float fx = (x & 1) ? 0.5f : 0.f, fy = (y & 1) ? 0.5f : 0.f;
        const int cx1 = min(cx + 1, a.Wc - 1), cy1 = min(cy + 1, a.Hc - 1);
        const int cxa = min(cx, a.Wc - 1), cya = min(cy, a.Hc - 1);
        const float2 v00 = ld_field<COH>(a.Vc + (int64_t)cya * a.vcpitch + cxa);
        const float2 v01 = ld_field<COH>(a.Vc + (int64_t)cya * a.vcpitch + cx1);
        const float2 v10 = ld_field<COH>(a.Vc + (int64_t)cy1 * a.vcpitch + cxa);
        const float2 v11 = ld_field<COH>(a.Vc + (int64_t)cy1 * a.vcpitch + cx1);
        const float wx0 = 1.f - fx, wy0 = 1.f - fy;
        float2 r;
        r.x = 2.f * (wy0 * (wx0 * v00.x + fx * v01.x) + fy * (wx0 * v10.x + fx * v11.x));
        r.y = 2.f * (wy0 * (wx0 * v00.y + fx * v01.y) + fy * (wx0 * v10.y + fx * v11.y));
        return r;
    }
    return make_float2(0.f, 0.f);
}

// V0 with the mode fixed at compile time, for pixels inside the image.
template <bool COH, int MODE>
__device__ __forceinline__ float2 fetch_v0_ct(const IterArgs &a, int x, int y)
{
    if (MODE == V0_ZERO) return make_float2(0.f, 0.f);
    return fetch_v0_rt<COH>(a, MODE, x, y);
}

// Global-memory sampler for warps beyond the staged margin (rare).
template <typename T>
__device__ __noinline__ Sample sample_global(const T *__restrict__ P, int H, int W, int pitch, int x, int y, float dx,
                                             float dy)
{
    return sample_level(P, H, W, pitch, x, y, dx, dy);
}

// Bilinear value and gradient of a level image at (x + dx, y + dy), from the
// staged tile when the border-remapped taps lie within REACH px of (x, y).
// st points at staged element (row sy0, column sx0).  Same arithmetic as
// sample_level.
template <typename T, int SP>
__device__ __forceinline__ Sample sample_staged(const T *__restrict__ st, int sx0, int sy0, const T *__restrict__ Pg,
                                                int H, int W, int pitch, int x, int y, float dx, float dy)
{
    const float lim_x = (float)(W + 4), lim_y = (float)(H + 4);
    const float cdx = fminf(fmaxf(dx, -lim_x), lim_x);
    const float cdy = fminf(fmaxf(dy, -lim_y), lim_y);
    const float flx = floorf(cdx), fly = floorf(cdy);
    float fx = cdx - flx, fy = cdy - fly;
    int x0 = x + (int)flx, y0 = y + (int)fly;
    if (x0 < 0) { x0 = 0; fx = 0.f; }
    if (x0 > W - 2) { x0 = W - 2; fx = 1.f; }
    if (y0 < 0) { y0 = 0; fy = 0.f; }
    if (y0 > H - 2) { y0 = H - 2; fy = 1.f; }
    if (abs(x0 - x) > kBlockReach || abs(y0 - y) > kBlockReach) return sample_global(Pg, H, W, pitch, x, y, dx, dy);
    const T *rm = st + (y0 - 1 - sy0) * SP + (x0 - 1 - sx0);
    const T *r0 = rm + SP, *r1 = rm + 2 * SP, *rp = rm + 3 * SP;
    const float e0 = to_f(rm[1]), e1 = to_f(rm[2]);
    const float q00 = to_f(r0[0]), q01 = to_f(r0[1]), q02 = to_f(r0[2]), q03 = to_f(r0[3]);
    const float q10 = to_f(r1[0]), q11 = to_f(r1[1]), q12 = to_f(r1[2]), q13 = to_f(r1[3]);
    const float e2 = to_f(rp[1]), e3 = to_f(rp[2]);
    const float wx0 = 1.f - fx, wy0 = 1.f - fy;
    Sample s;
    s.val = wy0 * (wx0 * q01 + fx * q02) + fy * (wx0 * q11 + fx * q12);
    const float dxa0 = 0.5f * (q02 - q00), dxb0 = 0.5f * (q03 - q01);
    const float dxa1 = 0.5f * (q12 - q10), dxb1 = 0.5f * (q13 - q11);
    s.gx = wy0 * (wx0 * dxa0 + fx * dxb0) + fy * (wx0 * dxa1 + fx * dxb1);
    const float dya0 = 0.5f * (q11 - e0), dyb0 = 0.5f * (q12 - e1);
    const float dya1 = 0.5f * (e2 - q01), dyb1 = 0.5f * (e3 - q02);
    s.gy = wy0 * (wx0 * dya0 + fx * dyb0) + fy * (wx0 * dya1 + fx * dyb1);
    return s;
}

// Packed FP32 (two lanes per instruction, each lane rounded as the scalar
// operation): lane x carries frame 1, lane y frame 2.
__device__ __forceinline__ float2 fma2(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }
__device__ __forceinline__ float2 sub2(float2 a, float2 b)
{
    return __ffma2_rn(b, make_float2(-1.f, -1.f), a);  // b * -1 is exact: one rounding, as a - b
}

struct Sample2 { float2 val, gx, gy; };

// Bilinear value and doubled gradient (undivided central differences) of a
// staged 4x4 neighbourhood, for the two frames at once: rm1, rm2 point at
// the tap left of column x0 in row y0-1 of each frame's staged tile; f_x,
// f_y hold each frame's fractions.  Interpolation as a + f (b - a); the
// row interpolation of the column differences equals the difference of row
// interpolations (gy).  Each lane rounds as the scalar operations would.
template <typename T, int SP>
__device__ __forceinline__ Sample2 bilin_staged2(const T *__restrict__ rm1, const T *__restrict__ rm2, float2 f_x,
                                                 float2 f_y)
{
    auto ld2 = [&](int off) { return make_float2(to_f(rm1[off]), to_f(rm2[off])); };
    const float2 e0 = ld2(1), e1 = ld2(2);
    const float2 q00 = ld2(SP), q01 = ld2(SP + 1), q02 = ld2(SP + 2), q03 = ld2(SP + 3);
    const float2 q10 = ld2(2 * SP), q11 = ld2(2 * SP + 1), q12 = ld2(2 * SP + 2), q13 = ld2(2 * SP + 3);
    const float2 e2 = ld2(3 * SP + 1), e3 = ld2(3 * SP + 2);
    Sample2 s;
    const float2 v0 = fma2(f_x, sub2(q02, q01), q01), v1 = fma2(f_x, sub2(q12, q11), q11);
    s.val = fma2(f_y, sub2(v1, v0), v0);
    const float2 da0 = sub2(q02, q00), db0 = sub2(q03, q01), da1 = sub2(q12, q10), db1 = sub2(q13, q11);
    const float2 gx0 = fma2(f_x, sub2(db0, da0), da0), gx1 = fma2(f_x, sub2(db1, da1), da1);
    s.gx = fma2(f_y, sub2(gx1, gx0), gx0);
    const float2 vm = fma2(f_x, sub2(e1, e0), e0), vp = fma2(f_x, sub2(e3, e2), e2);
    const float2 gy0 = sub2(v1, vm), gy1 = sub2(vp, v0);
    s.gy = fma2(f_y, sub2(gy1, gy0), gy0);
    return s;
}

// Bilinear value and doubled gradient (undivided central differences) of a
// staged 4x4 neighbourhood for the two frames at once, with each
// interpolation written (1 - f) a + f b, which is exact at f = 0 and f = 1:
// a sample taken at the tap to the left with fraction 1 equals the sample at
// the next tap with fraction 0.  rm1, rm2 point at the tap left of column x0
// in row y0-1 of each frame's staged tile; w0 = 1 - f and w1 = f hold the
// two frames' weights (lane x frame 1, lane y frame 2); each lane rounds as
// the scalar operations would.
template <typename T, int SP>
__device__ __forceinline__ Sample2 bilin_weighted2(const T *__restrict__ rm1, const T *__restrict__ rm2, float2 wx0,
                                                   float2 wx1, float2 wy0, float2 wy1)
{
    auto ld2 = [&](int off) { return make_float2(to_f(rm1[off]), to_f(rm2[off])); };
    auto lerp = [](float2 w0, float2 w1, float2 a, float2 b) { return fma2(w1, b, __fmul2_rn(w0, a)); };
    const float2 e0 = ld2(1), e1 = ld2(2);
    const float2 q00 = ld2(SP), q01 = ld2(SP + 1), q02 = ld2(SP + 2), q03 = ld2(SP + 3);
    const float2 q10 = ld2(2 * SP), q11 = ld2(2 * SP + 1), q12 = ld2(2 * SP + 2), q13 = ld2(2 * SP + 3);
    const float2 e2 = ld2(3 * SP + 1), e3 = ld2(3 * SP + 2);
    Sample2 s;
    const float2 v0 = lerp(wx0, wx1, q01, q02), v1 = lerp(wx0, wx1, q11, q12);
    s.val = lerp(wy0, wy1, v0, v1);
    const float2 gx0 = lerp(wx0, wx1, sub2(q02, q00), sub2(q03, q01));
    const float2 gx1 = lerp(wx0, wx1, sub2(q12, q10), sub2(q13, q11));
    s.gx = lerp(wy0, wy1, gx0, gx1);
    const float2 vm = lerp(wx0, wx1, e0, e1), vp = lerp(wx0, wx1, e2, e3);
    s.gy = lerp(wy0, wy1, sub2(v1, vm), sub2(vp, v0));
    return s;
}

// The five products of one pixel from the staged tile: frame 2 sampled at
// integer offset (ix, iy) with fractions (fx2, fy2), frame 1 at -(ix, iy) - 1
// with fractions 1 - (fx2, fy2); base indexes the staged element left of and
// above the pixel.
template <typename T, int SP, bool VAR>
__device__ __forceinline__ void products_staged(const T *__restrict__ st1, const T *__restrict__ st2, int base, int ix,
                                                int iy, float fx2, float fy2, const IterArgs &a, float2 V0, float p[5])
{
    const int off = iy * SP + ix;
    const Sample2 s12 = bilin_weighted2<T, SP>(st1 + (base - off - SP - 1), st2 + (base + off),
                                               make_float2(fx2, 1.f - fx2), make_float2(1.f - fx2, fx2),
                                               make_float2(fy2, 1.f - fy2), make_float2(1.f - fy2, fy2));
    // doubled gradients: G = (g1 + g2) / 2 = (2 g1 + 2 g2) / 4
    const float Gx = 0.25f * (s12.gx.x + s12.gx.y);
    const float Gy = 0.25f * (s12.gy.x + s12.gy.y);
    const float It = s12.val.y - s12.val.x;
    const float r = (VAR && a.inc) ? -It : Gx * V0.x + Gy * V0.y - It;
    p[0] = Gx * Gx;
    p[1] = Gx * Gy;
    p[2] = Gy * Gy;
    p[3] = Gx * r;
    p[4] = Gy * r;
}

// Products of one pixel (x, y) of a tile whose staged region lies inside
// the image: no clamping or border remap is needed while the warp stays
// within REACH px.  Frame 2 samples at k + h with integer part (ix, iy) =
// floor(h) and fraction f; frame 1 at k - h, taken as integer part
// -(ix, iy) - 1 with fraction 1 - f, which is floor(-h) and its fraction
// unless a component of h is an integer, where the weight 1 on the next tap
// gives the same sample exactly.  Both stencils then lie within REACH + 1 px
// and one integer test checks both.  Farther warps take the general sampler.
template <typename T, int SP, bool VAR = false>
__device__ __forceinline__ void products_interior(const T *__restrict__ st1, const T *__restrict__ st2, int sx0,
                                                  int sy0, const IterArgs &a, int x, int y, float2 V0, float p[5])
{
    const float hx = 0.5f * V0.x, hy = 0.5f * V0.y;
    const float flx = floorf(hx), fly = floorf(hy);
    const int ix = (int)flx, iy = (int)fly;
    if (((unsigned)(ix + kBlockReach) | (unsigned)(iy + kBlockReach)) < (unsigned)(2 * kBlockReach)) {
        products_staged<T, SP, VAR>(st1, st2, (y - 1 - sy0) * SP + (x - 1 - sx0), ix, iy, hx - flx, hy - fly, a, V0,
                                    p);
    } else {
        const T *P1 = static_cast<const T *>(a.P1), *P2 = static_cast<const T *>(a.P2);
        const Sample s1 = sample_global(P1, a.H, a.W, a.pitch, x, y, -hx, -hy);
        const Sample s2 = sample_global(P2, a.H, a.W, a.pitch, x, y, hx, hy);
        const float Gx = 0.5f * (s1.gx + s2.gx), Gy = 0.5f * (s1.gy + s2.gy);
        const float It = s2.val - s1.val;
        const float r = (VAR && a.inc) ? -It : Gx * V0.x + Gy * V0.y - It;
        p[0] = Gx * Gx;
        p[1] = Gx * Gy;
        p[2] = Gy * Gy;
        p[3] = Gx * r;
        p[4] = Gy * r;
    }
}

// The same without the branch to the general sampler: returns false, with
// products of an in-reach stand-in offset, when the warp leaves the staged
// margin; the caller then recomputes the pixel with products_interior.
// Keeps the hot loop free of a divergent branch and a call.
template <typename T, int SP, bool VAR = false>
__device__ __forceinline__ bool products_staged_only(const T *__restrict__ st1, const T *__restrict__ st2, int sx0,
                                                     int sy0, const IterArgs &a, int x, int y, float2 V0, float p[5])
{
    const float hx = 0.5f * V0.x, hy = 0.5f * V0.y;
    const float flx = floorf(hx), fly = floorf(hy);
    const int ix = (int)flx, iy = (int)fly;
    const bool near = ((unsigned)(ix + kBlockReach) | (unsigned)(iy + kBlockReach)) < (unsigned)(2 * kBlockReach);
    products_staged<T, SP, VAR>(st1, st2, (y - 1 - sy0) * SP + (x - 1 - sx0), near ? ix : 0, near ? iy : 0, hx - flx,
                                hy - fly, a, V0, p);
    return near;
}

// Phase 1 of a tile whose staged box lies inside the image: every pixel of
// the product region is inside the image and takes the staged fast path, so
// the loop needs no bounds or border checks; the V0 mode is a template
// parameter.  V0 of the thread's next pixel is loaded one iteration ahead.
// First iteration of the phase-1 loop (pixel idx = tid + i NT of the
// RW x RW product region) that may touch staged band b: the last row of
// iteration i is (i + 1) NT - 1 over RW, and product row r reads staged rows
// r .. r + 2 REACH + 3.
template <int KR, int SHB>
__host__ __device__ constexpr int first_iter_of_band(int b)
{
    constexpr int NT = BlockShape<KR>::NT, RW = BlockShape<KR>::RW;
    int i = 0;
    while (i * NT < RW * RW && ((i + 1) * NT - 1) / RW + 2 * kBlockReach + 3 < b * SHB) ++i;
    return i;
}

// The same for rows visited bottom up (bands waited from the last to the
// first): the lowest product row of iteration i is RW - 1 - ((i + 1) NT - 1)
// over RW, and product row r reads staged rows from r + SLACK on.
template <int KR, int SHB, int SLACK>
__host__ __device__ constexpr int first_iter_of_band_up(int b)
{
    constexpr int NT = BlockShape<KR>::NT, RW = BlockShape<KR>::RW;
    int i = 0;
    while (i * NT < RW * RW && RW - 1 - ((i + 1) * NT - 1) / RW + SLACK >= (b + 1) * SHB) ++i;
    return i;
}

// With bars (TMA staging in three bands), the loop waits for band b just
// before the first iteration that can touch it, so the first rows of
// products overlap the copies of the later bands.
template <typename T, int KR, bool COH, int MODE, int SP, bool VAR>
__device__ __forceinline__ void products_tile_interior(const IterArgs &a, const T *__restrict__ st1,
                                                       const T *__restrict__ st2, int sx0, int sy0, int px0, int py0,
                                                       float *prod, uint64_t *bars, unsigned parity, int *err)
{
    using BS = BlockShape<KR>;
    using SS = StageShape<T, KR>;
    static_assert(SS::NBAND == 3, "three staging bands");
    static_assert((BS::RW * BS::RW + BS::NT - 1) / BS::NT <= 32, "one bit per pixel of a thread");
    constexpr int NT = BS::NT, RW = BS::RW, RWP = BS::RWP, PLANE = RW * RWP;
    constexpr bool UP = RowOrder<T, KR>::bottom_up;
    constexpr int DX = NT % RW, DY = UP ? -(NT / RW) : NT / RW, DW = UP ? -1 : 1;
    constexpr int I1 = first_iter_of_band<KR, SS::SHB>(1), I2 = first_iter_of_band<KR, SS::SHB>(2);
    constexpr int J1 = first_iter_of_band_up<KR, SS::SHB, RowOrder<T, KR>::slack>(1);
    constexpr int J0 = first_iter_of_band_up<KR, SS::SHB, RowOrder<T, KR>::slack>(0);
    const int tid = threadIdx.x;
    int ry = tid / RW, rx = tid - (tid / RW) * RW;
    if (UP) ry = RW - 1 - ry;
    float2 V0n = make_float2(0.f, 0.f);
    if (tid < RW * RW) V0n = fetch_v0_ct<COH, MODE>(a, px0 + rx, py0 + ry);
    auto wait_band = [&](int b) {
        if (bars && !mbar_wait_bounded(bars + b, parity, 2000000000LL)) {
            // report; the tile's results are then undefined
            if (err) atomicExch(err, 1);
            mbar_wait_bounded(bars + b, parity, 1000000000LL);
        }
    };
    unsigned far = 0, bit = 1;  // bit k: the thread's k-th pixel left the staged margin
    auto pixel = [&](int idx) {
        const float2 V0c = V0n;
        const int gx = px0 + rx, gy = py0 + ry;
        float *q = prod + ry * RWP + rx;
        rx += DX;
        ry += DY;
        if (rx >= RW) {
            rx -= RW;
            ry += DW;
        }
        if (idx + NT < RW * RW) V0n = fetch_v0_ct<COH, MODE>(a, px0 + rx, py0 + ry);
        float p[5];
        if (!products_staged_only<T, SP, VAR>(st1, st2, sx0, sy0, a, gx, gy, V0c, p)) far |= bit;
        bit <<= 1;
        if (VAR && a.mask && !__ldg(a.mask + (int64_t)gy * a.W + gx)) p[0] = p[1] = p[2] = p[3] = p[4] = 0.f;
        q[0] = p[0];
        q[PLANE] = p[1];
        q[2 * PLANE] = p[2];
        q[3 * PLANE] = p[3];
        q[4 * PLANE] = p[4];
    };
    int idx = tid;
    if (UP) {
        wait_band(2);
        for (; idx < RW * RW && idx < J1 * NT; idx += NT) pixel(idx);
        wait_band(1);
        for (; idx < RW * RW && idx < J0 * NT; idx += NT) pixel(idx);
        wait_band(0);
    } else {
        wait_band(0);
        for (; idx < RW * RW && idx < I1 * NT; idx += NT) pixel(idx);
        wait_band(1);
        for (; idx < RW * RW && idx < I2 * NT; idx += NT) pixel(idx);
        wait_band(2);
    }
    for (; idx < RW * RW; idx += NT) pixel(idx);
    // the pixels whose warp left the staged margin (rare), again with the
    // general sampler; the thread's k-th pixel is tid + k NT
    for (int k = 0; far != 0; ++k, far >>= 1) {
        if (!(far & 1u)) continue;
        const int i = tid + k * NT;
        const int py = UP ? RW - 1 - i / RW : i / RW, px = i - (i / RW) * RW;
        const int gx = px0 + px, gy = py0 + py;
        float p[5];
        products_interior<T, SP, VAR>(st1, st2, sx0, sy0, a, gx, gy, fetch_v0_ct<COH, MODE>(a, gx, gy), p);
        if (VAR && a.mask && !__ldg(a.mask + (int64_t)gy * a.W + gx)) p[0] = p[1] = p[2] = p[3] = p[4] = 0.f;
        float *q = prod + py * RWP + px;
        q[0] = p[0];
        q[PLANE] = p[1];
        q[2 * PLANE] = p[2];
        q[3 * PLANE] = p[3];
        q[4 * PLANE] = p[4];
    }
}

// Window sums of one line of the product planes, in place: for outputs
// o = 0 .. TS-1, line[o*stride] <- sum_{j=0}^{2KR} line[(o+j)*stride].
// Outputs are formed block by block (blocks of WIN = 2KR+1): the sums of a
// block are suffix sums of its own values plus prefix sums of the next 2KR
// values.  Each value is loaded once and kept in registers from the step
// that reads it as the "next" block to the step that uses it as the current
// one; a step writes only its own block's outputs, whose values are already
// in registers, so the line can be overwritten in place.
template <int KR, int TS, bool TAIL>
__device__ __forceinline__ void window_step(float *line, int stride, int b0, float (&cur)[2 * KR + 1])
{
    constexpr int WIN = 2 * KR + 1, N = TS + 2 * KR;
    float nxt[WIN];
#pragma unroll
    for (int i = 0; i < WIN; ++i) nxt[i] = (!TAIL || b0 + WIN + i < N) ? line[(b0 + WIN + i) * stride] : 0.f;
#pragma unroll
    for (int i = WIN - 2; i >= 0; --i) cur[i] += cur[i + 1];  // suffix sums
    line[b0 * stride] = cur[0];
    float pre = 0.f;
#pragma unroll
    for (int i = 1; i < WIN; ++i) {
        pre += nxt[i - 1];
        if (!TAIL || b0 + i < TS) line[(b0 + i) * stride] = cur[i] + pre;
    }
#pragma unroll
    for (int i = 0; i < WIN; ++i) cur[i] = nxt[i];
}

template <int KR, int TS>
__device__ __forceinline__ void window_sums_inplace(float *line, int stride)
{
    constexpr int WIN = 2 * KR + 1, N = TS + 2 * KR;
    constexpr int NFULL = (N - WIN) / WIN;  // steps whose next block lies wholly inside the line
    constexpr int NB = (TS + WIN - 1) / WIN;
    float cur[WIN];
#pragma unroll
    for (int i = 0; i < WIN; ++i) cur[i] = line[i * stride];
    int b = 0;
#pragma unroll 1
    for (; b < NFULL && b < NB; ++b) window_step<KR, TS, false>(line, stride, b * WIN, cur);
    for (; b < NB; ++b) window_step<KR, TS, true>(line, stride, b * WIN, cur);
}

// Weighted window sums of one line, in place (Gaussian window):
// line[o*stride] <- sum_{j=0}^{2KR} w(j - KR) line[(o+j)*stride] for
// o = 0 .. TS-1, with w(d) = wg[|d|].  The 2KR+1 values under the window sit
// in a register ring (value n in slot n mod WIN); output o is written after
// its own value was read and no later output needs it.
template <int KR, int TS>
__device__ __forceinline__ void window_wsums_inplace(float *line, int stride, const float *wg)
{
    constexpr int WIN = 2 * KR + 1;
    float ring[WIN];
#pragma unroll
    for (int i = 0; i < WIN - 1; ++i) ring[i] = line[i * stride];
#pragma unroll 1
    for (int o0 = 0; o0 < TS; o0 += WIN) {
#pragma unroll
        for (int k = 0; k < WIN; ++k) {
            if (o0 + k < TS) {
                ring[(k + WIN - 1) % WIN] = line[(o0 + k + WIN - 1) * stride];
                float acc = 0.f;
#pragma unroll
                for (int j = 0; j < WIN; ++j) acc = fmaf(wg[j < KR ? KR - j : j - KR], ring[(k + j) % WIN], acc);
                line[(o0 + k) * stride] = acc;
            }
        }
    }
}

// 1/d for the solve: the MUFU approximation (rcp.approx) refined by one
// Newton-Raphson step for the root of 1/y - d, y1 = y0 + y0 (1 - d y0), with
// no slow path.  Normal d and 1/d only (the solve reaches it with det above
// eps_rel (Sxx + Syy)^2 > 0); subnormals flush to zero.
__device__ __forceinline__ float recip_newton(float d)
{
    float y0;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(y0) : "f"(d));
    return fmaf(y0, fmaf(-d, y0, 1.f), y0);
}

// Phase 4 of the forward iteration: the guarded 2x2 solve of pixel (gx, gy)
// from its window sums S = (Sxx, Sxy, Syy, Sxr, Syr) and the store of V.
template <bool VAR>
struct SolveStoreT {
    template <bool COH>
    __device__ __forceinline__ void apply(const IterArgs &a, int mode, int gx, int gy, const float (&S)[5]) const
    {
        const float sxx = S[0], sxy = S[1], syy = S[2], sxr = S[3], syr = S[4];
        const float tr = sxx + syy;
        const float det = sxx * syy - sxy * sxy;
        float2 V;
        if (!(tr > a.eps_abs) || det <= a.eps_rel * tr * tr) {
            V = fetch_v0_rt<COH>(a, mode, gx, gy);
        } else {
            const float inv = recip_newton(det);
            V = make_float2((syy * sxr - sxy * syr) * inv, (sxx * syr - sxy * sxr) * inv);
            if (VAR && a.inc) {  // increment form: V = V0(m) + H^-1 (Sxr, Syr)
                const float2 V0 = fetch_v0_rt<COH>(a, mode, gx, gy);
                V.x += V0.x;
                V.y += V0.y;
            }
        }
        if (VAR && a.s_out) {  // reverse mode: keep the window sums for the solve adjoint
            const size_t o = (size_t)gy * a.s_pitch + gx;
#pragma unroll
            for (int c = 0; c < 5; ++c) a.s_out[c * a.s_plane + o] = S[c];
        }
        if (a.u_out) {
            if (VAR && a.mask && !__ldg(a.mask + (int64_t)gy * a.W + gx)) V = make_float2(no_vector(), no_vector());
            a.u_out[(int64_t)gy * a.W + gx] = V.x;
            a.v_out[(int64_t)gy * a.W + gx] = V.y;
        } else {
            a.Vout[(int64_t)gy * a.vpitch + gx] = V;
        }
    }
};

using SolveStore = SolveStoreT<false>;

// Phases 0-3 of one tile, then epi.apply() per output pixel (phase 4).
// VAR: the tile honours the estimator variants of a (increment form,
// Gaussian window); without it the kernel carries no code for them.
// TMA staging needs tensor maps tm1, tm2 of the two level images and NBAND
// mbarriers tma_bars (shared memory): with init_bars the tile initialises
// them (one tile per CTA), else the caller did and made them visible to the
// CTA; parity is the phase this tile's copies complete (the number of
// earlier TMA tiles of the CTA, mod 2).  Returns true when the tile was
// staged by TMA.
// Side work a caller may slot into the tile's phases: after_products(tid)
// runs after phase 1's loop and after_rows(tid) after phase 2's, each before
// the phase's closing barrier.
struct NoSide {
    __device__ __forceinline__ void after_products(int) const {}
    __device__ __forceinline__ void after_rows(int) const {}
};

template <typename T, int KR, bool COH, typename Epi = SolveStore, bool VAR = false, typename Side = NoSide>
__device__ __forceinline__ bool block_tile(const IterArgs &a, int mode, int bx, int by, float4 *smem_f4,
                                           const CUtensorMap *tm1 = nullptr, const CUtensorMap *tm2 = nullptr,
                                           int *err = nullptr, const Epi &epi = Epi(), uint64_t *tma_bars = nullptr,
                                           unsigned parity = 0, bool init_bars = false, const Side &side = Side())
{
    using BS = BlockShape<KR>;
    using SS = StageShape<T, KR>;
    constexpr int TS = BS::TS, NT = BS::NT, RW = BS::RW, RWP = BS::RWP, SH = SS::SHT;
    constexpr int SP = SS::SP, NV = SS::NV, VEC = SS::VEC, STG = SS::STG;
    constexpr int NBAND = SS::NBAND, SHB = SS::SHB;
    constexpr int PLANE = RW * RWP;

    float *prod = reinterpret_cast<float *>(smem_f4);                // [5][RW][RWP]
    T *stage = reinterpret_cast<T *>(prod + ProdFloats<KR>::v);     // [2][STG]: SH rows of SP
    uint64_t *bars = nullptr;                                      // set when staged by TMA

    const int tid = threadIdx.x;
    const int H = a.H, W = a.W, pitch = a.pitch;
    const int tx0 = bx * TS, ty0 = by * TS;
    constexpr int R = BS::R;                                       // window radius
    const int px0 = tx0 - R, py0 = ty0 - R;                        // product region origin
    constexpr bool UP = RowOrder<T, KR>::bottom_up;
    const int sy0 = py0 - kBlockReach - 1 - RowOrder<T, KR>::slack;  // staged row origin
    const int sxn = px0 - kBlockReach - 1;
    const int sx0 = (sxn >= 0 ? sxn / VEC : -((-sxn + VEC - 1) / VEC)) * VEC;  // floor to a VEC multiple
    const T *P1 = static_cast<const T *>(a.P1);
    const T *P2 = static_cast<const T *>(a.P2);

    // phase 0: stage both frames (rows sy0 .. sy0+SH-1, columns sx0 .. sx0+SP-1).
    // A box inside the image: two TMA copies.  Otherwise 16-byte chunks
    // inside the image rows are copied asynchronously; chunks that straddle
    // the left or right border are filled element by element with clamped
    // columns.  Rows are clamped as a whole.
    const bool vec_ok = sx0 >= 0 && sx0 + SP <= W;
    const bool interior = vec_ok && sy0 >= 0 && sy0 + SH <= H;
    if (tm1 != nullptr && tma_bars != nullptr && interior && (smem_u32(stage) & 127u) == 0) {
        // NBAND bands of SHB rows per frame, band b of both frames on barrier b
        if (tid == 0) {
            if (init_bars)
                for (int b = 0; b < NBAND; ++b) mbar_init(&tma_bars[b], 1);
            // order earlier generic-proxy accesses of the buffer (a previous
            // tile of this CTA) before the copies
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
            for (int k = 0; k < NBAND; ++k) {
                const int b = UP ? NBAND - 1 - k : k;  // the band phase 1 needs first, first
                mbar_expect_tx(&tma_bars[b], (unsigned)(2 * SHB * SP * sizeof(T)));
                tma_load_2d(stage + b * SHB * SP, tm1, sx0, sy0 + b * SHB, &tma_bars[b]);
                tma_load_2d(stage + STG + b * SHB * SP, tm2, sx0, sy0 + b * SHB, &tma_bars[b]);
            }
        }
        if (init_bars) __syncthreads();  // barriers initialised before anyone waits on them
        bars = tma_bars;
    } else {
        for (int t = tid; t < 2 * SH * NV; t += NT) {
            const int f = t >= SH * NV ? 1 : 0;
            const int r = t - f * SH * NV;
            const int row = r / NV, v = r - row * NV;
            const int gy = min(max(sy0 + row, 0), H - 1);
            const int gx0 = sx0 + v * VEC;
            const T *src = (f ? P2 : P1) + (int64_t)gy * pitch;
            T *dst = stage + f * STG + row * SP + v * VEC;
            if (gx0 >= 0 && gx0 + VEC <= W) {
                cp_async16(dst, src + gx0);
            } else {
#pragma unroll
                for (int e = 0; e < VEC; ++e) dst[e] = src[min(max(gx0 + e, 0), W - 1)];
            }
        }
        cp_async_wait_all();
        __syncthreads();
    }

    // phase 1: products on tile + halo.  A tile whose staged rows and columns
    // all lie inside the image needs no clamping or border remap.
    // Pixels at least REACH+1 px from every border take the same fast path
    // inside border tiles too (their taps never clamp or remap).
    if (interior) {
        const T *st2 = stage + STG;
        if (mode == V0_SAME)
            products_tile_interior<T, KR, COH, V0_SAME, SP, VAR>(a, stage, st2, sx0, sy0, px0, py0, prod, bars, parity,
                                                           err);
        else if (mode == V0_UP)
            products_tile_interior<T, KR, COH, V0_UP, SP, VAR>(a, stage, st2, sx0, sy0, px0, py0, prod, bars, parity, err);
        else
            products_tile_interior<T, KR, COH, V0_ZERO, SP, VAR>(a, stage, st2, sx0, sy0, px0, py0, prod, bars, parity,
                                                           err);
        // every band has landed before the CTA can finish (no copy in flight at exit)
        if (bars && tid == 0)
            for (int b = 0; b < NBAND; ++b) mbar_wait_bounded(&bars[b], parity, 1000000000LL);
    } else {
        // index step in rows and columns (rows in the order of RowOrder)
        constexpr int DX = NT % RW, DY = UP ? -(NT / RW) : NT / RW, DW = UP ? -1 : 1;
        int ry = tid / RW, rx = tid - (tid / RW) * RW;
        if (UP) ry = RW - 1 - ry;
        // V0 of the thread's next pixel is loaded one iteration ahead
        float2 V0n = make_float2(0.f, 0.f);
        if (tid < RW * RW && py0 + ry >= 0 && py0 + ry < H && px0 + rx >= 0 && px0 + rx < W)
            V0n = fetch_v0_rt<COH>(a, mode, px0 + rx, py0 + ry);
        for (int idx = tid; idx < RW * RW; idx += NT) {
            const int gy = py0 + ry, gx = px0 + rx;
            const float2 V0c = V0n;
            int nry = ry + DY, nrx = rx + DX;
            if (nrx >= RW) { nrx -= RW; nry += DW; }
            if (idx + NT < RW * RW && py0 + nry >= 0 && py0 + nry < H && px0 + nrx >= 0 && px0 + nrx < W)
                V0n = fetch_v0_rt<COH>(a, mode, px0 + nrx, py0 + nry);
            float p[5] = {0.f, 0.f, 0.f, 0.f, 0.f};
            if (gx > kBlockReach && gx < W - kBlockReach - 2 && gy > kBlockReach && gy < H - kBlockReach - 2) {
                products_interior<T, SP, VAR>(stage, stage + STG, sx0, sy0, a, gx, gy, V0c, p);
            } else if (gy >= 0 && gy < H && gx >= 0 && gx < W) {
                const float2 V0 = V0c;
                const float hx = 0.5f * V0.x, hy = 0.5f * V0.y;
                const Sample s1 = sample_staged<T, SP>(stage, sx0, sy0, P1, H, W, pitch, gx, gy, -hx, -hy);
                const Sample s2 = sample_staged<T, SP>(stage + STG, sx0, sy0, P2, H, W, pitch, gx, gy, hx, hy);
                const float Gx = 0.5f * (s1.gx + s2.gx), Gy = 0.5f * (s1.gy + s2.gy);
                const float It = s2.val - s1.val;
                const float r = (VAR && a.inc) ? -It : Gx * V0.x + Gy * V0.y - It;
                p[0] = Gx * Gx;
                p[1] = Gx * Gy;
                p[2] = Gy * Gy;
                p[3] = Gx * r;
                p[4] = Gy * r;
            }
            // a masked pixel leaves the window sums
            if (VAR && a.mask && gy >= 0 && gy < H && gx >= 0 && gx < W && !__ldg(a.mask + (int64_t)gy * W + gx))
                p[0] = p[1] = p[2] = p[3] = p[4] = 0.f;
            float *q = prod + ry * RWP + rx;
            q[0] = p[0];
            q[PLANE] = p[1];
            q[2 * PLANE] = p[2];
            q[3 * PLANE] = p[3];
            q[4 * PLANE] = p[4];
            ry = nry;
            rx = nrx;
        }
    }
    side.after_products(tid);
    __syncthreads();

    // phase 2: horizontal window sums, one (row, channel) per thread
    // (weighted sums with the Gaussian window)
    if (VAR && a.gauss) {
        for (int t = tid; t < 5 * RW; t += NT) {
            const int c = t / RW, row = t - c * RW;
            window_wsums_inplace<R, TS>(prod + c * PLANE + row * RWP, 1, a.wg);
        }
    } else {
        for (int t = tid; t < 5 * RW; t += NT) {
            const int c = t / RW, row = t - c * RW;
            window_sums_inplace<R, TS>(prod + c * PLANE + row * RWP, 1);
        }
    }
    side.after_rows(tid);
    __syncthreads();

    // phase 3: vertical window sums, one (column, channel) per thread
    if (VAR && a.gauss) {
        for (int t = tid; t < 5 * TS; t += NT) {
            const int c = t / TS, col = t - c * TS;
            window_wsums_inplace<R, TS>(prod + c * PLANE + col, RWP, a.wg);
        }
    } else {
        for (int t = tid; t < 5 * TS; t += NT) {
            const int c = t / TS, col = t - c * TS;
            window_sums_inplace<R, TS>(prod + c * PLANE + col, RWP);
        }
    }
    __syncthreads();

    // phase 4: per output pixel, the epilogue (guarded solve and store)
    for (int idx = tid; idx < TS * TS; idx += NT) {
        const int oy = idx / TS, ox = idx - oy * TS;
        const int gy = ty0 + oy, gx = tx0 + ox;
        if (gy >= H || gx >= W) continue;
        const float *q = prod + oy * RWP + ox;
        const float S[5] = {q[0], q[PLANE], q[2 * PLANE], q[3 * PLANE], q[4 * PLANE]};
        epi.template apply<COH>(a, mode, gx, gy, S);
    }
    return bars != nullptr;
}

// One tile per CTA; blockIdx.z selects the pair.  VAR: estimator variants.
template <typename T, int KR, bool VAR>
__global__ void __launch_bounds__(BlockShape<KR>::NT, BlockShape<KR>::MINB) k_iter_block(const __grid_constant__ BlockParams prm)
{
    extern __shared__ __align__(128) float4 smem_f4[];
    __shared__ __align__(8) uint64_t s_bar[StageShape<T, KR>::NBAND];
    const int z = blockIdx.z;
    if (prm.use_tma) {
        block_tile<T, KR, false, SolveStoreT<VAR>, VAR>(prm.a[z], prm.mode, blockIdx.x, blockIdx.y + prm.by0, smem_f4,
                                                        &prm.tm[z][0], &prm.tm[z][1], prm.err, SolveStoreT<VAR>(),
                                                        s_bar, 0u, true);
    } else {
        block_tile<T, KR, false, SolveStoreT<VAR>, VAR>(prm.a[z], prm.mode, blockIdx.x, blockIdx.y + prm.by0,
                                                        smem_f4);
    }
}

// ---------------------------------------------------------------------------
// Persistent batched launch: many pairs of unequal size, all (level,
// iteration) stages, in one launch.  Work units (stage, pair, tile) are
// handed out in the order of a schedule built on the host; a unit of stage
// s waits until every tile of stage s-1 of its pair is done (a per-(stage,
// pair) counter).  Units are claimed in schedule order by resident CTAs,
// each CTA one unit ahead of the one it runs; a unit depends only on
// earlier units, so the earliest unfinished unit is always being run by its
// CTA (any unit before it in that CTA is finished) and the launch cannot
// stall on itself.  The wait is bounded
// by an iteration count and a %globaltimer deadline; on expiry the CTA
// records an error word and leaves, and the host reports OFV_ERR_TIMEOUT.
// ---------------------------------------------------------------------------
struct BatchPair {
    const void *P1[16], *P2[16];  // level images of the two frames
    int H[16], W[16], pitch[16];
    float2 *vb[2];                // ping-pong fields (pitch vpitch)
    float *u, *v;                 // caller's outputs
    int vpitch;
};

struct QueueParams {
    const BatchPair *pairs;  // [npairs]
    const int4 *unit_desc;   // [total_units] (stage, pair, tile, tiles of the pair's previous stage)
    int total_units, npairs;
    int L, IT, kr;
    float eps_rel, eps_abs;
    int inc, gauss;          // estimator variants (as IterArgs)
    float wg[kBlockMaxKR + 1];
    int *head;               // next unclaimed unit
    int *done;               // [stages * npairs] finished tiles
    int *error;              // 0, or 1 + the unit whose wait expired
    long long timeout_ns;
    int spin_limit;
    const CUtensorMap *tmaps;  // [pair][16 levels][2 frames] for TMA staging, or null
    int *tma_err;              // set to 1 when a TMA wait expires, or null
    int *host_err;             // mapped host word: 1 + the unit whose wait expired, or null
};

__device__ __forceinline__ int ld_acquire(const int *p)
{
    int v;
    asm volatile("ld.acquire.gpu.global.s32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

// The persistent kernel's side work (see NoSide): thread 0 publishes the
// unit it claimed for after this tile, and a thread with no line in the
// row pass reads that unit's descriptor and looks once whether its
// dependency is already complete, so the next unit starts without those
// round trips.
struct QueueSide {
    const QueueParams *q;
    int next;          // thread 0: the claimed next unit
    int side_tid;      // the thread that prefetches
    int *s_next;
    int4 *s_dec;       // prefetched descriptor
    int *s_dec_unit;   // its unit (-1: none)
    int *s_dec_ok;     // 1: its dependency was seen complete
    __device__ __forceinline__ void after_products(int tid) const
    {
        if (tid == 0) *s_next = next;
    }
    __device__ __forceinline__ void after_rows(int tid) const
    {
        if (tid != side_tid) return;
        const int n = *s_next;
        if (n >= q->total_units) return;
        const int4 d = __ldg(q->unit_desc + n);
        *s_dec_ok = d.x == 0 || ld_acquire(q->done + (d.x - 1) * q->npairs + d.y) >= d.w;
        *s_dec = d;
        *s_dec_unit = n;
    }
};

template <typename T, int KR, bool VAR>
__global__ void __launch_bounds__(BlockShape<KR>::NT, BlockShape<KR>::MINB) k_iter_queue(const __grid_constant__ QueueParams q)
{
    constexpr int TS = BlockShape<KR>::TS;
    extern __shared__ __align__(128) float4 smem_f4[];
    __shared__ int s_unit, s_fail, s_next, s_dec_unit, s_dec_ok;
    __shared__ int4 s_dec;
    __shared__ __align__(8) uint64_t s_bar[StageShape<T, KR>::NBAND];
    const int S = q.L * q.IT;
    unsigned tma_uses = 0;  // TMA-staged tiles of this CTA so far
    if (q.tmaps && threadIdx.x == 0)
        for (int b = 0; b < StageShape<T, KR>::NBAND; ++b) mbar_init(&s_bar[b], 1);  // visible after the loop's first barrier
    if (threadIdx.x == 0) {
        s_unit = atomicAdd(q.head, 1);
        s_fail = 0;
        s_dec_unit = -1;
    }
    __syncthreads();
    // thread 0: the (stage, pair) whose previous stage it last saw complete
    int checked = -1;
    for (;;) {
        const int unit = s_unit;
        if (unit >= q.total_units) break;
        // the unit's descriptor, prefetched during the previous tile when
        // this CTA ran one
        const bool pre = s_dec_unit == unit;
        const int4 d = pre ? s_dec : __ldg(q.unit_desc + unit);
        const bool pre_ok = pre && s_dec_ok;
        const int s = d.x, p = d.y, tile = d.z, need = d.w;
        const int key = s * q.npairs + p;
        const BatchPair &bp = q.pairs[p];
        const int l = q.L - 1 - s / q.IT, t = s % q.IT;
        // the next unit is claimed now and read after this tile, so the
        // claim's round trip overlaps the tile's work
        int next = 0;
        if (threadIdx.x == 0) next = atomicAdd(q.head, 1);
        if (s > 0 && threadIdx.x == 0 && !pre_ok && checked != key) {
            const int *cnt = q.done + (s - 1) * q.npairs + p;
            const long long t0 = global_ns();
            int spins = 0;
            while (ld_acquire(cnt) < need) {
                if (++spins > q.spin_limit || global_ns() - t0 > q.timeout_ns) {
                    atomicCAS(q.error, 0, 1 + unit);
                    if (q.host_err) *reinterpret_cast<volatile int *>(q.host_err) = 1 + unit;
                    s_fail = 1;
                    break;
                }
                __nanosleep(128);
            }
            checked = key;
        }
        __syncthreads();
        if (s_fail) break;
        IterArgs a = {};
        a.P1 = bp.P1[l];
        a.P2 = bp.P2[l];
        a.H = bp.H[l];
        a.W = bp.W[l];
        a.pitch = bp.pitch[l];
        a.vpitch = bp.vpitch;
        a.vcpitch = bp.vpitch;
        a.kr = q.kr;
        a.eps_rel = q.eps_rel;
        a.eps_abs = q.eps_abs;
        if (VAR) {
            a.inc = q.inc;
            a.gauss = q.gauss;
#pragma unroll
            for (int d = 0; d <= kBlockMaxKR; ++d) a.wg[d] = q.wg[d];
        }
        int mode = V0_ZERO;
        if (s > 0 && t == 0) {
            mode = V0_UP;
            a.Vc = bp.vb[(s - 1) & 1];
            a.Hc = bp.H[l + 1];
            a.Wc = bp.W[l + 1];
        } else if (s > 0) {
            mode = V0_SAME;
            a.V0 = bp.vb[(s - 1) & 1];
        }
        if (s == S - 1) {
            a.u_out = bp.u;
            a.v_out = bp.v;
        } else {
            a.Vout = bp.vb[s & 1];
        }
        const int ntx = (a.W + TS - 1) / TS;
        const CUtensorMap *tm = q.tmaps ? q.tmaps + ((size_t)p * 16 + l) * 2 : nullptr;
        const QueueSide side{&q, next, BlockShape<KR>::NT - 1, &s_next, &s_dec, &s_dec_unit, &s_dec_ok};
        if (block_tile<T, KR, true, SolveStoreT<VAR>, VAR, QueueSide>(a, mode, tile % ntx, tile / ntx, smem_f4, tm,
                                                                      tm ? tm + 1 : nullptr, q.tma_err,
                                                                      SolveStoreT<VAR>(), q.tmaps ? s_bar : nullptr,
                                                                      tma_uses & 1u, false, side))
            ++tma_uses;
        __threadfence();
        __syncthreads();
        if (threadIdx.x == 0) {
            atomicAdd(q.done + key, 1);
            s_unit = next;
        }
        __syncthreads();
    }
}

// Host launchers, explicitly instantiated per level storage type T and
// variant flag VAR in k_block_{f32,f16,bf16}.cu (VAR = false, plus the
// reverse-mode stage kernel) and k_block_var_{f32,f16,bf16}.cu (VAR = true).
// shape: the tile shape v (the estimator variants, VAR = true, have the
// default shape only)
template <typename T, bool VAR>
cudaError_t launch_block_t(const BlockParams &p, int kr, int npairs, cudaStream_t s, int nrows = 0, int shape = 0);
template <typename T, bool VAR>
cudaError_t launch_queue_t(const QueueParams &q, int kr, int ctas, cudaStream_t s, int shape = 0);
template <typename T, bool VAR>
int queue_occupancy_t(int kr, int shape = 0);

// Output tile edge of the block kernel for radius kr and tile shape v.
inline int block_tile_size(int kr, int v = 0) { return block_tile_edge(kr, v); }

}  // namespace ofv
