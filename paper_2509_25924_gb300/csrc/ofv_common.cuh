// Shared device helpers and launch descriptors of the OFV CUDA path.
#pragma once

#include <cuda.h>  // CUtensorMap
#include <cuda_runtime.h>
#include <cmath>
#include <cuda_fp16.h>
#include <cuda_bf16.h>
#include <stdint.h>

namespace ofv {

enum Store : int { ST_F32 = 0, ST_F16 = 1, ST_BF16 = 2 };
enum In : int { IN_U8 = 0, IN_U16 = 1, IN_F32 = 2 };

// Source of the field V0 that the first warp of an iteration uses.
enum V0Mode : int {
    V0_ZERO = 0,  // coarsest level, first iteration: V0 = 0
    V0_SAME = 1,  // previous iteration of the same level
    V0_UP = 2     // first iteration of a finer level: 2 * bilinear(Vc, x/2, y/2)
};

// Pairs of one time-resolved sequence processed by one iteration launch, and
// frames ingested or reduced by one launch.
constexpr int kMaxPairsPerLaunch = 8;
constexpr int kMaxWindowRadius = 16;  // largest KR
constexpr int kMaxFramesPerLaunch = kMaxPairsPerLaunch + 1;

// Level images are stored with a row pitch (elements) that is a multiple of
// 64, so every row starts 128-byte aligned in all storage types.
constexpr int kPitchAlign = 64;
inline int pitch_for(int w) { return (w + kPitchAlign - 1) / kPitchAlign * kPitchAlign; }

__device__ __forceinline__ float ld_store(const float *p) { return __ldg(p); }
__device__ __forceinline__ float ld_store(const __half *p) { return __half2float(__ldg(p)); }
__device__ __forceinline__ float ld_store(const __nv_bfloat16 *p) { return __bfloat162float(__ldg(p)); }

__device__ __forceinline__ float to_f(float v) { return v; }
__device__ __forceinline__ float to_f(__half v) { return __half2float(v); }
__device__ __forceinline__ float to_f(__nv_bfloat16 v) { return __bfloat162float(v); }

__device__ __forceinline__ void st_store(float *p, float v) { *p = v; }
__device__ __forceinline__ void st_store(__half *p, float v) { *p = __float2half_rn(v); }
__device__ __forceinline__ void st_store(__nv_bfloat16 *p, float v) { *p = __float2bfloat16_rn(v); }

__device__ __forceinline__ int clampi(int v, int lo, int hi) { return v < lo ? lo : (v > hi ? hi : v); }

// One level of one pair, as seen by an iteration kernel.
struct IterArgs {
    const void *P1, *P2;  // level images (storage type), pitch `pitch` elements
    int H, W, pitch;
    const float2 *V0;     // V0_SAME: field of the previous iteration, pitch vpitch
    const float2 *Vc;     // V0_UP: field of level l+1 (Hc x Wc), pitch vcpitch
    int Hc, Wc, vcpitch;
    float2 *Vout;         // interleaved output (pitch vpitch), or null when planar
    float *u_out, *v_out; // planar dense output (level 0, last iteration)
    int vpitch;
    int kr;
    float eps_rel, eps_abs;
    const uint8_t *mask;  // region mask of the level (dense rows of W, 0 = masked), or null
    float *s_out;         // reverse mode: the five window sums of every pixel, plane c at s_out + c s_plane
    size_t s_plane;       //   (rows of s_pitch floats), or null
    int s_pitch;
    int inc;              // 1: increment form, r = -It and V = V0(m) + H^-1 (Sxr, Syr)
    int gauss;            // 1: window tap (a, b) weighted wg[|a|] wg[|b|]; 0: uniform box
    float wg[kMaxWindowRadius + 1];  // Gaussian window weights exp(-d^2 / (2 sigma^2)), d = 0..KR
};

// Estimator variants of an iteration (host side): the increment form and
// the Gaussian window weights of radius kr and width sigma.
inline void set_iter_variant(IterArgs &a, int kr, int window_gauss, float sigma, int increment_form)
{
    a.inc = increment_form ? 1 : 0;
    a.gauss = window_gauss ? 1 : 0;
    for (int d = 0; d <= kMaxWindowRadius; ++d)
        a.wg[d] = (a.gauss && d <= kr) ? (float)std::exp(-(double)d * d / (2.0 * (double)sigma * sigma)) : 1.f;
}

// Host-side launchers (defined in the kernel translation units).
// Tile kernel: one CTA per 32x32 output tile, products staged in shared memory.
cudaError_t launch_iter_fused(const IterArgs &a, int store, int mode, cudaStream_t s);
// Block-tiled kernel (KR 1..10): npairs pairs of equal level size in one launch.
// tm (optional): 2 * npairs tensor maps (frame 1 and frame 2 of pair k at
// 2k, 2k+1) of the level images with the box of block_stage_box; tiles whose
// staged box lies inside the image are then loaded by TMA.  err (optional):
// device-visible word set to 1 if a TMA wait expires.
bool block_supports(int kr);
// The forward solve's reciprocal of x[0..n-1] into y (device arrays), for tests.
cudaError_t launch_recip(const float *x, float *y, int n, cudaStream_t s);
// by0, nby: tile rows by0 .. by0+nby-1 only (nby 0: to the bottom of the level).
// shape: the tile shape (0 default, 1 the alternative; the estimator
// variants run the default shape).
cudaError_t launch_iter_block(const IterArgs *a, int npairs, int store, int mode, cudaStream_t s,
                              const CUtensorMap *const *tm = nullptr, int *err = nullptr, int by0 = 0, int nby = 0,
                              int shape = 0);
// TMA box of the block kernel's staging (columns, rows of one band) for this
// storage, radius and tile shape.
void block_stage_box(int store, int kr, int *cols, int *rows, int shape = 0);

struct PlainBufs {
    float *prod;  // 5 planes, each H x pitch floats
    float *hsum;  // 5 planes, each H x pitch floats
    float2 *vtmp; // up-sampled V0 plane (pitch vpitch)
    size_t plane; // elements per plane
};
cudaError_t launch_iter_plain(const IterArgs &a, const PlainBufs &b, int store, int mode,
                              cudaStream_t s);

struct IngestArgs {
    const void *raw;   // H x W input, dense
    void *out;         // level 0 storage, pitch elements
    float *tmp;        // FP32 scratch (H x pitch) used when the pre-filter is on
    const float *w25;  // pre-filter weights (device)
    int H, W, pitch;
    int in_type, bits;
    int nr;
    float eps_n;
    int prefilter;
};
// Ingest nframes (1 or 2) frames in one launch.
cudaError_t launch_ingest_frames(const IngestArgs *f, int nframes, int store, cudaStream_t s);

struct ReduceArgs {
    const void *src; int Hs, Ws, spitch;
    void *dst; int Hd, Wd, dpitch;
};
// Reduce one level of nframes (1 or 2) frames in one launch.
cudaError_t launch_reduce_frames(const ReduceArgs *f, int nframes, int store, cudaStream_t s);

// Any number of frames of any sizes in one launch: f on the host, dev_f the
// same descriptors in device memory, valid until the launch has run.
cudaError_t launch_ingest_list(const IngestArgs *f, const IngestArgs *dev_f, int nframes, int store, cudaStream_t s);
cudaError_t launch_reduce_list(const ReduceArgs *f, const ReduceArgs *dev_f, int nframes, int store, cudaStream_t s);

// Warm start: the starting field of the coarsest level from a level-0
// field, out(i, j) = (u, v)(2^level i, 2^level j) / 2^level (pitch vpitch).
struct SeedArgs {
    const float *u, *v;  // level-0 field, dense rows of W0
    int W0, level;
    float2 *out;
    int H, W, vpitch;    // the level's size
};
cudaError_t launch_seed_fields(const SeedArgs *a, int n, cudaStream_t s);

// Region mask of every level from the level-0 mask (H x W bytes, nonzero =
// valid): out[l](i, j) = mask(2^l i, 2^l j) != 0, dense rows of Ws[l].
cudaError_t launch_mask_levels(const uint8_t *mask, int W, uint8_t *const *out, const int *Hs, const int *Ws, int L,
                               cudaStream_t s);

// The output of a masked pixel (no vector).
__device__ __forceinline__ float no_vector() { return __int_as_float(0x7fc00000); }

cudaError_t launch_read_level(const void *src, int H, int W, int pitch, int store, float *dst,
                              cudaStream_t s);

}  // namespace ofv
