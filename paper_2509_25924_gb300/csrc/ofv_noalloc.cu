// Allocation-free variant of ofv_compute for callers that cannot allocate
// device memory: plug-in hosts whose device memory is owned by someone
// else's allocator, or real-time loops that forbid any allocation after
// start-up.  It runs the same kernels as ofv_compute (image tiles staged by
// cp.async, as it keeps no TMA tensor maps), but its workspace (pyramids of
// both frames and the two ping-pong fields) lives in one file-scope device
// array of fixed size instead of a handle's cudaMalloc.
//
// The array is a module global: every GPU on which this library's kernels
// are loaded holds OFV_NOALLOC_SCRATCH_BYTES of it until the process exits.
// Host code cannot use the array's name as a device address (on the host it
// names a stand-in); its device address is looked up once per device with
// cudaGetSymbolAddress and then passed to the kernels.
#include <cuda_runtime.h>

#include <cmath>
#include <cstdio>
#include <mutex>

#include "../../include/ofv.h"
#include "k_block.cuh"
#include "ofv_handle.h"

namespace ofv {
void set_error_message(const char *msg);
}

using namespace ofv;

static __device__ __align__(256) unsigned char g_noalloc_scratch[OFV_NOALLOC_SCRATCH_BYTES];

namespace {

constexpr int kMaxDevices = 64;
constexpr int kLevels = 16;
std::mutex g_setup_mu;
void *g_scratch_addr[kMaxDevices];

ofv_status na_fail(ofv_status st, const char *msg)
{
    set_error_message(msg);
    return st;
}

size_t na_align(size_t v) { return (v + 255) / 256 * 256; }

// Device address of the scratch array on the current device; looked up on
// the first call per device.
ofv_status scratch_for_device(void **out)
{
    int dev = -1;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return na_fail(OFV_ERR_CUDA, "ofv_compute_noalloc: cudaGetDevice failed");
    if (dev < 0 || dev >= kMaxDevices) return na_fail(OFV_ERR_UNSUPPORTED, "ofv_compute_noalloc: device ordinal >= 64");
    std::lock_guard<std::mutex> lk(g_setup_mu);
    if (!g_scratch_addr[dev]) {
        void *p = nullptr;
        e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess || !p) {
            char buf[256];
            snprintf(buf, sizeof buf, "ofv_compute_noalloc: cudaGetSymbolAddress of the scratch array failed: %s",
                     cudaGetErrorString(e));
            return na_fail(OFV_ERR_CUDA, buf);
        }
        g_scratch_addr[dev] = p;
    }
    *out = g_scratch_addr[dev];
    return OFV_OK;
}

}  // namespace

extern "C" ofv_status ofv_compute_noalloc(int H, int W, const ofv_params *p, const float *w25, const void *I1,
                                          const void *I2, float *u, float *v, ofv_stream_t s)
{
    char msg[320];
    if (!p || !I1 || !I2 || !u || !v || u == v)
        return na_fail(OFV_ERR_INVALID_ARG, "ofv_compute_noalloc: NULL pointer or u == v");
    if (p->levels_psl < 0 || p->levels_psl >= kLevels || p->kernel_radius < 1 || p->kernel_radius > 16 ||
        p->iterations < 1 || p->iterations > 64 || p->norm_radius < 0 || p->norm_radius > 16 ||
        (p->input != OFV_IN_U8 && p->input != OFV_IN_U16 && p->input != OFV_IN_F32) ||
        (p->input != OFV_IN_F32 && (p->bit_depth < 1 || p->bit_depth > (p->input == OFV_IN_U8 ? 8 : 16))) ||
        (p->storage != OFV_STORE_F32 && p->storage != OFV_STORE_F16 && p->storage != OFV_STORE_BF16) ||
        (p->prefilter != 0 && p->prefilter != 1) || !(p->det_rel_eps >= 0.f) || !std::isfinite(p->det_rel_eps) ||
        !(p->det_abs_eps >= 0.f) || !std::isfinite(p->det_abs_eps) || !(p->norm_eps > 0.f) ||
        !std::isfinite(p->norm_eps) || (p->window != OFV_WINDOW_BOX && p->window != OFV_WINDOW_GAUSS) ||
        (p->window == OFV_WINDOW_GAUSS && (!(p->window_sigma > 0.f) || !std::isfinite(p->window_sigma))) ||
        (p->increment_form != 0 && p->increment_form != 1) || p->max_batch < 0 ||
        p->max_batch > kMaxPairsPerLaunch || p->warm_start < 0 || p->warm_start > 7 * kMaxPairsPerLaunch ||
        tile_shape_of(*p) < 0)
        return na_fail(OFV_ERR_INVALID_ARG, "ofv_compute_noalloc: parameter out of range (see ofv_params)");
    if (p->path != OFV_PATH_FUSED)
        return na_fail(OFV_ERR_UNSUPPORTED, "ofv_compute_noalloc: only the fused path is available without allocation");
    if (p->prefilter && !w25)
        return na_fail(OFV_ERR_INVALID_ARG, "ofv_compute_noalloc: prefilter = 1 needs the 25 weights (w25)");
    if (H < 1 || W < 1 || (int64_t)H * W > 2147483647LL)
        return na_fail(OFV_ERR_SHAPE, "ofv_compute_noalloc: H and W must be positive with H*W < 2^31");

    const int L = p->levels_psl + 1;
    int Hs[kLevels], Ws[kLevels], pitch[kLevels];
    Hs[0] = H;
    Ws[0] = W;
    for (int l = 1; l < L; ++l) {
        Hs[l] = (Hs[l - 1] + 1) / 2;
        Ws[l] = (Ws[l - 1] + 1) / 2;
    }
    const int minsz = 2 * p->kernel_radius + 1 > 8 ? 2 * p->kernel_radius + 1 : 8;
    if (Hs[L - 1] < minsz || Ws[L - 1] < minsz) {
        snprintf(msg, sizeof msg, "ofv_compute_noalloc: coarsest level %dx%d is below max(8, 2KR+1)=%d",
                 Hs[L - 1], Ws[L - 1], minsz);
        return na_fail(OFV_ERR_SHAPE, msg);
    }
    for (int l = 0; l < L; ++l) pitch[l] = pitch_for(Ws[l]);
    const int vpitch = pitch_for(W);
    const int sb = p->storage == OFV_STORE_F32 ? 4 : 2;

    // layout of the scratch array (offsets in bytes)
    size_t off = 0, lvl_off[2][kLevels], vb_off[2], tmp_off[2] = {0, 0};
    for (int f = 0; f < 2; ++f)
        for (int l = 0; l < L; ++l) {
            lvl_off[f][l] = off;
            off = na_align(off + (size_t)Hs[l] * pitch[l] * sb);
        }
    for (int k = 0; k < 2; ++k) {
        vb_off[k] = off;
        off = na_align(off + (size_t)H * vpitch * sizeof(float2));
    }
    if (p->prefilter)
        for (int k = 0; k < 2; ++k) {
            tmp_off[k] = off;
            off = na_align(off + (size_t)H * pitch[0] * sizeof(float));
        }
    if (off > (size_t)OFV_NOALLOC_SCRATCH_BYTES) {
        snprintf(msg, sizeof msg,
                 "ofv_compute_noalloc: %dx%d with PSL %d needs %zu workspace bytes, more than the fixed %zu-byte "
                 "scratch array; use ofv_create/ofv_compute",
                 H, W, p->levels_psl, off, (size_t)OFV_NOALLOC_SCRATCH_BYTES);
        return na_fail(OFV_ERR_SHAPE, msg);
    }

    void *scratch = nullptr;
    ofv_status st = scratch_for_device(&scratch);
    if (st != OFV_OK) return st;
    char *base = static_cast<char *>(scratch);
    cudaStream_t cs = (cudaStream_t)s;

    // steps 1-2: ingest both frames into level 0, then the pyramid
    IngestArgs ia[2];
    const void *fr[2] = {I1, I2};
    for (int k = 0; k < 2; ++k) {
        IngestArgs &a = ia[k];
        a.raw = fr[k];
        a.out = base + lvl_off[k][0];
        a.tmp = p->prefilter ? reinterpret_cast<float *>(base + tmp_off[k]) : nullptr;
        a.w25 = w25;
        a.H = H;
        a.W = W;
        a.pitch = pitch[0];
        a.in_type = p->input;
        a.bits = p->bit_depth;
        a.nr = p->norm_radius;
        a.eps_n = p->norm_eps;
        a.prefilter = p->prefilter;
    }
    cudaError_t e = launch_ingest_frames(ia, 2, p->storage, cs);
    for (int l = 1; l < L && e == cudaSuccess; ++l) {
        ReduceArgs ra[2];
        for (int k = 0; k < 2; ++k) {
            ra[k].src = base + lvl_off[k][l - 1];
            ra[k].Hs = Hs[l - 1];
            ra[k].Ws = Ws[l - 1];
            ra[k].spitch = pitch[l - 1];
            ra[k].dst = base + lvl_off[k][l];
            ra[k].Hd = Hs[l];
            ra[k].Wd = Ws[l];
            ra[k].dpitch = pitch[l];
        }
        e = launch_reduce_frames(ra, 2, p->storage, cs);
    }

    // steps 3-6: coarse to fine; every buffer is written before it is read,
    // so nothing left in the array by an earlier call is ever used
    float2 *vbuf[2] = {reinterpret_cast<float2 *>(base + vb_off[0]), reinterpret_cast<float2 *>(base + vb_off[1])};
    int cur = 0;
    bool have = false;
    for (int l = L - 1; l >= 0 && e == cudaSuccess; --l) {
        for (int t = 0; t < p->iterations && e == cudaSuccess; ++t) {
            IterArgs a = {};
            a.P1 = base + lvl_off[0][l];
            a.P2 = base + lvl_off[1][l];
            a.H = Hs[l];
            a.W = Ws[l];
            a.pitch = pitch[l];
            a.vpitch = vpitch;
            a.vcpitch = vpitch;
            a.kr = p->kernel_radius;
            a.eps_rel = p->det_rel_eps;
            a.eps_abs = p->det_abs_eps;
            set_iter_variant(a, p->kernel_radius, p->window == OFV_WINDOW_GAUSS, p->window_sigma, p->increment_form);
            int mode;
            if (t == 0 && l == L - 1) {
                mode = V0_ZERO;
            } else if (t == 0) {
                mode = V0_UP;
                a.Vc = vbuf[cur];
                a.Hc = Hs[l + 1];
                a.Wc = Ws[l + 1];
            } else {
                mode = V0_SAME;
                a.V0 = vbuf[cur];
            }
            const int nxt = have ? 1 - cur : 0;
            if (l == 0 && t == p->iterations - 1) {
                a.u_out = u;
                a.v_out = v;
            } else {
                a.Vout = vbuf[nxt];
            }
            e = block_supports(p->kernel_radius)
                    ? launch_iter_block(&a, 1, p->storage, mode, cs, nullptr, nullptr, 0, 0, tile_shape_of(*p))
                    : launch_iter_fused(a, p->storage, mode, cs);
            cur = nxt;
            have = true;
        }
    }
    if (e != cudaSuccess) {
        snprintf(msg, sizeof msg, "ofv_compute_noalloc: kernel launch failed: %s", cudaGetErrorString(e));
        return na_fail(OFV_ERR_CUDA, msg);
    }
    return OFV_OK;
}
