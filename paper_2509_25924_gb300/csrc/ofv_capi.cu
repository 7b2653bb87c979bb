// C ABI of the OFV estimator: handle, workspace, argument checks and the
// level loop of Sec. 2 (normalize -> pyramid -> per level IT Gauss-Newton
// iterations of Eq. 2 -> up-sample to the next finer level).
//
// Several pairs of a time-resolved sequence are processed together: their
// frames are ingested and reduced in shared launches and each (level,
// iteration) of the fused path is one launch over all of them, which keeps
// the coarse levels from leaving the GPU idle.
#include <cuda_runtime.h>
#include <cudaTypedefs.h>
#include <nvtx3/nvToolsExt.h>

#include <atomic>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <new>
#include <vector>

#include "../../include/ofv.h"
#include "ofv_common.cuh"
#include "ofv_handle.h"

using namespace ofv;

namespace {

thread_local char g_err[1024] = "no error";

ofv_status fail(ofv_status st, const char *fmt, ...)
{
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(g_err, sizeof g_err, fmt, ap);
    va_end(ap);
    return st;
}

ofv_status cuda_fail(cudaError_t e, const char *where)
{
    return fail(OFV_ERR_CUDA, "%s: %s (%s)", where, cudaGetErrorString(e), cudaGetErrorName(e));
}

}  // namespace

namespace {

struct DeviceGuard {
    int prev = -1;
    bool ok = true;
    explicit DeviceGuard(int dev)
    {
        if (cudaGetDevice(&prev) != cudaSuccess) { ok = false; return; }
        if (prev != dev && cudaSetDevice(dev) != cudaSuccess) ok = false;
    }
    ~DeviceGuard()
    {
        int cur = -1;
        if (prev >= 0 && cudaGetDevice(&cur) == cudaSuccess && cur != prev) cudaSetDevice(prev);
    }
};

ofv_status check_params(const ofv_params *p)
{
    if (!p) return fail(OFV_ERR_INVALID_ARG, "params is NULL");
    if (p->levels_psl < 0 || p->levels_psl > kMaxLevels - 1)
        return fail(OFV_ERR_INVALID_ARG, "levels_psl=%d outside 0..%d", p->levels_psl, kMaxLevels - 1);
    if (p->kernel_radius < 1 || p->kernel_radius > 16)
        return fail(OFV_ERR_INVALID_ARG, "kernel_radius=%d outside 1..16", p->kernel_radius);
    if (p->iterations < 1 || p->iterations > 64)
        return fail(OFV_ERR_INVALID_ARG, "iterations=%d outside 1..64", p->iterations);
    if (p->norm_radius < 0 || p->norm_radius > 16)
        return fail(OFV_ERR_INVALID_ARG, "norm_radius=%d outside 0..16", p->norm_radius);
    if (p->input != OFV_IN_U8 && p->input != OFV_IN_U16 && p->input != OFV_IN_F32)
        return fail(OFV_ERR_INVALID_ARG, "input=%d is not an ofv_input_t", p->input);
    if (p->input != OFV_IN_F32) {
        const int maxb = p->input == OFV_IN_U8 ? 8 : 16;
        if (p->bit_depth < 1 || p->bit_depth > maxb)
            return fail(OFV_ERR_INVALID_ARG, "bit_depth=%d outside 1..%d", p->bit_depth, maxb);
    }
    if (p->storage != OFV_STORE_F32 && p->storage != OFV_STORE_F16 && p->storage != OFV_STORE_BF16)
        return fail(OFV_ERR_INVALID_ARG, "storage=%d is not an ofv_storage_t", p->storage);
    if (p->path != OFV_PATH_FUSED && p->path != OFV_PATH_PLAIN && p->path != OFV_PATH_TILE)
        return fail(OFV_ERR_INVALID_ARG, "path=%d is not an ofv_path_t", p->path);
    if (p->prefilter != 0 && p->prefilter != 1)
        return fail(OFV_ERR_INVALID_ARG, "prefilter=%d is not 0 or 1", p->prefilter);
    if (!(p->det_rel_eps >= 0.f) || !std::isfinite(p->det_rel_eps) || !(p->det_abs_eps >= 0.f) ||
        !std::isfinite(p->det_abs_eps) || !(p->norm_eps > 0.f) || !std::isfinite(p->norm_eps))
        return fail(OFV_ERR_INVALID_ARG, "guard / normalization epsilons must be finite (norm_eps > 0)");
    if (p->max_batch < 0 || p->max_batch > kMaxBatch)
        return fail(OFV_ERR_INVALID_ARG, "max_batch=%d outside 0..%d", p->max_batch, kMaxBatch);
    if (p->window != OFV_WINDOW_BOX && p->window != OFV_WINDOW_GAUSS)
        return fail(OFV_ERR_INVALID_ARG, "window=%d is not an ofv_window_t", p->window);
    if (p->window == OFV_WINDOW_GAUSS && (!(p->window_sigma > 0.f) || !std::isfinite(p->window_sigma)))
        return fail(OFV_ERR_INVALID_ARG, "window_sigma=%g must be finite and > 0 for the Gaussian window",
                    (double)p->window_sigma);
    if (p->increment_form != 0 && p->increment_form != 1)
        return fail(OFV_ERR_INVALID_ARG, "increment_form=%d is not 0 or 1", p->increment_form);
    if (p->warm_start < 0 || p->warm_start > 7 * kMaxBatch)
        return fail(OFV_ERR_INVALID_ARG, "warm_start=%d outside 0..%d", p->warm_start, 7 * kMaxBatch);
    if (tile_shape_of(*p) < 0)
        return fail(OFV_ERR_INVALID_ARG, "tile_edge=%d: 0, %d or %d for KR %d on the fused path", p->tile_edge,
                    block_tile_edge(p->kernel_radius, 0), block_tile_edge(p->kernel_radius, 1), p->kernel_radius);
    return OFV_OK;
}

ofv_status last_launch(cudaError_t e, const char *what)
{
    if (e != cudaSuccess) return cuda_fail(e, what);
    return OFV_OK;
}

cudaEvent_t pool_event(ofv_handle *h)
{
    if (h->pool_next < h->pool.size()) return h->pool[h->pool_next++];
    cudaEvent_t e = nullptr;
    if (cudaEventCreate(&e) != cudaSuccess) return nullptr;
    h->pool.push_back(e);
    h->pool_next = h->pool.size();
    return e;
}

// Bracket a launch with events when timing is on.
struct ProfScope {
    ofv_handle *h;
    cudaStream_t s;
    int cls;
    double bytes;
    cudaEvent_t e0 = nullptr;
    ProfScope(ofv_handle *h_, cudaStream_t s_, int cls_, double bytes_) : h(h_), s(s_), cls(cls_), bytes(bytes_)
    {
        if (h->prof) {
            e0 = pool_event(h);
            if (e0) cudaEventRecord(e0, s);
        }
    }
    ~ProfScope()
    {
        if (h->prof && e0) {
            cudaEvent_t e1 = pool_event(h);
            if (e1) {
                cudaEventRecord(e1, s);
                h->recs.push_back(ProfRec{cls, e0, e1, bytes});
            }
        }
    }
};

// cuTensorMapEncodeTiled, looked up once through the runtime (no link to
// the driver library).
PFN_cuTensorMapEncodeTiled_v12000 tensor_map_encoder_impl()
{
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    static bool tried = false;
    if (!tried) {
        tried = true;
        void *ptr = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &ptr, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(ptr);
        else
            cudaGetLastError();
    }
    return fn;
}

// Tensor maps of the level images for the block kernel's staged box (see
// encode_block_map).  Levels smaller than the box never have an interior
// tile and keep cp.async.
void encode_tensor_maps(ofv_handle *h)
{
    int cols = 0, rows = 0;
    block_stage_box(h->p.storage, h->p.kernel_radius, &cols, &rows, tile_shape_of(h->p));
    for (int l = 0; l < h->L; ++l) {
        h->tma_ok[l] = 0;
        if (cols < 1 || h->Ws[l] < cols || h->Hs[l] < rows) continue;
        bool ok = true;
        for (int f = 0; f < h->nslots && ok; ++f)
            ok = encode_block_map(&h->tmap[f][l], h->lvl[f][l], h->Ws[l], h->Hs[l], h->pitch[l], h->p.storage,
                                  h->p.kernel_radius, tile_shape_of(h->p));
        h->tma_ok[l] = ok ? 1 : 0;
    }
}

// Steps 1-2: ingest nf frames (frames[k] into pyramid slot slots[k]) and
// reduce them, nf frames per launch.
ofv_status build_pyramids(ofv_handle *h, const void *const *frames, const int *slots, int nf, cudaStream_t s,
                          int tset = 0)
{
    const ofv_params &p = h->p;
    const int sb = store_bytes(p.storage), ib = input_bytes(p.input);
    nvtxRangePushA("ofv ingest and pyramid");
    struct RangePop {
        ~RangePop() { nvtxRangePop(); }
    } pop_at_return;
    IngestArgs ia[kMaxFramesPerLaunch];
    for (int k = 0; k < nf; ++k) {
        IngestArgs &a = ia[k];
        a.raw = frames[k];
        a.out = h->lvl[slots[k]][0];
        a.tmp = h->tmp[tset * kMaxFramesPerLaunch + k];
        a.w25 = h->w25;
        a.H = h->H;
        a.W = h->W;
        a.pitch = h->pitch[0];
        a.in_type = p.input;
        a.bits = p.bit_depth;
        a.nr = p.norm_radius;
        a.eps_n = p.norm_eps;
        a.prefilter = p.prefilter;
    }
    {
        const double N = (double)h->H * h->W;
        ProfScope ps(h, s, OFV_K_INGEST, nf * N * (ib + sb));
        ofv_status st = last_launch(launch_ingest_frames(ia, nf, p.storage, s), "ingest launch");
        if (st != OFV_OK) return st;
    }
    for (int l = 1; l < h->L; ++l) {
        ReduceArgs ra[kMaxFramesPerLaunch];
        for (int k = 0; k < nf; ++k) {
            ReduceArgs &r = ra[k];
            r.src = h->lvl[slots[k]][l - 1];
            r.Hs = h->Hs[l - 1];
            r.Ws = h->Ws[l - 1];
            r.spitch = h->pitch[l - 1];
            r.dst = h->lvl[slots[k]][l];
            r.Hd = h->Hs[l];
            r.Wd = h->Ws[l];
            r.dpitch = h->pitch[l];
        }
        const double bytes = nf * (double)sb * ((double)h->Hs[l - 1] * h->Ws[l - 1] + (double)h->Hs[l] * h->Ws[l]);
        ProfScope ps(h, s, OFV_K_REDUCE, bytes);
        ofv_status st = last_launch(launch_reduce_frames(ra, nf, p.storage, s), "reduce launch");
        if (st != OFV_OK) return st;
    }
    return OFV_OK;
}

// Steps 3-6 for np pairs: pair k uses pyramid slots s1[k], s2[k], field
// buffers vbuf[2k], vbuf[2k+1], and writes u[k], v[k].  With iu, iv (warm
// start) pair k starts its coarsest level from the level-0 field iu[k],
// iv[k] (H x W dense) decimated to that level, else from zero.
ofv_status run_levels(ofv_handle *h, int np, const int *s1, const int *s2, float *const *u, float *const *v,
                      cudaStream_t s, int vset = 0, const float *const *iu = nullptr, const float *const *iv = nullptr)
{
    const ofv_params &p = h->p;
    const int sb = store_bytes(p.storage);
    float2 *const *vbuf = h->vbuf + 2 * h->B * vset;
    int cur = 0;  // vbuf[2k + cur] holds the latest field of pair k
    bool have = false;
    if (iu && iv) {
        SeedArgs sa[kMaxBatch];
        for (int k = 0; k < np; ++k) {
            sa[k].u = iu[k];
            sa[k].v = iv[k];
            sa[k].W0 = h->W;
            sa[k].level = h->L - 1;
            sa[k].out = vbuf[2 * k];
            sa[k].H = h->Hs[h->L - 1];
            sa[k].W = h->Ws[h->L - 1];
            sa[k].vpitch = h->vpitch;
        }
        ofv_status st = last_launch(launch_seed_fields(sa, np, s), "warm-start field launch");
        if (st != OFV_OK) return st;
        have = true;  // vbuf[2k + 0] holds the starting field
    }
    // NVTX ranges name each level's launches for profilers (no cost without one)
    static const char *const kLevelRange[kMaxLevels] = {
        "ofv level 0", "ofv level 1", "ofv level 2", "ofv level 3", "ofv level 4", "ofv level 5",
        "ofv level 6", "ofv level 7", "ofv level 8", "ofv level 9", "ofv level 10", "ofv level 11",
        "ofv level 12", "ofv level 13", "ofv level 14", "ofv level 15"};
    for (int l = h->L - 1; l >= 0; --l) {
        nvtxRangePushA(kLevelRange[l]);
        struct RangePop {
            ~RangePop() { nvtxRangePop(); }
        } pop_at_level_end;
        for (int t = 0; t < p.iterations; ++t) {
            int mode;
            if (t == 0 && l == h->L - 1) mode = have ? V0_SAME : V0_ZERO;
            else if (t == 0) mode = V0_UP;
            else mode = V0_SAME;
            const bool last = (l == 0 && t == p.iterations - 1);
            const int nxt = have ? 1 - cur : 0;
            IterArgs a[kMaxBatch];
            for (int k = 0; k < np; ++k) {
                IterArgs &x = a[k];
                memset(&x, 0, sizeof x);
                x.P1 = h->lvl[s1[k]][l];
                x.P2 = h->lvl[s2[k]][l];
                x.H = h->Hs[l];
                x.W = h->Ws[l];
                x.pitch = h->pitch[l];
                x.vpitch = h->vpitch;
                x.vcpitch = h->vpitch;
                x.kr = p.kernel_radius;
                x.eps_rel = p.det_rel_eps;
                x.eps_abs = p.det_abs_eps;
                set_iter_variant(x, p.kernel_radius, p.window == OFV_WINDOW_GAUSS, p.window_sigma, p.increment_form);
                x.mask = h->mask_on ? h->mask_lvl[l] : nullptr;
                if (mode == V0_UP) {
                    x.Vc = vbuf[2 * k + cur];
                    x.Hc = h->Hs[l + 1];
                    x.Wc = h->Ws[l + 1];
                } else if (mode == V0_SAME) {
                    x.V0 = vbuf[2 * k + cur];
                }
                if (last) {
                    x.u_out = u[k];
                    x.v_out = v[k];
                } else {
                    x.Vout = vbuf[2 * k + nxt];
                }
            }
            const double Nl = (double)h->Hs[l] * h->Ws[l];
            const double vread = mode == V0_SAME ? 8.0 * Nl
                                 : mode == V0_UP ? 8.0 * (double)h->Hs[l + 1] * h->Ws[l + 1]
                                                 : 0.0;
            const double bytes = np * (2.0 * sb * Nl + 8.0 * Nl + vread);
            ProfScope ps(h, s, OFV_K_ITERATE, bytes);
            cudaError_t e = cudaSuccess;
            if (p.path == OFV_PATH_FUSED && block_supports(p.kernel_radius)) {
                const CUtensorMap *tm[2 * kMaxBatch];
                for (int k = 0; k < np; ++k) {
                    tm[2 * k] = &h->tmap[s1[k]][l];
                    tm[2 * k + 1] = &h->tmap[s2[k]][l];
                }
                const bool use = h->tma_ok[l] && h->tma_err_d;
                e = launch_iter_block(a, np, p.storage, mode, s, use ? tm : nullptr, h->tma_err_d, 0, 0,
                                      tile_shape_of(p));
            } else {
                for (int k = 0; k < np && e == cudaSuccess; ++k)
                    e = p.path == OFV_PATH_PLAIN ? launch_iter_plain(a[k], h->plain, p.storage, mode, s)
                                                 : launch_iter_fused(a[k], p.storage, mode, s);
            }
            ofv_status st = last_launch(e, "iteration launch");
            if (st != OFV_OK) return st;
            cur = nxt;
            have = true;
        }
    }
    return OFV_OK;
}

// The groups of a time-resolved sequence: group g holds pairs f0 .. f0+np-1
// (frames f0 .. f0+np, f0 = g B).  Frame f lives in pyramid slot f mod NS;
// group g ingests its frames except f0, whose pyramid group g-1 built.
//
// With K group streams (NS = K B + 1), group g runs on stream g mod K with
// field buffers and pre-filter scratch of that stream, so the coarse levels
// of one group overlap the fine levels of the others.  Group g waits for
// the pyramids of group g-1 (frame f0) before its iterations, and before
// ingesting for group g-K-1, whose last frame's slot it reuses (the other
// reused slots belong to group g-K, which ran before it on its own stream).
// One stream: everything in order on the caller's stream (also while kernel
// timing is on, so that launch events time single kernels).
struct GroupRunner {
    ofv_handle *h;
    cudaStream_t s;
    int K;  // group streams in use (1: the caller's stream)
    int last = -1;
    GroupRunner(ofv_handle *h_, cudaStream_t s_) : h(h_), s(s_), K(h_->prof ? 1 : h_->nstreams) {}

    cudaStream_t stream_of(int g) const { return K > 1 ? h->gs[g % K] : s; }
    static int ev(int g) { return g & (kGroupEvents - 1); }

    ofv_status begin()
    {
        if (K == 1) return OFV_OK;
        cudaError_t e = cudaEventRecord(h->gstart, s);
        for (int k = 0; k < K && e == cudaSuccess; ++k) e = cudaStreamWaitEvent(h->gs[k], h->gstart, 0);
        return e == cudaSuccess ? OFV_OK : cuda_fail(e, "ordering the group streams");
    }

    // fr[k] = frame f0 + k (k = 0 .. np), device pointers; before_ingest
    // (optional) is an event the group's stream waits for first.  iu, iv
    // (warm start): pair k starts from the level-0 field iu[k], iv[k], which
    // group g-lag wrote; the iterations then wait for group g-lag (lag <= 7,
    // within the event ring).
    ofv_status group(int g, int f0, int np, const void *const *fr, float *const *uu, float *const *vv,
                     cudaEvent_t before_ingest = nullptr, const float *const *iu = nullptr,
                     const float *const *iv = nullptr, int lag = 1)
    {
        const int NS = h->nslots;
        cudaStream_t cs = stream_of(g);
        cudaError_t e = cudaSuccess;
        if (K > 1 && g >= K + 1) e = cudaStreamWaitEvent(cs, h->gev[ev(g - K - 1)][1], 0);
        if (e == cudaSuccess && before_ingest) e = cudaStreamWaitEvent(cs, before_ingest, 0);
        if (e != cudaSuccess) return cuda_fail(e, "ordering a group");
        const void *nfr[kMaxSlots];
        int slots[kMaxSlots];
        int nf = 0;
        for (int f = (f0 == 0 ? 0 : f0 + 1); f <= f0 + np; ++f) {
            nfr[nf] = fr[f - f0];
            slots[nf] = f % NS;
            ++nf;
        }
        ofv_status st = build_pyramids(h, nfr, slots, nf, cs, g % K);
        if (st != OFV_OK) return st;
        if (K > 1) {
            e = cudaEventRecord(h->gev[ev(g)][0], cs);
            if (e == cudaSuccess && g >= 1) e = cudaStreamWaitEvent(cs, h->gev[ev(g - 1)][0], 0);
            if (e != cudaSuccess) return cuda_fail(e, "ordering a group");
        }
        if (K > 1 && iu && g >= lag) {
            e = cudaStreamWaitEvent(cs, h->gev[ev(g - lag)][1], 0);
            if (e != cudaSuccess) return cuda_fail(e, "ordering a warm-started group");
        }
        int s1[kMaxBatch], s2[kMaxBatch];
        for (int k = 0; k < np; ++k) {
            s1[k] = (f0 + k) % NS;
            s2[k] = (f0 + k + 1) % NS;
        }
        st = run_levels(h, np, s1, s2, uu, vv, cs, g % K, iu, iv);
        if (st != OFV_OK) return st;
        if (K > 1) {
            e = cudaEventRecord(h->gev[ev(g)][1], cs);
            if (e != cudaSuccess) return cuda_fail(e, "ordering a group");
        }
        h->last_s1 = s1[np - 1];
        h->last_s2 = s2[np - 1];
        last = g;
        return OFV_OK;
    }

    // the caller's stream waits for the last K groups
    ofv_status end()
    {
        if (K == 1 || last < 0) return OFV_OK;
        cudaError_t e = cudaSuccess;
        for (int g = last; g >= 0 && g > last - K && e == cudaSuccess; --g)
            e = cudaStreamWaitEvent(s, h->gev[ev(g)][1], 0);
        return e == cudaSuccess ? OFV_OK : cuda_fail(e, "joining the group streams");
    }
};

// Pairs per group of a sequence and, with a warm start from the pair d
// steps back, how many groups back that pair lies (it is then pair k of
// group g - lag): d <= B gives groups of d pairs and lag 1; a multiple d of
// B (with allow_lag, up to 7 B) keeps groups of B and a lag of d / B groups,
// so the groups in between overlap as without a warm start.
ofv_status group_size(const ofv_handle *h, int *gb, int *lag, bool allow_lag)
{
    const int d = h->p.warm_start;
    *lag = 1;
    if (d <= h->B) {
        *gb = d > 0 ? d : h->B;
        return OFV_OK;
    }
    if (!allow_lag || d % h->B != 0 || d / h->B > 7)
        return fail(OFV_ERR_INVALID_ARG,
                    "warm_start=%d: needs d <= %d (the pairs per launch)%s", d, h->B,
                    allow_lag ? " or a multiple of it up to 7 times" : " for a sequence from host memory");
    *gb = h->B;
    *lag = d / h->B;
    return OFV_OK;
}

ofv_status pending_error(const ofv_handle *h, const char *where)
{
    if (tma_expired(h)) return fail(OFV_ERR_TIMEOUT, "%s: a TMA copy of an earlier launch did not complete", where);
    cudaError_t e = cudaPeekAtLastError();
    if (e != cudaSuccess) {
        cudaGetLastError();
        return cuda_fail(e, where);
    }
    return OFV_OK;
}

}  // namespace

namespace ofv {
namespace {
std::atomic<int> g_fail_alloc{0};  // > 0: that many allocations from now, the last one fails
}

cudaError_t dev_alloc(void **p, size_t bytes)
{
    int n = g_fail_alloc.load();
    while (n > 0 && !g_fail_alloc.compare_exchange_weak(n, n - 1)) {
    }
    if (n == 1) {
        *p = nullptr;
        return cudaErrorMemoryAllocation;
    }
    return cudaMalloc(p, bytes);
}

// Record a failure message for ofv_last_error() from another translation unit.
void set_error_message(const char *msg) { fail(OFV_OK, "%s", msg); }

ofv_status fail_msg(ofv_status st, const char *fmt, ...)
{
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(g_err, sizeof g_err, fmt, ap);
    va_end(ap);
    return st;
}

ofv_status cuda_fail_msg(cudaError_t e, const char *where) { return cuda_fail(e, where); }

ofv_status handle_pyramids(ofv_handle *h, const void *const *frames, const int *slots, int nf, cudaStream_t s)
{
    return build_pyramids(h, frames, slots, nf, s);
}

// 2-D tensor map of a level image (W x H elements of the storage type, row
// stride pitch elements) with the block kernel's TMA box for radius kr; no
// swizzle, out-of-bounds fill unused (only boxes inside the image are
// copied).  False when the encoder is unavailable or refuses.
bool encode_block_map(CUtensorMap *m, const void *base, int W, int H, int pitch, int store, int kr, int shape)
{
    PFN_cuTensorMapEncodeTiled_v12000 enc = tensor_map_encoder_impl();
    int cols = 0, rows = 0;
    block_stage_box(store, kr, &cols, &rows, shape);
    if (!enc || cols < 1) return false;
    const CUtensorMapDataType dt = store == OFV_STORE_F16    ? CU_TENSOR_MAP_DATA_TYPE_FLOAT16
                                   : store == OFV_STORE_BF16 ? CU_TENSOR_MAP_DATA_TYPE_BFLOAT16
                                                             : CU_TENSOR_MAP_DATA_TYPE_FLOAT32;
    const cuuint64_t dim[2] = {(cuuint64_t)W, (cuuint64_t)H};
    const cuuint64_t stride[1] = {(cuuint64_t)pitch * store_bytes(store)};
    const cuuint32_t box[2] = {(cuuint32_t)cols, (cuuint32_t)rows};
    const cuuint32_t estr[2] = {1, 1};
    return enc(m, dt, 2, const_cast<void *>(base), dim, stride, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
               CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
               CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}
}  // namespace ofv

extern "C" {

void ofv_default_params(ofv_params *p)
{
    if (!p) return;
    p->levels_psl = 2;
    p->kernel_radius = 4;
    p->iterations = 3;
    p->norm_radius = 0;
    p->input = OFV_IN_U16;
    p->bit_depth = 12;
    p->storage = OFV_STORE_F32;
    p->path = OFV_PATH_FUSED;
    p->prefilter = 0;
    p->det_rel_eps = 1e-6f;
    p->det_abs_eps = 1e-20f;
    p->norm_eps = 1e-2f;
    p->max_batch = 0;
    p->window = OFV_WINDOW_BOX;
    p->window_sigma = 0.f;
    p->increment_form = 0;
    p->warm_start = 0;
    p->tile_edge = 0;
}

ofv_status ofv_create(int H, int W, const ofv_params *p, ofv_handle **out)
{
    if (!out) return fail(OFV_ERR_INVALID_ARG, "out is NULL");
    *out = nullptr;
    ofv_status st = check_params(p);
    if (st != OFV_OK) return st;
    if (H < 1 || W < 1) return fail(OFV_ERR_SHAPE, "H=%d W=%d must be positive", H, W);
    if ((int64_t)H * W > 2147483647LL) return fail(OFV_ERR_SHAPE, "H*W=%lld exceeds 2^31-1", (long long)H * W);
    const int L = p->levels_psl + 1;
    int Hs[kMaxLevels], Ws[kMaxLevels];
    Hs[0] = H;
    Ws[0] = W;
    for (int l = 1; l < L; ++l) {
        Hs[l] = (Hs[l - 1] + 1) / 2;
        Ws[l] = (Ws[l - 1] + 1) / 2;
    }
    const int minsz = 2 * p->kernel_radius + 1 > 8 ? 2 * p->kernel_radius + 1 : 8;
    if (Hs[L - 1] < minsz || Ws[L - 1] < minsz)
        return fail(OFV_ERR_SHAPE, "coarsest level %dx%d is below max(8, 2KR+1)=%d (H=%d W=%d PSL=%d KR=%d)",
                    Hs[L - 1], Ws[L - 1], minsz, H, W, p->levels_psl, p->kernel_radius);

    ofv_handle *h = new (std::nothrow) ofv_handle();
    if (!h) return fail(OFV_ERR_ALLOC, "host allocation of the handle failed");
    h->H = H;
    h->W = W;
    h->p = *p;
    h->L = L;
    // pairs per launch: enough pixels per launch (~16 Mp) to fill the GPU at
    // the coarse levels, within the workspace that costs
    if (p->max_batch > 0) {
        h->B = p->max_batch;
    } else {
        const long long b = (16LL << 20) / ((long long)H * W);
        h->B = (int)(b < 1 ? 1 : (b > kMaxBatch ? kMaxBatch : b));
    }
    // several streams for the groups of a sequence (fused path): the coarse
    // levels of one group overlap the finer levels of the others
    h->nstreams = p->path == OFV_PATH_FUSED ? kGroupStreams : 1;
    h->nslots = h->nstreams * h->B + 1;
    if (cudaGetDevice(&h->device) != cudaSuccess) {
        delete h;
        return fail(OFV_ERR_CUDA, "cudaGetDevice failed");
    }
    for (int l = 0; l < L; ++l) {
        h->Hs[l] = Hs[l];
        h->Ws[l] = Ws[l];
        h->pitch[l] = pitch_for(Ws[l]);
    }
    h->vpitch = pitch_for(W);
    const int sb = store_bytes(p->storage);

    // arena layout
    size_t off = 0;
    size_t lvl_off[kMaxSlots][kMaxLevels];
    for (int f = 0; f < h->nslots; ++f)
        for (int l = 0; l < L; ++l) {
            lvl_off[f][l] = off;
            off = align_up(off + (size_t)Hs[l] * h->pitch[l] * sb, 256);
        }
    size_t vb_off[2 * kGroupStreams * kMaxBatch];
    for (int k = 0; k < 2 * h->B * h->nstreams; ++k) {
        vb_off[k] = off;
        off = align_up(off + (size_t)H * h->vpitch * sizeof(float2), 256);
    }
    const size_t w_off = off;
    off = align_up(off + 25 * sizeof(float), 256);
    size_t tmp_off[kGroupStreams * kMaxFramesPerLaunch] = {};
    if (p->prefilter)
        for (int k = 0; k < (h->B + 1) * h->nstreams; ++k) {
            tmp_off[k] = off;
            off = align_up(off + (size_t)H * h->pitch[0] * sizeof(float), 256);
        }
    size_t prod_off = 0, hsum_off = 0, vtmp_off = 0;
    const size_t plane = (size_t)H * h->pitch[0];
    if (p->path == OFV_PATH_PLAIN) {
        prod_off = off;
        off = align_up(off + 5 * plane * sizeof(float), 256);
        hsum_off = off;
        off = align_up(off + 5 * plane * sizeof(float), 256);
        vtmp_off = off;
        off = align_up(off + (size_t)H * h->vpitch * sizeof(float2), 256);
    }
    h->arena_bytes = off;
    cudaError_t e = dev_alloc(&h->arena, off);
    if (e != cudaSuccess) {
        cudaGetLastError();
        delete h;
        return fail(OFV_ERR_ALLOC, "cudaMalloc of %zu workspace bytes failed: %s", off, cudaGetErrorString(e));
    }
    char *base = static_cast<char *>(h->arena);
    for (int f = 0; f < h->nslots; ++f)
        for (int l = 0; l < L; ++l) h->lvl[f][l] = base + lvl_off[f][l];
    for (int k = 0; k < 2 * h->B * h->nstreams; ++k) h->vbuf[k] = reinterpret_cast<float2 *>(base + vb_off[k]);
    h->w25 = reinterpret_cast<float *>(base + w_off);
    for (int t = 0; t < h->nstreams; ++t)
        for (int k = 0; k <= h->B; ++k)
            h->tmp[t * kMaxFramesPerLaunch + k] =
                p->prefilter ? reinterpret_cast<float *>(base + tmp_off[t * (h->B + 1) + k]) : nullptr;
    if (p->path == OFV_PATH_PLAIN) {
        h->plain.prod = reinterpret_cast<float *>(base + prod_off);
        h->plain.hsum = reinterpret_cast<float *>(base + hsum_off);
        h->plain.vtmp = reinterpret_cast<float2 *>(base + vtmp_off);
        h->plain.plane = plane;
    }
    float ident[25] = {0};
    ident[12] = 1.f;
    e = cudaMemcpy(h->w25, ident, sizeof ident, cudaMemcpyHostToDevice);
    if (e != cudaSuccess) {
        cudaFree(h->arena);
        delete h;
        return cuda_fail(e, "initialising the pre-filter weights");
    }
    h->last_s1 = 0;
    h->last_s2 = 1;
    if (h->nstreams > 1) {
        for (int k = 0; k < h->nstreams && e == cudaSuccess; ++k)
            e = cudaStreamCreateWithFlags(&h->gs[k], cudaStreamNonBlocking);
        for (int r = 0; r < kGroupEvents && e == cudaSuccess; ++r)
            for (int k = 0; k < 2 && e == cudaSuccess; ++k)
                e = cudaEventCreateWithFlags(&h->gev[r][k], cudaEventDisableTiming);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&h->gstart, cudaEventDisableTiming);
        if (e != cudaSuccess) {
            cudaGetLastError();
            ofv_destroy(h);  // frees what was made
            return fail(OFV_ERR_CUDA, "creating the group streams");
        }
    }
    if (p->path == OFV_PATH_FUSED && block_supports(p->kernel_radius)) {
        // TMA staging of interior tiles: the error word and one tensor map
        // per (slot, level); a level whose map cannot be made keeps cp.async
        if (cudaHostAlloc(reinterpret_cast<void **>(&h->tma_err_h), sizeof(int), cudaHostAllocMapped) == cudaSuccess &&
            cudaHostGetDevicePointer(reinterpret_cast<void **>(&h->tma_err_d), h->tma_err_h, 0) == cudaSuccess) {
            *h->tma_err_h = 0;
            encode_tensor_maps(h);
        } else {
            cudaGetLastError();
            if (h->tma_err_h) cudaFreeHost(h->tma_err_h);
            h->tma_err_h = h->tma_err_d = nullptr;
        }
    }
    *out = h;
    return OFV_OK;
}

ofv_status ofv_destroy(ofv_handle *h)
{
    if (!h) return OFV_OK;
    DeviceGuard g(h->device);
    ofv_status st = OFV_OK;
    cudaError_t e = cudaDeviceSynchronize();
    if (e != cudaSuccess) st = cuda_fail(e, "synchronising before destroy");
    for (cudaEvent_t ev : h->pool) cudaEventDestroy(ev);
    if (h->stage) cudaFree(h->stage);
    if (h->batch_arena) cudaFree(h->batch_arena);
    if (h->bw_arena) cudaFree(h->bw_arena);
    if (h->strip_arena) cudaFree(h->strip_arena);
    if (h->tma_err_h) cudaFreeHost(h->tma_err_h);
    for (int k = 0; k < kGroupStreams; ++k)
        if (h->gs[k]) cudaStreamDestroy(h->gs[k]);
    for (int r = 0; r < kGroupEvents; ++r)
        for (int k = 0; k < 2; ++k)
            if (h->gev[r][k]) cudaEventDestroy(h->gev[r][k]);
    if (h->gstart) cudaEventDestroy(h->gstart);
    if (h->hs_stage) cudaFree(h->hs_stage);
    if (h->hs_ready) {
        for (int r = 0; r < kHostRing; ++r)
            for (int k = 0; k < 3; ++k) cudaEventDestroy(h->hs_ev[r][k]);
        cudaStreamDestroy(h->hs_stream[0]);
        cudaStreamDestroy(h->hs_stream[1]);
    }
    if (h->mask_arena) cudaFree(h->mask_arena);
    if (h->qerr_h) cudaFreeHost(h->qerr_h);
    if (h->arena) cudaFree(h->arena);
    delete h;
    return st;
}

void ofv_debug_fail_alloc(int n) { g_fail_alloc.store(n > 0 ? n : 0); }

ofv_status ofv_debug_reciprocal(const float *x, float *y, int n, ofv_stream_t s)
{
    if (n < 0 || (n > 0 && (!x || !y))) return fail_msg(OFV_ERR_INVALID_ARG, "ofv_debug_reciprocal: bad arguments");
    const cudaError_t e = launch_recip(x, y, n, (cudaStream_t)s);
    return e == cudaSuccess ? OFV_OK : cuda_fail_msg(e, "ofv_debug_reciprocal");
}

ofv_status ofv_debug_poison(ofv_handle *h, ofv_stream_t s)
{
    if (!h) return fail(OFV_ERR_INVALID_ARG, "handle is NULL");
    DeviceGuard g(h->device);
    if (!g.ok) return fail(OFV_ERR_CUDA, "cannot select the handle's device");
    cudaStream_t cs = (cudaStream_t)s;
    char *base = static_cast<char *>(h->arena);
    const size_t w0 = reinterpret_cast<char *>(h->w25) - base, w1 = align_up(w0 + 25 * sizeof(float), 256);
    cudaError_t e = cudaMemsetAsync(base, 0xFF, w0, cs);  // all-ones bytes: NaN in every float
    if (e == cudaSuccess && h->arena_bytes > w1) e = cudaMemsetAsync(base + w1, 0xFF, h->arena_bytes - w1, cs);
    if (e == cudaSuccess && h->stage) e = cudaMemsetAsync(h->stage, 0xFF, h->stage_bytes, cs);
    if (e == cudaSuccess && h->hs_stage) e = cudaMemsetAsync(h->hs_stage, 0xFF, h->hs_bytes, cs);
    if (e == cudaSuccess && h->bw_arena) e = cudaMemsetAsync(h->bw_arena, 0xFF, h->bw_bytes, cs);
    if (e == cudaSuccess && h->strip_arena) e = cudaMemsetAsync(h->strip_arena, 0xFF, h->strip_bytes, cs);
    if (e == cudaSuccess && h->batch_arena) e = cudaMemsetAsync(h->batch_arena, 0xFF, h->batch_bytes, cs);
    h->batch_sched_key.clear();  // the schedule and tensor maps in the batch arena are gone
    h->batch_maps_key.clear();
    return e == cudaSuccess ? OFV_OK : cuda_fail(e, "poisoning the workspace");
}

ofv_status ofv_set_mask(ofv_handle *h, const uint8_t *mask, ofv_stream_t s)
{
    if (!h) return fail(OFV_ERR_INVALID_ARG, "handle is NULL");
    DeviceGuard g(h->device);
    if (!g.ok) return fail(OFV_ERR_CUDA, "cannot select the handle's device");
    if (!mask) {
        h->mask_on = 0;
        return OFV_OK;
    }
    if (!h->mask_arena) {
        size_t off[kMaxLevels], total = 0;
        for (int l = 0; l < h->L; ++l) {
            off[l] = total;
            total += align_up((size_t)h->Hs[l] * h->Ws[l], 256);
        }
        if (dev_alloc(&h->mask_arena, total) != cudaSuccess) {
            cudaGetLastError();
            h->mask_arena = nullptr;
            return fail(OFV_ERR_ALLOC, "cudaMalloc of %zu mask bytes failed", total);
        }
        for (int l = 0; l < h->L; ++l) h->mask_lvl[l] = static_cast<uint8_t *>(h->mask_arena) + off[l];
    }
    cudaError_t e = launch_mask_levels(mask, h->W, h->mask_lvl, h->Hs, h->Ws, h->L, (cudaStream_t)s);
    if (e != cudaSuccess) return cuda_fail(e, "mask level launch");
    h->mask_on = 1;
    return OFV_OK;
}

ofv_status ofv_set_prefilter(ofv_handle *h, const float *w25, ofv_stream_t s)
{
    if (!h || !w25) return fail(OFV_ERR_INVALID_ARG, "handle or weights is NULL");
    DeviceGuard g(h->device);
    cudaError_t e = cudaMemcpyAsync(h->w25, w25, 25 * sizeof(float), cudaMemcpyDeviceToDevice, (cudaStream_t)s);
    if (e != cudaSuccess) return cuda_fail(e, "copying pre-filter weights");
    return OFV_OK;
}

ofv_status ofv_compute(ofv_handle *h, const void *I1, const void *I2, float *u, float *v, ofv_stream_t s)
{
    if (!h) return fail(OFV_ERR_INVALID_ARG, "handle is NULL");
    if (!I1 || !I2 || !u || !v) return fail(OFV_ERR_INVALID_ARG, "I1, I2, u and v must be non-NULL");
    if (u == v) return fail(OFV_ERR_INVALID_ARG, "u and v must be distinct buffers");
    DeviceGuard g(h->device);
    if (!g.ok) return fail(OFV_ERR_CUDA, "cannot select the handle's device");
    ofv_status st = pending_error(h, "error pending before ofv_compute");
    if (st != OFV_OK) return st;
    cudaStream_t cs = (cudaStream_t)s;
    const void *fr[2] = {I1, I2};
    const int slots[2] = {0, 1};
    st = build_pyramids(h, fr, slots, 2, cs);
    if (st != OFV_OK) return st;
    h->last_s1 = 0;
    h->last_s2 = 1;
    const int s1[1] = {0}, s2[1] = {1};
    float *uu[1] = {u}, *vv[1] = {v};
    return run_levels(h, 1, s1, s2, uu, vv, cs);
}

ofv_status ofv_compute_host(ofv_handle *h, const void *I1, const void *I2, float *u, float *v, ofv_stream_t s)
{
    if (!h) return fail(OFV_ERR_INVALID_ARG, "handle is NULL");
    if (!I1 || !I2 || !u || !v) return fail(OFV_ERR_INVALID_ARG, "I1, I2, u and v must be non-NULL");
    DeviceGuard g(h->device);
    if (!g.ok) return fail(OFV_ERR_CUDA, "cannot select the handle's device");
    const size_t N = (size_t)h->H * h->W;
    const size_t in_b = align_up(N * input_bytes(h->p.input), 256);
    const size_t out_b = align_up(N * sizeof(float), 256);
    const size_t need = 2 * in_b + 2 * out_b;
    if (!h->stage) {
        cudaError_t e = dev_alloc(&h->stage, need);
        if (e != cudaSuccess) {
            cudaGetLastError();
            h->stage = nullptr;
            return fail(OFV_ERR_ALLOC, "cudaMalloc of %zu staging bytes failed", need);
        }
        h->stage_bytes = need;
    }
    char *b = static_cast<char *>(h->stage);
    void *d1 = b, *d2 = b + in_b;
    float *du = reinterpret_cast<float *>(b + 2 * in_b), *dv = reinterpret_cast<float *>(b + 2 * in_b + out_b);
    cudaStream_t cs = (cudaStream_t)s;
    const size_t ib = N * input_bytes(h->p.input);
    cudaError_t e = cudaMemcpyAsync(d1, I1, ib, cudaMemcpyHostToDevice, cs);
    if (e == cudaSuccess) e = cudaMemcpyAsync(d2, I2, ib, cudaMemcpyHostToDevice, cs);
    if (e != cudaSuccess) return cuda_fail(e, "host-to-device copy of the frames");
    ofv_status st = ofv_compute(h, d1, d2, du, dv, s);
    if (st != OFV_OK) return st;
    e = cudaMemcpyAsync(u, du, N * sizeof(float), cudaMemcpyDeviceToHost, cs);
    if (e == cudaSuccess) e = cudaMemcpyAsync(v, dv, N * sizeof(float), cudaMemcpyDeviceToHost, cs);
    if (e != cudaSuccess) return cuda_fail(e, "device-to-host copy of the field");
    return OFV_OK;
}

ofv_status ofv_compute_sequence(ofv_handle *h, int n_frames, const void *frames, size_t frame_stride_bytes,
                                float *u, float *v, size_t field_stride, ofv_stream_t s)
{
    if (!h) return fail(OFV_ERR_INVALID_ARG, "handle is NULL");
    if (!frames || !u || !v) return fail(OFV_ERR_INVALID_ARG, "frames, u and v must be non-NULL");
    if (n_frames < 2) return fail(OFV_ERR_INVALID_ARG, "n_frames=%d must be >= 2", n_frames);
    const size_t N = (size_t)h->H * h->W;
    if (frame_stride_bytes < N * input_bytes(h->p.input))
        return fail(OFV_ERR_INVALID_ARG, "frame_stride_bytes=%zu is smaller than one frame", frame_stride_bytes);
    if (field_stride < N) return fail(OFV_ERR_INVALID_ARG, "field_stride=%zu is smaller than one field", field_stride);
    DeviceGuard g(h->device);
    if (!g.ok) return fail(OFV_ERR_CUDA, "cannot select the handle's device");
    ofv_status st = pending_error(h, "error pending before ofv_compute_sequence");
    if (st != OFV_OK) return st;
    cudaStream_t cs = (cudaStream_t)s;
    const char *fb = static_cast<const char *>(frames);
    const int npairs = n_frames - 1;
    int GB, lag;  // pairs per group; groups back to a warm start's source
    if ((st = group_size(h, &GB, &lag, true)) != OFV_OK) return st;
    const int d = h->p.warm_start;
    GroupRunner gr(h, cs);
    if ((st = gr.begin()) != OFV_OK) return st;
    for (int f0 = 0, g = 0; f0 < npairs; f0 += GB, ++g) {
        const int np = npairs - f0 < GB ? npairs - f0 : GB;
        const void *fr[kMaxSlots];
        for (int f = f0; f <= f0 + np; ++f) fr[f - f0] = fb + (size_t)f * frame_stride_bytes;
        float *uu[kMaxBatch], *vv[kMaxBatch];
        const float *iu[kMaxBatch], *iv[kMaxBatch];
        for (int k = 0; k < np; ++k) {
            uu[k] = u + (size_t)(f0 + k) * field_stride;
            vv[k] = v + (size_t)(f0 + k) * field_stride;
            if (d > 0 && f0 >= d) {  // pair f0+k-d is pair k of group g-lag
                iu[k] = u + (size_t)(f0 + k - d) * field_stride;
                iv[k] = v + (size_t)(f0 + k - d) * field_stride;
            }
        }
        const bool warm = d > 0 && f0 >= d;
        if ((st = gr.group(g, f0, np, fr, uu, vv, nullptr, warm ? iu : nullptr, warm ? iv : nullptr, lag)) !=
            OFV_OK)
            return st;
    }
    return gr.end();
}

ofv_status ofv_compute_sequence_host(ofv_handle *h, int n_frames, const void *frames, size_t frame_stride_bytes,
                                     float *u, float *v, size_t field_stride, ofv_stream_t s)
{
    if (!h) return fail(OFV_ERR_INVALID_ARG, "handle is NULL");
    if (!frames || !u || !v) return fail(OFV_ERR_INVALID_ARG, "frames, u and v must be non-NULL");
    if (u == v) return fail(OFV_ERR_INVALID_ARG, "u and v must be distinct buffers");
    if (n_frames < 2) return fail(OFV_ERR_INVALID_ARG, "n_frames=%d must be >= 2", n_frames);
    const size_t N = (size_t)h->H * h->W;
    const size_t fb = N * input_bytes(h->p.input);
    if (frame_stride_bytes < fb)
        return fail(OFV_ERR_INVALID_ARG, "frame_stride_bytes=%zu is smaller than one frame", frame_stride_bytes);
    if (field_stride < N) return fail(OFV_ERR_INVALID_ARG, "field_stride=%zu is smaller than one field", field_stride);
    DeviceGuard g(h->device);
    if (!g.ok) return fail(OFV_ERR_CUDA, "cannot select the handle's device");
    ofv_status st = pending_error(h, "error pending before ofv_compute_sequence_host");
    if (st != OFV_OK) return st;
    cudaStream_t cs = (cudaStream_t)s;
    int B, lag;  // pairs per group; the warm start's source is the previous group (lag 1)
    if ((st = group_size(h, &B, &lag, false)) != OFV_OK) return st;
    const int d = h->p.warm_start;
    // device ring: per slot B+1 frames and B fields (u and v)
    const size_t in_b = align_up(fb * (size_t)(B + 1), 256);
    const size_t out_b = align_up(N * sizeof(float) * (size_t)B, 256);
    const size_t slot_b = in_b + 2 * out_b;
    const size_t need = slot_b * kHostRing;
    if (!h->hs_ready) {
        cudaError_t e = cudaStreamCreateWithFlags(&h->hs_stream[0], cudaStreamNonBlocking);
        if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&h->hs_stream[1], cudaStreamNonBlocking);
        for (int r = 0; r < kHostRing && e == cudaSuccess; ++r)
            for (int k = 0; k < 3 && e == cudaSuccess; ++k)
                e = cudaEventCreateWithFlags(&h->hs_ev[r][k], cudaEventDisableTiming);
        if (e != cudaSuccess) return cuda_fail(e, "creating the copy streams");
        h->hs_ready = 1;
    }
    if (need > h->hs_bytes) {
        if (h->hs_stage) {
            cudaError_t e = cudaDeviceSynchronize();
            if (e != cudaSuccess) return cuda_fail(e, "waiting before growing the host pipeline ring");
            cudaFree(h->hs_stage);
            h->hs_stage = nullptr;
            h->hs_bytes = 0;
        }
        if (dev_alloc(&h->hs_stage, need) != cudaSuccess) {
            cudaGetLastError();
            h->hs_stage = nullptr;
            return fail(OFV_ERR_ALLOC, "cudaMalloc of %zu ring bytes failed", need);
        }
        h->hs_bytes = need;
    }
    cudaStream_t up = h->hs_stream[0], down = h->hs_stream[1];
    const char *hf = static_cast<const char *>(frames);
    const int npairs = n_frames - 1;
    // The copy streams start after the work already queued on s.
    cudaError_t e = cudaEventRecord(h->hs_ev[0][1], cs);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(up, h->hs_ev[0][1], 0);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(down, h->hs_ev[0][1], 0);
    if (e != cudaSuccess) return cuda_fail(e, "ordering the copy streams");
    // Group c (pairs c*B .. c*B+np-1) uses ring slot c mod kHostRing: its
    // new frames go up on stream `up`, the group runs on its group stream
    // (GroupRunner), its fields come down on stream `down`.  A slot is
    // reused once the group that last used it has finished (frames) and
    // gone down (fields).
    GroupRunner gr(h, cs);
    if ((st = gr.begin()) != OFV_OK) return st;
    int c = 0;
    for (int f0 = 0; f0 < npairs; f0 += B, ++c) {
        const int r = c % kHostRing;
        const int np = npairs - f0 < B ? npairs - f0 : B;
        char *slot = static_cast<char *>(h->hs_stage) + (size_t)r * slot_b;
        float *du = reinterpret_cast<float *>(slot + in_b), *dv = reinterpret_cast<float *>(slot + in_b + out_b);
        const int fa = f0 == 0 ? 0 : f0 + 1, fz = f0 + np;  // frames to ingest
        if (c >= kHostRing) {
            e = cudaStreamWaitEvent(up, h->hs_ev[r][1], 0);  // group c - kHostRing done
            if (e != cudaSuccess) return cuda_fail(e, "ordering the frame upload");
        }
        if (frame_stride_bytes == fb) {
            e = cudaMemcpyAsync(slot, hf + (size_t)fa * fb, fb * (size_t)(fz - fa + 1), cudaMemcpyHostToDevice, up);
        } else {
            for (int f = fa; f <= fz && e == cudaSuccess; ++f)
                e = cudaMemcpyAsync(slot + (size_t)(f - fa) * fb, hf + (size_t)f * frame_stride_bytes, fb,
                                    cudaMemcpyHostToDevice, up);
        }
        cudaStream_t gsc = gr.stream_of(c);
        if (e == cudaSuccess) e = cudaEventRecord(h->hs_ev[r][0], up);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(gsc, h->hs_ev[r][0], 0);
        if (e == cudaSuccess && c >= kHostRing) e = cudaStreamWaitEvent(gsc, h->hs_ev[r][2], 0);  // fields gone down
        if (e != cudaSuccess) return cuda_fail(e, "uploading frames");
        const void *fr[kMaxSlots];
        fr[0] = nullptr;  // frame f0 > 0 is already in its pyramid slot
        for (int f = fa; f <= fz; ++f) fr[f - f0] = slot + (size_t)(f - fa) * fb;
        float *uu[kMaxBatch], *vv[kMaxBatch];
        const float *iu[kMaxBatch], *iv[kMaxBatch];
        const bool warm = d > 0 && f0 >= d;  // then groups hold d pairs: pair f0+k-d is pair k of group c-1
        char *pslot = static_cast<char *>(h->hs_stage) + (size_t)((c + kHostRing - 1) % kHostRing) * slot_b;
        for (int k = 0; k < np; ++k) {
            uu[k] = du + (size_t)k * N;
            vv[k] = dv + (size_t)k * N;
            if (warm) {
                iu[k] = reinterpret_cast<const float *>(pslot + in_b) + (size_t)k * N;
                iv[k] = reinterpret_cast<const float *>(pslot + in_b + out_b) + (size_t)k * N;
            }
        }
        if ((st = gr.group(c, f0, np, fr, uu, vv, nullptr, warm ? iu : nullptr, warm ? iv : nullptr)) != OFV_OK)
            return st;
        e = cudaEventRecord(h->hs_ev[r][1], gsc);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(down, h->hs_ev[r][1], 0);
        if (e == cudaSuccess) {
            if (field_stride == N) {
                e = cudaMemcpyAsync(u + (size_t)f0 * N, du, N * sizeof(float) * np, cudaMemcpyDeviceToHost, down);
                if (e == cudaSuccess)
                    e = cudaMemcpyAsync(v + (size_t)f0 * N, dv, N * sizeof(float) * np, cudaMemcpyDeviceToHost, down);
            } else {
                for (int k = 0; k < np && e == cudaSuccess; ++k) {
                    e = cudaMemcpyAsync(u + (size_t)(f0 + k) * field_stride, du + (size_t)k * N, N * sizeof(float),
                                        cudaMemcpyDeviceToHost, down);
                    if (e == cudaSuccess)
                        e = cudaMemcpyAsync(v + (size_t)(f0 + k) * field_stride, dv + (size_t)k * N,
                                            N * sizeof(float), cudaMemcpyDeviceToHost, down);
                }
            }
        }
        if (e == cudaSuccess) e = cudaEventRecord(h->hs_ev[r][2], down);
        if (e != cudaSuccess) return cuda_fail(e, "downloading fields");
    }
    // s reaches its end only after the last fields are in host memory
    if ((st = gr.end()) != OFV_OK) return st;
    e = cudaStreamWaitEvent(cs, h->hs_ev[(c - 1) % kHostRing][2], 0);
    if (e != cudaSuccess) return cuda_fail(e, "joining the copy streams");
    return OFV_OK;
}

}  // extern "C"

extern "C" {

ofv_status ofv_graph_create(ofv_handle *h, const void *I1, const void *I2, float *u, float *v, ofv_graph **out)
{
    if (!out) return fail(OFV_ERR_INVALID_ARG, "out is NULL");
    *out = nullptr;
    if (!h || !I1 || !I2 || !u || !v || u == v)
        return fail(OFV_ERR_INVALID_ARG, "handle, I1, I2, u, v must be non-NULL and u != v");
    DeviceGuard g(h->device);
    if (!g.ok) return fail(OFV_ERR_CUDA, "cannot select the handle's device");
    // the eager run below uses the handle's workspace and claim counters on
    // a stream of its own: earlier work on the handle must be finished
    cudaError_t e = cudaDeviceSynchronize();
    if (e != cudaSuccess) return cuda_fail(e, "waiting for earlier work before recording");
    cudaStream_t cs = nullptr;
    e = cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking);
    if (e != cudaSuccess) return cuda_fail(e, "creating the capture stream");
    const bool prof = h->prof;
    h->prof = false;
    // one eager run sets kernel attributes outside the capture
    ofv_status st = ofv_compute(h, I1, I2, u, v, (ofv_stream_t)cs);
    if (st == OFV_OK) {
        e = cudaStreamSynchronize(cs);
        if (e != cudaSuccess) st = cuda_fail(e, "warm-up run before capture");
    }
    cudaGraph_t graph = nullptr;
    if (st == OFV_OK) {
        e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
        if (e != cudaSuccess) {
            st = cuda_fail(e, "beginning stream capture");
        } else {
            st = ofv_compute(h, I1, I2, u, v, (ofv_stream_t)cs);
            e = cudaStreamEndCapture(cs, &graph);
            if (st == OFV_OK && e != cudaSuccess) st = cuda_fail(e, "ending stream capture");
        }
    }
    h->prof = prof;
    cudaGraphExec_t exec = nullptr;
    if (st == OFV_OK) {
        e = cudaGraphInstantiate(&exec, graph, 0);
        if (e != cudaSuccess) st = cuda_fail(e, "instantiating the graph");
    }
    cudaStreamDestroy(cs);
    if (st != OFV_OK) {
        if (graph) cudaGraphDestroy(graph);
        return st;
    }
    ofv_graph *gr = new (std::nothrow) ofv_graph{h, graph, exec, nullptr};
    if (!gr) {
        cudaGraphExecDestroy(exec);
        cudaGraphDestroy(graph);
        return fail(OFV_ERR_ALLOC, "host allocation of the graph handle failed");
    }
    *out = gr;
    return OFV_OK;
}

ofv_status ofv_graph_launch(ofv_graph *g, ofv_stream_t s)
{
    if (!g) return fail(OFV_ERR_INVALID_ARG, "graph is NULL");
    if (tma_expired(g->h)) return fail(OFV_ERR_TIMEOUT, "ofv_graph_launch: a TMA copy of an earlier launch did not complete");
    DeviceGuard dg(g->h->device);
    cudaError_t e = cudaGraphLaunch(g->exec, (cudaStream_t)s);
    if (e != cudaSuccess) return cuda_fail(e, "launching the graph");
    return OFV_OK;
}

ofv_status ofv_graph_destroy(ofv_graph *g)
{
    if (!g) return OFV_OK;
    DeviceGuard dg(g->h->device);
    cudaGraphExecDestroy(g->exec);
    cudaGraphDestroy(g->graph);
    if (g->arena) cudaFree(g->arena);  // waits for the graph's last launch
    delete g;
    return OFV_OK;
}

ofv_status ofv_level_shape(const ofv_handle *h, int level, int *H, int *W)
{
    if (!h || !H || !W) return fail(OFV_ERR_INVALID_ARG, "NULL argument");
    if (level < 0 || level >= h->L) return fail(OFV_ERR_INVALID_ARG, "level=%d outside 0..%d", level, h->L - 1);
    *H = h->Hs[level];
    *W = h->Ws[level];
    return OFV_OK;
}

ofv_status ofv_read_level(ofv_handle *h, int frame, int level, float *dst, ofv_stream_t s)
{
    if (!h || !dst) return fail(OFV_ERR_INVALID_ARG, "NULL argument");
    if (frame != 0 && frame != 1) return fail(OFV_ERR_INVALID_ARG, "frame=%d must be 0 or 1", frame);
    if (level < 0 || level >= h->L) return fail(OFV_ERR_INVALID_ARG, "level=%d outside 0..%d", level, h->L - 1);
    DeviceGuard g(h->device);
    const int slot = frame == 0 ? h->last_s1 : h->last_s2;
    return last_launch(launch_read_level(h->lvl[slot][level], h->Hs[level], h->Ws[level], h->pitch[level],
                                         h->p.storage, dst, (cudaStream_t)s),
                       "read_level launch");
}

ofv_status ofv_profile_enable(ofv_handle *h, int enable)
{
    if (!h) return fail(OFV_ERR_INVALID_ARG, "handle is NULL");
    DeviceGuard g(h->device);
    if (enable) {
        cudaError_t e = cudaDeviceSynchronize();
        if (e != cudaSuccess) return cuda_fail(e, "synchronising before enabling timing");
        h->recs.clear();
        h->pool_next = 0;
    }
    h->prof = enable != 0;
    return OFV_OK;
}

ofv_status ofv_profile_read(ofv_handle *h, int k, double *total_ms, int64_t *launches, double *alg_bytes)
{
    if (!h || !total_ms || !launches || !alg_bytes) return fail(OFV_ERR_INVALID_ARG, "NULL argument");
    if (k < 0 || k >= OFV_K_COUNT) return fail(OFV_ERR_INVALID_ARG, "kernel class %d outside 0..%d", k, OFV_K_COUNT - 1);
    DeviceGuard g(h->device);
    double ms = 0.0, bytes = 0.0;
    int64_t n = 0;
    for (const ProfRec &r : h->recs) {
        if (r.cls != k) continue;
        cudaError_t e = cudaEventSynchronize(r.e1);
        if (e != cudaSuccess) return cuda_fail(e, "waiting for a timing event");
        float t = 0.f;
        e = cudaEventElapsedTime(&t, r.e0, r.e1);
        if (e != cudaSuccess) return cuda_fail(e, "reading a timing event");
        ms += t;
        bytes += r.bytes;
        ++n;
    }
    *total_ms = ms;
    *launches = n;
    *alg_bytes = bytes;
    return OFV_OK;
}

const char *ofv_last_error(void) { return g_err; }

const char *ofv_status_string(ofv_status s)
{
    switch (s) {
    case OFV_OK: return "OFV_OK";
    case OFV_ERR_INVALID_ARG: return "OFV_ERR_INVALID_ARG";
    case OFV_ERR_SHAPE: return "OFV_ERR_SHAPE";
    case OFV_ERR_ALLOC: return "OFV_ERR_ALLOC";
    case OFV_ERR_CUDA: return "OFV_ERR_CUDA";
    case OFV_ERR_TIMEOUT: return "OFV_ERR_TIMEOUT";
    case OFV_ERR_UNSUPPORTED: return "OFV_ERR_UNSUPPORTED";
    }
    return "OFV_ERR_UNKNOWN";
}

int ofv_version(void) { return 200; }

}  // extern "C"
