// One displacement field computed as horizontal strips, each with its own
// workspace: the decomposition that spreads a single large field over
// several GPUs (the paper names 2 or 3 GPUs as the way to raise the rate
// further, Conclusions), here run strip after strip on one device.
//
// At every level the strips own whole tile rows of the block kernel's tile
// grid (so each output pixel is computed by the same tile, with the same
// window-sum order, as in the single-field computation).  A strip builds the
// rows of its pyramid it reads -- its own rows plus a redundant image halo
// wide enough for the staged tiles, the window and warps up to max_disp --
// from an input view of the rows below and above it, so images need no
// exchange.  After every Gauss-Newton iteration each strip copies, from the
// strips that own them, the rows of the new field its next iteration reads
// (its window halo, or the coarse rows the up-sampling of the next finer
// level reads).  A field computed this way equals the single-field result
// bitwise as long as no warp reaches farther than max_disp.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstring>

#include "../../include/ofv.h"
#include "k_block.cuh"
#include "ofv_handle.h"

using namespace ofv;

namespace {

struct Range {
    int a, b;  // rows a .. b-1
    bool empty() const { return b <= a; }
};
Range clip(Range r, int n) { return Range{std::max(r.a, 0), std::min(r.b, n)}; }
Range hull(Range x, Range y)
{
    if (x.empty()) return y;
    if (y.empty()) return x;
    return Range{std::min(x.a, y.a), std::max(x.b, y.b)};
}
Range meet(Range x, Range y) { return Range{std::max(x.a, y.a), std::min(x.b, y.b)}; }

struct StripPlan {
    int L;
    int Hs[kMaxLevels], Ws[kMaxLevels];
    Range own[kMaxLevels];   // rows the strip's tiles output
    Range fld[kMaxLevels];   // rows of the level's field its iterations read
    Range up[kMaxLevels];    // rows of level l+1's field its first iteration at level l reads
    Range img[kMaxLevels];   // rows of the level image it computes (all correct)
    Range ingest;            // input rows it ingests into level 0
};

// Owned tile rows: the level's tile rows shared out evenly over the strips.
Range owned(int Hl, int ts, int nstrips, int strip)
{
    const int T = (Hl + ts - 1) / ts;
    const int t0 = (int)((long long)strip * T / nstrips), t1 = (int)((long long)(strip + 1) * T / nstrips);
    return Range{std::min(t0 * ts, Hl), std::min(t1 * ts, Hl)};
}

ofv_status plan_strip(int H, int W, const ofv_params &p, int nstrips, int max_disp, int strip, StripPlan *o)
{
    const int L = p.levels_psl + 1, KR = p.kernel_radius;
    o->L = L;
    o->Hs[0] = H;
    o->Ws[0] = W;
    for (int l = 1; l < L; ++l) {
        o->Hs[l] = (o->Hs[l - 1] + 1) / 2;
        o->Ws[l] = (o->Ws[l - 1] + 1) / 2;
    }
    const int ts = block_tile_size(KR, std::max(tile_shape_of(p), 0));
    Range need[kMaxLevels];
    for (int l = 0; l < L; ++l) {
        const int Hl = o->Hs[l];
        o->own[l] = owned(Hl, ts, nstrips, strip);
        if (o->own[l].empty()) {
            o->fld[l] = o->up[l] = need[l] = Range{0, 0};
            continue;
        }
        // products of the tiles' window halo read V0 there
        o->fld[l] = clip(Range{o->own[l].a - KR, o->own[l].b + KR}, Hl);
        // images: the staged box of a tile reaches KR + REACH + 4 rows past
        // the tile, and the three staging bands up to 2 more; warps beyond the
        // staged margin read up to |V|/2 + 2 rows away (V of the level)
        const int warp = (max_disp + (1 << (l + 1)) - 1) / (1 << (l + 1)) + 2;
        const int margin = KR + kBlockReach + 8 + warp;
        need[l] = clip(Range{o->own[l].a - margin, o->own[l].b + margin}, Hl);
    }
    for (int l = 0; l + 1 < L; ++l) {
        if (o->fld[l].empty()) {
            o->up[l] = Range{0, 0};
            continue;
        }
        // up-sampling at level l reads coarse rows y/2 and y/2 + 1 (clamped)
        o->up[l] = clip(Range{o->fld[l].a >> 1, ((o->fld[l].b - 1) >> 1) + 2}, o->Hs[l + 1]);
    }
    o->up[L - 1] = Range{0, 0};
    // image rows, coarse to fine: a level-l row i reads level l-1 rows 2i-2 .. 2i+2
    o->img[L - 1] = need[L - 1];
    for (int l = L - 2; l >= 0; --l) {
        Range src{0, 0};
        if (!o->img[l + 1].empty())
            src = clip(Range{2 * o->img[l + 1].a - 2, 2 * o->img[l + 1].b + 1}, o->Hs[l]);
        Range r = hull(need[l], src);
        r.a &= ~1;  // a reduce view starts on an even row
        o->img[l] = r;
    }
    // local normalization (NR) and the pre-filter (2) read neighbours too
    const int reach0 = p.norm_radius + (p.prefilter ? 2 : 0);
    o->ingest = clip(Range{o->img[0].a - reach0, o->img[0].b + reach0}, H);
    (void)W;
    return OFV_OK;
}

ofv_status check_strip_args(int H, int W, const ofv_params *p, int nstrips, int max_disp)
{
    if (!p) return fail_msg(OFV_ERR_INVALID_ARG, "strips: params is NULL");
    if (H < 1 || W < 1) return fail_msg(OFV_ERR_SHAPE, "strips: H=%d W=%d must be positive", H, W);
    if (nstrips < 1 || nstrips > 64) return fail_msg(OFV_ERR_INVALID_ARG, "strips: nstrips=%d outside 1..64", nstrips);
    if (max_disp < 0 || max_disp > 4096)
        return fail_msg(OFV_ERR_INVALID_ARG, "strips: max_disp=%d outside 0..4096", max_disp);
    if (p->levels_psl < 0 || p->levels_psl >= kMaxLevels)
        return fail_msg(OFV_ERR_INVALID_ARG, "strips: levels_psl=%d outside 0..%d", p->levels_psl, kMaxLevels - 1);
    if (p->path != OFV_PATH_FUSED || !block_supports(p->kernel_radius))
        return fail_msg(OFV_ERR_UNSUPPORTED, "strips: the fused path with KR 1..10 only");
    if (tile_shape_of(*p) < 0) return fail_msg(OFV_ERR_INVALID_ARG, "strips: tile_edge=%d", p->tile_edge);
    return OFV_OK;
}

}  // namespace

extern "C" ofv_status ofv_strip_plan(int H, int W, const ofv_params *params, int nstrips, int max_disp, int level,
                                     int strip, ofv_strip_rows *out)
{
    ofv_status st = check_strip_args(H, W, params, nstrips, max_disp);
    if (st != OFV_OK) return st;
    if (!out) return fail_msg(OFV_ERR_INVALID_ARG, "ofv_strip_plan: out is NULL");
    if (strip < 0 || strip >= nstrips) return fail_msg(OFV_ERR_INVALID_ARG, "ofv_strip_plan: strip %d", strip);
    if (level < 0 || level > params->levels_psl) return fail_msg(OFV_ERR_INVALID_ARG, "ofv_strip_plan: level %d", level);
    StripPlan pl;
    plan_strip(H, W, *params, nstrips, max_disp, strip, &pl);
    out->own_row0 = pl.own[level].a;
    out->own_row1 = pl.own[level].b;
    out->img_row0 = pl.img[level].a;
    out->img_row1 = pl.img[level].b;
    out->fld_row0 = pl.fld[level].a;
    out->fld_row1 = pl.fld[level].b;
    out->up_row0 = pl.up[level].a;
    out->up_row1 = pl.up[level].b;
    out->ingest_row0 = level == 0 ? pl.ingest.a : 0;
    out->ingest_row1 = level == 0 ? pl.ingest.b : 0;
    return OFV_OK;
}

namespace {

// Workspace of one strip: its pyramids of both frames and two ping-pong fields
// (full-size buffers, of which it computes only its rows).
struct StripBufs {
    void *lvl[2][kMaxLevels];
    float2 *fld[2];
};

ofv_status strip_workspace(ofv_handle *h, int nstrips, StripBufs *sb, float **tmp)
{
    const int L = h->L, sbytes = store_bytes(h->p.storage);
    size_t off = 0;
    auto take = [&](size_t bytes) {
        const size_t o = off;
        off = align_up(off + bytes, 256);
        return o;
    };
    size_t lo[64][2][kMaxLevels], fo[64][2], to[2] = {0, 0};
    for (int d = 0; d < nstrips; ++d) {
        for (int f = 0; f < 2; ++f)
            for (int l = 0; l < L; ++l) lo[d][f][l] = take((size_t)h->Hs[l] * h->pitch[l] * sbytes);
        for (int k = 0; k < 2; ++k) fo[d][k] = take((size_t)h->H * h->vpitch * sizeof(float2));
    }
    if (h->p.prefilter)
        for (int f = 0; f < 2; ++f) to[f] = take((size_t)h->H * h->pitch[0] * sizeof(float));
    if (off > h->strip_bytes) {
        if (h->strip_arena) {
            cudaFree(h->strip_arena);
            h->strip_arena = nullptr;
            h->strip_bytes = 0;
        }
        if (dev_alloc(&h->strip_arena, off) != cudaSuccess) {
            cudaGetLastError();
            h->strip_arena = nullptr;
            return fail_msg(OFV_ERR_ALLOC, "ofv_compute_strips: cudaMalloc of %zu bytes failed", off);
        }
        h->strip_bytes = off;
    }
    char *base = static_cast<char *>(h->strip_arena);
    for (int d = 0; d < nstrips; ++d) {
        for (int f = 0; f < 2; ++f)
            for (int l = 0; l < L; ++l) sb[d].lvl[f][l] = base + lo[d][f][l];
        for (int k = 0; k < 2; ++k) sb[d].fld[k] = reinterpret_cast<float2 *>(base + fo[d][k]);
    }
    tmp[0] = h->p.prefilter ? reinterpret_cast<float *>(base + to[0]) : nullptr;
    tmp[1] = h->p.prefilter ? reinterpret_cast<float *>(base + to[1]) : nullptr;
    return OFV_OK;
}

}  // namespace

extern "C" ofv_status ofv_compute_strips(ofv_handle *h, int nstrips, int max_disp, const void *I1, const void *I2,
                                         float *u, float *v, ofv_stream_t stream)
{
    if (!h) return fail_msg(OFV_ERR_INVALID_ARG, "ofv_compute_strips: handle is NULL");
    if (!I1 || !I2 || !u || !v || u == v)
        return fail_msg(OFV_ERR_INVALID_ARG, "ofv_compute_strips: NULL pointer or u == v");
    const ofv_params &p = h->p;
    ofv_status st = check_strip_args(h->H, h->W, &p, nstrips, max_disp);
    if (st != OFV_OK) return st;
    if (h->mask_on) return fail_msg(OFV_ERR_UNSUPPORTED, "ofv_compute_strips: a region mask is set");
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess || (dev != h->device && cudaSetDevice(h->device) != cudaSuccess))
        return fail_msg(OFV_ERR_CUDA, "ofv_compute_strips: cannot select the handle's device");
    struct Restore {
        int d, cur;
        ~Restore()
        {
            if (d >= 0 && d != cur) cudaSetDevice(d);
        }
    } restore{dev, h->device};
    cudaStream_t s = (cudaStream_t)stream;
    StripBufs sb[64];
    float *tmp[2];
    st = strip_workspace(h, nstrips, sb, tmp);
    if (st != OFV_OK) return st;
    StripPlan pl[64];
    for (int d = 0; d < nstrips; ++d) plan_strip(h->H, h->W, p, nstrips, max_disp, d, &pl[d]);
    const int L = h->L, IT = p.iterations, ib = input_bytes(p.input);
    cudaError_t e = cudaSuccess;
    auto launch_fail = [&](const char *what) { return cuda_fail_msg(e, what); };

    // steps 1-2 per strip: ingest its input rows, reduce its image rows
    for (int d = 0; d < nstrips; ++d) {
        const Range in = pl[d].ingest;
        if (in.empty()) continue;
        IngestArgs ia[2];
        const void *fr[2] = {I1, I2};
        for (int f = 0; f < 2; ++f) {
            IngestArgs &a = ia[f];
            memset(&a, 0, sizeof a);
            a.raw = static_cast<const char *>(fr[f]) + (size_t)in.a * h->W * ib;
            a.out = static_cast<char *>(sb[d].lvl[f][0]) + (size_t)in.a * h->pitch[0] * store_bytes(p.storage);
            a.tmp = tmp[f];
            a.w25 = h->w25;
            a.H = in.b - in.a;
            a.W = h->W;
            a.pitch = h->pitch[0];
            a.in_type = p.input;
            a.bits = p.bit_depth;
            a.nr = p.norm_radius;
            a.eps_n = p.norm_eps;
            a.prefilter = p.prefilter;
        }
        if ((e = launch_ingest_frames(ia, 2, p.storage, s)) != cudaSuccess) return launch_fail("strips: ingest");
        for (int l = 1; l < L; ++l) {
            const Range out = pl[d].img[l];
            if (out.empty()) continue;
            const Range src = clip(Range{2 * out.a - 2, 2 * out.b + 1}, h->Hs[l - 1]);  // src.a even
            ReduceArgs ra[2];
            const int dst0 = src.a / 2;
            for (int f = 0; f < 2; ++f) {
                ReduceArgs &r = ra[f];
                r.src = static_cast<char *>(sb[d].lvl[f][l - 1]) + (size_t)src.a * h->pitch[l - 1] * store_bytes(p.storage);
                r.Hs = src.b - src.a;
                r.Ws = h->Ws[l - 1];
                r.spitch = h->pitch[l - 1];
                r.dst = static_cast<char *>(sb[d].lvl[f][l]) + (size_t)dst0 * h->pitch[l] * store_bytes(p.storage);
                r.Hd = std::min(h->Hs[l] - dst0, (r.Hs + 1) / 2);
                r.Wd = h->Ws[l];
                r.dpitch = h->pitch[l];
            }
            if ((e = launch_reduce_frames(ra, 2, p.storage, s)) != cudaSuccess) return launch_fail("strips: reduce");
        }
    }

    // steps 3-6: coarse to fine, every strip's tiles, then the halo copies
    const int shape = tile_shape_of(p);
    const int ts = block_tile_size(p.kernel_radius, shape);
    int cur = 0;
    for (int l = L - 1; l >= 0; --l) {
        for (int t = 0; t < IT; ++t) {
            const int mode = (l == L - 1 && t == 0) ? V0_ZERO : (t == 0 ? V0_UP : V0_SAME);
            const bool last = l == 0 && t == IT - 1;
            const int nxt = (l == L - 1 && t == 0) ? 0 : 1 - cur;
            for (int d = 0; d < nstrips; ++d) {
                const Range own = pl[d].own[l];
                if (own.empty()) continue;
                IterArgs a;
                memset(&a, 0, sizeof a);
                a.P1 = sb[d].lvl[0][l];
                a.P2 = sb[d].lvl[1][l];
                a.H = h->Hs[l];
                a.W = h->Ws[l];
                a.pitch = h->pitch[l];
                a.vpitch = h->vpitch;
                a.vcpitch = h->vpitch;
                a.kr = p.kernel_radius;
                a.eps_rel = p.det_rel_eps;
                a.eps_abs = p.det_abs_eps;
                set_iter_variant(a, p.kernel_radius, p.window == OFV_WINDOW_GAUSS, p.window_sigma, p.increment_form);
                if (mode == V0_UP) {
                    a.Vc = sb[d].fld[cur];
                    a.Hc = h->Hs[l + 1];
                    a.Wc = h->Ws[l + 1];
                } else if (mode == V0_SAME) {
                    a.V0 = sb[d].fld[cur];
                }
                if (last) {
                    a.u_out = u;
                    a.v_out = v;
                } else {
                    a.Vout = sb[d].fld[nxt];
                }
                if ((e = launch_iter_block(&a, 1, p.storage, mode, s, nullptr, nullptr, own.a / ts,
                                           (own.b - own.a + ts - 1) / ts, shape)) != cudaSuccess)
                    return launch_fail("strips: iteration");
            }
            if (last) break;
            // the rows of the new field each strip reads next, from their owners
            for (int d = 0; d < nstrips; ++d) {
                const Range want = t + 1 < IT ? pl[d].fld[l] : pl[d].up[l - 1];
                if (want.empty()) continue;
                for (int o = 0; o < nstrips; ++o) {
                    if (o == d) continue;
                    const Range r = meet(want, pl[o].own[l]);
                    if (r.empty()) continue;
                    const size_t rowb = (size_t)h->vpitch * sizeof(float2);
                    e = cudaMemcpy2DAsync(sb[d].fld[nxt] + (size_t)r.a * h->vpitch, rowb,
                                          sb[o].fld[nxt] + (size_t)r.a * h->vpitch, rowb,
                                          (size_t)h->Ws[l] * sizeof(float2), (size_t)(r.b - r.a),
                                          cudaMemcpyDeviceToDevice, s);
                    if (e != cudaSuccess) return launch_fail("strips: halo copy");
                }
            }
            cur = nxt;
        }
    }
    if ((e = cudaGetLastError()) != cudaSuccess) return launch_fail("strips");
    return OFV_OK;
}
