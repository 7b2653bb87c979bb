// Batched entry point: many image pairs of unequal size in one persistent
// launch (a work queue of (stage, pair, tile) units), with an autotuner that
// picks the unit schedule and the number of persistent CTAs per batch
// signature.
#include <cuda_runtime.h>

#include <algorithm>
#include <new>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "../../include/ofv.h"
#include "k_block.cuh"
#include "ofv_handle.h"

namespace ofv {
#define OFV_EXTERN_QUEUE(T, VAR)                                                                   \
    extern template cudaError_t launch_queue_t<T, VAR>(const QueueParams &, int, int, cudaStream_t, int); \
    extern template int queue_occupancy_t<T, VAR>(int, int);
OFV_EXTERN_QUEUE(float, false)
OFV_EXTERN_QUEUE(float, true)
OFV_EXTERN_QUEUE(__half, false)
OFV_EXTERN_QUEUE(__half, true)
OFV_EXTERN_QUEUE(__nv_bfloat16, false)
OFV_EXTERN_QUEUE(__nv_bfloat16, true)
#undef OFV_EXTERN_QUEUE
}  // namespace ofv

using namespace ofv;

namespace {

constexpr long long kWaitTimeoutNs = 5000000000LL;  // 5 s
constexpr int kWaitSpinLimit = 200000000;

// The kernels with variant code run only when a variant is on.
// shape: the block kernel's tile shape (0 default, 1 alternative; the
// variant kernels have the default only).
cudaError_t launch_queue(int store, const QueueParams &q, int kr, int ctas, cudaStream_t s, int shape)
{
    const bool var = q.inc || q.gauss;
    switch (store) {
    case OFV_STORE_F16: return var ? launch_queue_t<__half, true>(q, kr, ctas, s, shape)
                                   : launch_queue_t<__half, false>(q, kr, ctas, s, shape);
    case OFV_STORE_BF16: return var ? launch_queue_t<__nv_bfloat16, true>(q, kr, ctas, s, shape)
                                    : launch_queue_t<__nv_bfloat16, false>(q, kr, ctas, s, shape);
    default:
        return var ? launch_queue_t<float, true>(q, kr, ctas, s, shape)
                   : launch_queue_t<float, false>(q, kr, ctas, s, shape);
    }
}

int queue_occupancy(int store, int kr, bool var, int shape)
{
    switch (store) {
    case OFV_STORE_F16:
        return var ? queue_occupancy_t<__half, true>(kr, shape) : queue_occupancy_t<__half, false>(kr, shape);
    case OFV_STORE_BF16:
        return var ? queue_occupancy_t<__nv_bfloat16, true>(kr, shape)
                   : queue_occupancy_t<__nv_bfloat16, false>(kr, shape);
    default: return var ? queue_occupancy_t<float, true>(kr, shape) : queue_occupancy_t<float, false>(kr, shape);
    }
}

struct DevGuard {
    int prev = -1;
    explicit DevGuard(int dev)
    {
        if (cudaGetDevice(&prev) == cudaSuccess && prev != dev) cudaSetDevice(dev);
    }
    ~DevGuard()
    {
        int cur = -1;
        if (prev >= 0 && cudaGetDevice(&cur) == cudaSuccess && cur != prev) cudaSetDevice(prev);
    }
};

// Unit list of one schedule, in claim order: per unit (stage, pair, tile,
// tiles of the pair's previous stage -- the count its dependency waits for).
void build_schedule(int schedule, int S, int n, const std::vector<std::vector<int>> &tiles, std::vector<int4> &desc)
{
    desc.clear();
    const int chunk = schedule > 0 ? schedule : n;
    for (int c0 = 0; c0 < n; c0 += chunk) {
        const int c1 = std::min(n, c0 + chunk);
        for (int s = 0; s < S; ++s)
            for (int p = c0; p < c1; ++p)
                for (int t = 0; t < tiles[p][s]; ++t) desc.push_back(make_int4(s, p, t, s > 0 ? tiles[p][s - 1] : 0));
    }
}

// One batch on stream cs.  record: the pass is being captured into a CUDA
// graph right after an eager pass of the same batch on the same handle, so
// every descriptor, the schedule and the tensor maps are already in the arena
// and the tuning is cached: the pass issues device work only (no host copies,
// no arena growth, no timing) and fails if anything would have to be uploaded.
ofv_status batched_impl(ofv_handle *h, int n, const ofv_pair *pairs, ofv_stream_t stream, bool record)
{
    if (!h || !pairs) return fail_msg(OFV_ERR_INVALID_ARG, "ofv_compute_batched: handle or pairs is NULL");
    if (n < 1 || n > 32767)
        return fail_msg(OFV_ERR_INVALID_ARG, "ofv_compute_batched: n=%d outside 1..32767 (one launch ingests all 2n frames)",
                        n);
    const ofv_params &p = h->p;
    if (p.path != OFV_PATH_FUSED || p.kernel_radius > 10)
        return fail_msg(OFV_ERR_UNSUPPORTED, "ofv_compute_batched: needs the fused path with KR <= 10");
    if (h->mask_on)
        return fail_msg(OFV_ERR_UNSUPPORTED, "ofv_compute_batched: a region mask is set (it has the handle's size)");
    const int L = h->L, IT = p.iterations, S = L * IT, KR = p.kernel_radius;
    const int minsz = 2 * KR + 1 > 8 ? 2 * KR + 1 : 8;
    const int sb = store_bytes(p.storage);
    const bool var = p.window == OFV_WINDOW_GAUSS || p.increment_form;
    // tile shapes the tuner may pick: the one tile_edge names, else both
    // (the variant kernels have the default shape only)
    std::vector<int> shapes;
    if (p.tile_edge != 0 || var)
        shapes.push_back(std::max(tile_shape_of(p), 0));
    else
        shapes = {0, 1};
    std::vector<std::vector<int>> Hs(n, std::vector<int>(L)), Ws(n, std::vector<int>(L));
    std::vector<std::vector<int>> tiles[2];  // [shape][pair][stage]: tiles of the stage's level
    for (int t : shapes) tiles[t].assign(n, std::vector<int>(S));
    for (int i = 0; i < n; ++i) {
        const ofv_pair &q = pairs[i];
        if (!q.I1 || !q.I2 || !q.u || !q.v || q.u == q.v)
            return fail_msg(OFV_ERR_INVALID_ARG, "ofv_compute_batched: pair %d has a NULL or aliased buffer", i);
        if (q.H < 1 || q.W < 1 || (int64_t)q.H * q.W > 2147483647LL)
            return fail_msg(OFV_ERR_SHAPE, "ofv_compute_batched: pair %d has H=%d W=%d", i, q.H, q.W);
        Hs[i][0] = q.H;
        Ws[i][0] = q.W;
        for (int l = 1; l < L; ++l) {
            Hs[i][l] = (Hs[i][l - 1] + 1) / 2;
            Ws[i][l] = (Ws[i][l - 1] + 1) / 2;
        }
        if (Hs[i][L - 1] < minsz || Ws[i][L - 1] < minsz)
            return fail_msg(OFV_ERR_SHAPE, "ofv_compute_batched: pair %d (%dx%d): coarsest level below %d", i, q.H,
                            q.W, minsz);
        for (int t : shapes) {
            const int TS = block_tile_size(KR, t);
            for (int s = 0; s < S; ++s) {
                const int l = L - 1 - s / IT;
                tiles[t][i][s] = ((Ws[i][l] + TS - 1) / TS) * ((Hs[i][l] + TS - 1) / TS);
            }
        }
    }
    DevGuard dg(h->device);
    cudaStream_t cs = (cudaStream_t)stream;
    cudaError_t e = cudaPeekAtLastError();
    if (e != cudaSuccess) {
        cudaGetLastError();
        return cuda_fail_msg(e, "error pending before ofv_compute_batched");
    }
    if (tma_expired(h))
        return fail_msg(OFV_ERR_TIMEOUT, "ofv_compute_batched: a TMA copy of an earlier launch did not complete");
    if (!h->qerr_h) {
        if (cudaHostAlloc(reinterpret_cast<void **>(&h->qerr_h), sizeof(int), cudaHostAllocMapped) != cudaSuccess ||
            cudaHostGetDevicePointer(reinterpret_cast<void **>(&h->qerr_d), h->qerr_h, 0) != cudaSuccess) {
            cudaGetLastError();
            if (h->qerr_h) cudaFreeHost(h->qerr_h);
            h->qerr_h = h->qerr_d = nullptr;
            return fail_msg(OFV_ERR_ALLOC, "ofv_compute_batched: page-locked error word");
        }
        *h->qerr_h = 0;
    }
    if (const int u = *static_cast<volatile int *>(h->qerr_h))
        return fail_msg(OFV_ERR_TIMEOUT, "ofv_compute_batched: a dependency wait of work unit %d expired", u - 1);

    // workspace: per pair two pyramids and two fields, then the queue data
    std::vector<size_t> lvl_off(2 * (size_t)n * L), vb_off(2 * (size_t)n), tmp_off(2 * (size_t)n, 0);
    std::vector<int> vpitch(n);
    size_t off = 0;
    for (int i = 0; i < n; ++i) {
        for (int f = 0; f < 2; ++f)
            for (int l = 0; l < L; ++l) {
                lvl_off[((size_t)i * 2 + f) * L + l] = off;
                off = align_up(off + (size_t)Hs[i][l] * pitch_for(Ws[i][l]) * sb, 256);
            }
        vpitch[i] = pitch_for(Ws[i][0]);
        for (int k = 0; k < 2; ++k) {
            vb_off[2 * i + k] = off;
            off = align_up(off + (size_t)Hs[i][0] * vpitch[i] * sizeof(float2), 256);
        }
        if (p.prefilter)
            for (int f = 0; f < 2; ++f) {
                tmp_off[2 * i + f] = off;
                off = align_up(off + (size_t)Hs[i][0] * pitch_for(Ws[i][0]) * sizeof(float), 256);
            }
    }
    const size_t pairs_off = off;
    off = align_up(off + sizeof(BatchPair) * n, 256);
    const size_t tmaps_off = off;  // [pair][16 levels][2 frames] tensor maps
    off = align_up(off + sizeof(CUtensorMap) * 32 * (size_t)n, 256);
    const size_t maxgroups = (size_t)S * n;
    size_t maxunits = 1;  // units of the tile shape with the most tiles
    for (int t : shapes) {
        size_t u = 0;
        for (int i = 0; i < n; ++i)
            for (int st = 0; st < S; ++st) u += (size_t)tiles[t][i][st];
        maxunits = std::max(maxunits, u);
    }
    if (maxunits > 2147483647u)
        return fail_msg(OFV_ERR_SHAPE, "ofv_compute_batched: %zu work units exceed 2^31 - 1", maxunits);
    const size_t desc_off = off;
    off = align_up(off + sizeof(int4) * maxunits, 256);
    const size_t done_off = off;
    off = align_up(off + sizeof(int) * (maxgroups + 2), 256);  // done counters, head, error
    const size_t ing_off = off;  // ingest descriptors of the 2n frames, then the reduce ones per level
    off = align_up(off + sizeof(IngestArgs) * 2 * (size_t)n, 256);
    const size_t red_off = off;
    off = align_up(off + sizeof(ReduceArgs) * 2 * (size_t)n * (L > 1 ? L - 1 : 1), 256);
    if (off > h->batch_bytes) {
        if (record) return fail_msg(OFV_ERR_INVALID_ARG, "ofv_compute_batched: recording needs a prepared arena");
        if (h->batch_arena) {
            e = cudaStreamSynchronize(cs);
            cudaFree(h->batch_arena);
            h->batch_arena = nullptr;
            h->batch_bytes = 0;
        }
        h->batch_sched_key.clear();  // nothing uploaded lives in the new arena
        h->batch_maps_key.clear();
        e = dev_alloc(&h->batch_arena, off);
        if (e != cudaSuccess) {
            cudaGetLastError();
            h->batch_arena = nullptr;
            return fail_msg(OFV_ERR_ALLOC, "ofv_compute_batched: cudaMalloc of %zu bytes failed", off);
        }
        h->batch_bytes = off;
    }
    char *base = static_cast<char *>(h->batch_arena);
    auto lvl = [&](int i, int f, int l) { return (void *)(base + lvl_off[((size_t)i * 2 + f) * L + l]); };

    // steps 1-2: ingest every frame of the batch in one launch, then reduce
    // each level of every frame in one launch (descriptors in the arena)
    {
        std::vector<IngestArgs> ia(2 * (size_t)n);
        std::vector<ReduceArgs> ra(2 * (size_t)n * (L > 1 ? L - 1 : 1));
        for (int i = 0; i < n; ++i)
            for (int f = 0; f < 2; ++f) {
                IngestArgs &a = ia[2 * i + f];
                memset(&a, 0, sizeof a);
                a.raw = f ? pairs[i].I2 : pairs[i].I1;
                a.out = lvl(i, f, 0);
                a.tmp = p.prefilter ? reinterpret_cast<float *>(base + tmp_off[2 * i + f]) : nullptr;
                a.w25 = h->w25;
                a.H = Hs[i][0];
                a.W = Ws[i][0];
                a.pitch = pitch_for(Ws[i][0]);
                a.in_type = p.input;
                a.bits = p.bit_depth;
                a.nr = p.norm_radius;
                a.eps_n = p.norm_eps;
                a.prefilter = p.prefilter;
                for (int l = 1; l < L; ++l) {
                    ReduceArgs &r = ra[(size_t)(l - 1) * 2 * n + 2 * i + f];
                    r.src = lvl(i, f, l - 1);
                    r.Hs = Hs[i][l - 1];
                    r.Ws = Ws[i][l - 1];
                    r.spitch = pitch_for(Ws[i][l - 1]);
                    r.dst = lvl(i, f, l);
                    r.Hd = Hs[i][l];
                    r.Wd = Ws[i][l];
                    r.dpitch = pitch_for(Ws[i][l]);
                }
            }
        const IngestArgs *ia_d = reinterpret_cast<const IngestArgs *>(base + ing_off);
        const ReduceArgs *ra_d = reinterpret_cast<const ReduceArgs *>(base + red_off);
        if (!record) {
            e = cudaMemcpyAsync(base + ing_off, ia.data(), sizeof(IngestArgs) * ia.size(), cudaMemcpyHostToDevice, cs);
            if (e == cudaSuccess && L > 1)
                e = cudaMemcpyAsync(base + red_off, ra.data(), sizeof(ReduceArgs) * ra.size(), cudaMemcpyHostToDevice,
                                    cs);
            if (e != cudaSuccess) return cuda_fail_msg(e, "ofv_compute_batched: uploading frame descriptors");
        }
        e = launch_ingest_list(ia.data(), ia_d, 2 * n, p.storage, cs);
        if (e != cudaSuccess) return cuda_fail_msg(e, "ofv_compute_batched: ingest launch");
        for (int l = 1; l < L; ++l) {
            const size_t o = (size_t)(l - 1) * 2 * n;
            e = launch_reduce_list(ra.data() + o, ra_d + o, 2 * n, p.storage, cs);
            if (e != cudaSuccess) return cuda_fail_msg(e, "ofv_compute_batched: reduce launch");
        }
    }

    // pair descriptors
    std::vector<BatchPair> bp(n);
    for (int i = 0; i < n; ++i) {
        BatchPair &b = bp[i];
        memset(&b, 0, sizeof b);
        for (int l = 0; l < L; ++l) {
            b.P1[l] = lvl(i, 0, l);
            b.P2[l] = lvl(i, 1, l);
            b.H[l] = Hs[i][l];
            b.W[l] = Ws[i][l];
            b.pitch[l] = pitch_for(Ws[i][l]);
        }
        b.vb[0] = reinterpret_cast<float2 *>(base + vb_off[2 * i]);
        b.vb[1] = reinterpret_cast<float2 *>(base + vb_off[2 * i + 1]);
        b.u = pairs[i].u;
        b.v = pairs[i].v;
        b.vpitch = vpitch[i];
    }
    if (!record) {
        e = cudaMemcpyAsync(base + pairs_off, bp.data(), sizeof(BatchPair) * n, cudaMemcpyHostToDevice, cs);
        if (e != cudaSuccess) return cuda_fail_msg(e, "ofv_compute_batched: uploading pair descriptors");
    }

    // layout of the arena: its address, the pair sizes in order and the
    // parameters fix every address in it
    std::string mkey = std::to_string(reinterpret_cast<uintptr_t>(base)) + "/" + std::to_string(p.storage) + "/" +
                       std::to_string(KR) + "/" + std::to_string(L) + "/" + std::to_string(IT);
    for (int i = 0; i < n; ++i) mkey += "/" + std::to_string(Hs[i][0]) + "x" + std::to_string(Ws[i][0]);

    // TMA tensor maps of every pair's level images for one tile shape (its
    // staged box): encoded once per layout and shape, uploaded when they
    // change; levels smaller than the staged box never use theirs.  Returns
    // false (cp.async staging) when no map could be encoded.
    ofv_status mst = OFV_OK;
    auto ensure_maps = [&](int shape) -> bool {
        if (!h->tma_err_d) return false;
        const std::string k = mkey + "/t" + std::to_string(shape);
        auto mit = h->batch_maps.find(k);
        if (mit == h->batch_maps.end()) {
            std::vector<CUtensorMap> maps(32 * (size_t)n);
            memset(maps.data(), 0, sizeof(CUtensorMap) * maps.size());
            bool ok = true;
            for (int i = 0; i < n && ok; ++i)
                for (int l = 0; l < L && ok; ++l)
                    for (int f = 0; f < 2 && ok; ++f)
                        ok = encode_block_map(&maps[((size_t)i * 16 + l) * 2 + f], lvl(i, f, l), Ws[i][l], Hs[i][l],
                                              pitch_for(Ws[i][l]), p.storage, KR, shape);
            if (!ok) return false;
            if (h->batch_maps.size() > 64) h->batch_maps.clear();
            mit = h->batch_maps.emplace(k, std::move(maps)).first;
        }
        if (h->batch_maps_key != k) {
            if (record) {
                mst = fail_msg(OFV_ERR_INVALID_ARG, "ofv_compute_batched: recording needs uploaded tensor maps");
                return false;
            }
            e = cudaMemcpyAsync(base + tmaps_off, mit->second.data(), sizeof(CUtensorMap) * mit->second.size(),
                                cudaMemcpyHostToDevice, cs);
            if (e != cudaSuccess) {
                mst = cuda_fail_msg(e, "ofv_compute_batched: uploading tensor maps");
                return false;
            }
            h->batch_maps_key = k;
        }
        return true;
    };

    int dev = h->device, sms = 0;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);

    // batch signature for the autotuner
    std::vector<std::pair<int, int>> sizes;
    for (int i = 0; i < n; ++i) sizes.push_back({Hs[i][0], Ws[i][0]});
    std::sort(sizes.begin(), sizes.end());
    std::string key = "kr" + std::to_string(KR) + "l" + std::to_string(L) + "it" + std::to_string(IT) + "s" +
                      std::to_string(p.storage) + "v" + std::to_string(p.window) + std::to_string(p.increment_form) + "t" +
                      std::to_string(p.tile_edge);
    for (auto &sz : sizes) key += ":" + std::to_string(sz.first) + "x" + std::to_string(sz.second);

    std::vector<BatchTune> cands;
    auto it = h->tune.find(key);
    const bool tuning = it == h->tune.end();
    if (tuning && record) return fail_msg(OFV_ERR_INVALID_ARG, "ofv_compute_batched: recording needs a tuned batch");
    if (tuning) {
        for (int t : shapes) {
            const int occ = std::max(1, queue_occupancy(p.storage, KR, var, t));
            for (int sch : {0, 8})
                for (int c : {occ, occ - 1})
                    if (c >= 1 && (sch == 0 || sch < n)) cands.push_back(BatchTune{sch, c, t, 0.0});
        }
    } else {
        cands.push_back(it->second);
    }

    QueueParams q;
    memset(&q, 0, sizeof q);
    q.pairs = reinterpret_cast<const BatchPair *>(base + pairs_off);
    q.unit_desc = reinterpret_cast<const int4 *>(base + desc_off);
    q.npairs = n;
    q.L = L;
    q.IT = IT;
    q.kr = KR;
    q.eps_rel = p.det_rel_eps;
    q.eps_abs = p.det_abs_eps;
    {
        IterArgs v = {};
        set_iter_variant(v, KR, p.window == OFV_WINDOW_GAUSS, p.window_sigma, p.increment_form);
        q.inc = v.inc;
        q.gauss = v.gauss;
        for (int d = 0; d <= kBlockMaxKR; ++d) q.wg[d] = v.wg[d];
    }
    q.done = reinterpret_cast<int *>(base + done_off);
    q.head = q.done + maxgroups;
    q.error = q.head + 1;
    q.timeout_ns = kWaitTimeoutNs;
    q.spin_limit = kWaitSpinLimit;
    q.tma_err = h->tma_err_d;
    q.host_err = h->qerr_d;

    struct Events {  // timing events of the tuning pass, destroyed on every return
        cudaEvent_t a = nullptr, b = nullptr;
        ~Events()
        {
            if (a) cudaEventDestroy(a);
            if (b) cudaEventDestroy(b);
        }
    } ev;
    if (tuning) {
        cudaEventCreate(&ev.a);
        cudaEventCreate(&ev.b);
    }
    std::vector<int4> desc;
    // one persistent launch of candidate c (timed while tuning)
    auto run = [&](size_t c, bool timed) -> ofv_status {
        const int shape = cands[c].shape;
        const bool use_tma = ensure_maps(shape);
        if (mst != OFV_OK) return mst;
        q.tmaps = use_tma ? reinterpret_cast<const CUtensorMap *>(base + tmaps_off) : nullptr;
        build_schedule(cands[c].schedule, S, n, tiles[shape], desc);
        q.total_units = (int)desc.size();
        const std::string skey = mkey + "#" + std::to_string(cands[c].schedule) + "t" + std::to_string(shape);
        e = cudaSuccess;
        if (h->batch_sched_key != skey) {  // the schedule of this layout is not in the arena yet
            if (record) return fail_msg(OFV_ERR_INVALID_ARG, "ofv_compute_batched: recording needs the uploaded schedule");
            e = cudaMemcpyAsync(base + desc_off, desc.data(), sizeof(int4) * desc.size(), cudaMemcpyHostToDevice, cs);
            h->batch_sched_key = e == cudaSuccess ? skey : std::string();
        }
        if (e == cudaSuccess) e = cudaMemsetAsync(q.done, 0, sizeof(int) * (maxgroups + 2), cs);
        if (e != cudaSuccess) return cuda_fail_msg(e, "ofv_compute_batched: uploading the schedule");
        const int ctas = std::min(sms * cands[c].ctas_per_sm, std::max(1, q.total_units));
        if (timed) cudaEventRecord(ev.a, cs);
        e = launch_queue(p.storage, q, KR, ctas, cs, shape);
        if (e != cudaSuccess) return cuda_fail_msg(e, "ofv_compute_batched: persistent launch");
        if (timed) {
            cudaEventRecord(ev.b, cs);
            e = cudaEventSynchronize(ev.b);
            if (e != cudaSuccess) return cuda_fail_msg(e, "ofv_compute_batched: timing a candidate");
            float ms = 0.f;
            cudaEventElapsedTime(&ms, ev.a, ev.b);
            cands[c].ms = ms;
            if (const int u = *static_cast<volatile int *>(h->qerr_h))
                return fail_msg(OFV_ERR_TIMEOUT, "ofv_compute_batched: a dependency wait of work unit %d expired",
                                u - 1);
        }
        return OFV_OK;
    };
    int best = 0;
    for (size_t c = 0; c < cands.size(); ++c) {
        const ofv_status st = run(c, tuning);
        if (st != OFV_OK) return st;
        if (tuning && cands[c].ms < cands[best].ms) best = (int)c;
    }
    if (tuning) {
        h->tune[key] = cands[best];
        // Candidates of one tile shape compute the same fields; another shape
        // sums the windows in another order.  The fields left in place must be
        // the chosen configuration's, as in every later call of this signature.
        if (cands[best].shape != cands.back().shape) {
            const ofv_status st = run((size_t)best, false);
            if (st != OFV_OK) return st;
        }
    }
    if (!record) {
        h->last_tune = tuning ? cands[best] : cands[0];
        h->last_tuned = tuning ? 1 : 0;
    }
    return OFV_OK;
}

}  // namespace

extern "C" {

ofv_status ofv_compute_batched(ofv_handle *h, int n, const ofv_pair *pairs, ofv_stream_t stream)
{
    return batched_impl(h, n, pairs, stream, false);
}

ofv_status ofv_graph_create_batched(ofv_handle *h, int n, const ofv_pair *pairs, ofv_graph **out)
{
    if (!out) return fail_msg(OFV_ERR_INVALID_ARG, "ofv_graph_create_batched: out is NULL");
    *out = nullptr;
    if (!h || !pairs) return fail_msg(OFV_ERR_INVALID_ARG, "ofv_graph_create_batched: handle or pairs is NULL");
    DevGuard dg(h->device);
    // the eager passes use the handle's arena on a stream of their own:
    // earlier work on the handle must be finished
    cudaError_t e = cudaDeviceSynchronize();
    if (e != cudaSuccess) return cuda_fail_msg(e, "ofv_graph_create_batched: waiting for earlier work");
    cudaStream_t cs = nullptr;
    e = cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking);
    if (e != cudaSuccess) return cuda_fail_msg(e, "ofv_graph_create_batched: creating the capture stream");
    // eager pass: sizes the arena, uploads every descriptor, tunes a new
    // signature; after tuning a second pass uploads the chosen schedule
    ofv_status st = batched_impl(h, n, pairs, (ofv_stream_t)cs, false);
    if (st == OFV_OK && h->last_tuned) st = batched_impl(h, n, pairs, (ofv_stream_t)cs, false);
    if (st == OFV_OK) {
        e = cudaStreamSynchronize(cs);
        if (e != cudaSuccess) st = cuda_fail_msg(e, "ofv_graph_create_batched: eager pass");
    }
    cudaGraph_t graph = nullptr;
    if (st == OFV_OK) {
        e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
        if (e != cudaSuccess) {
            st = cuda_fail_msg(e, "ofv_graph_create_batched: beginning stream capture");
        } else {
            st = batched_impl(h, n, pairs, (ofv_stream_t)cs, true);
            e = cudaStreamEndCapture(cs, &graph);
            if (st == OFV_OK && e != cudaSuccess) st = cuda_fail_msg(e, "ofv_graph_create_batched: ending stream capture");
        }
    }
    cudaGraphExec_t exec = nullptr;
    if (st == OFV_OK) {
        e = cudaGraphInstantiate(&exec, graph, 0);
        if (e != cudaSuccess) st = cuda_fail_msg(e, "ofv_graph_create_batched: instantiating the graph");
    }
    cudaStreamDestroy(cs);
    ofv_graph *gr = nullptr;
    if (st == OFV_OK) {
        gr = new (std::nothrow) ofv_graph{h, graph, exec, h->batch_arena};
        if (!gr) st = fail_msg(OFV_ERR_ALLOC, "ofv_graph_create_batched: host allocation of the graph handle failed");
    }
    if (st != OFV_OK) {
        if (exec) cudaGraphExecDestroy(exec);
        if (graph) cudaGraphDestroy(graph);
        return st;
    }
    // the graph takes the arena: later batches of the handle get a new one
    h->batch_arena = nullptr;
    h->batch_bytes = 0;
    h->batch_sched_key.clear();
    h->batch_maps_key.clear();
    *out = gr;
    return OFV_OK;
}

ofv_status ofv_batch_tuning(const ofv_handle *h, int *schedule, int *ctas_per_sm, int *tile_edge, double *ms,
                            int *tuned)
{
    if (!h || !schedule || !ctas_per_sm || !tile_edge || !ms || !tuned)
        return fail_msg(OFV_ERR_INVALID_ARG, "NULL argument");
    *schedule = h->last_tune.schedule;
    *ctas_per_sm = h->last_tune.ctas_per_sm;
    *tile_edge = block_tile_size(h->p.kernel_radius, h->last_tune.shape);
    *ms = h->last_tune.ms;
    *tuned = h->last_tuned;
    return OFV_OK;
}

// A persistent launch whose one work unit waits on a counter that nothing
// increments; the wait must expire after about timeout_us and leave the
// error word set (1 + the unit) for the host, without a fault or a hang.
ofv_status ofv_queue_selftest(int timeout_us, int *error_word)
{
    if (!error_word || timeout_us < 1 || timeout_us > 10000000)
        return fail_msg(OFV_ERR_INVALID_ARG, "ofv_queue_selftest: bad arguments");
    *error_word = 0;
    void *mem = nullptr;
    const size_t bytes = 4096;
    cudaError_t e = cudaMalloc(&mem, bytes);
    if (e != cudaSuccess) return cuda_fail_msg(e, "ofv_queue_selftest: cudaMalloc");
    char *b = static_cast<char *>(mem);
    BatchPair bp;
    memset(&bp, 0, sizeof bp);
    bp.H[0] = bp.W[0] = bp.H[1] = bp.W[1] = 8;
    // stage 1 of pair 0: waits for the one tile of stage 0, which no unit runs
    const int4 unit = make_int4(1, 0, 0, 1);
    e = cudaMemcpy(b, &bp, sizeof bp, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(b + 2048, &unit, sizeof unit, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemset(b + 3072, 0, 64);
    QueueParams q;
    memset(&q, 0, sizeof q);
    q.pairs = reinterpret_cast<const BatchPair *>(b);
    q.unit_desc = reinterpret_cast<const int4 *>(b + 2048);
    q.total_units = 1;
    q.npairs = 1;
    q.L = 2;
    q.IT = 1;
    q.kr = 4;
    q.done = reinterpret_cast<int *>(b + 3072);
    q.head = q.done + 4;
    q.error = q.done + 5;
    q.timeout_ns = (long long)timeout_us * 1000;
    q.spin_limit = kWaitSpinLimit;
    // the mapped host word through which asynchronous batches report
    int *hw = nullptr, *hw_d = nullptr;
    if (e == cudaSuccess) e = cudaHostAlloc(reinterpret_cast<void **>(&hw), sizeof(int), cudaHostAllocMapped);
    if (e == cudaSuccess) e = cudaHostGetDevicePointer(reinterpret_cast<void **>(&hw_d), hw, 0);
    if (e == cudaSuccess) {
        *hw = 0;
        q.host_err = hw_d;
        e = launch_queue(OFV_STORE_F32, q, 4, 1, nullptr, 0);
    }
    int err = 0;
    if (e == cudaSuccess) e = cudaMemcpy(&err, q.error, sizeof(int), cudaMemcpyDeviceToHost);
    const int host_word = hw ? *static_cast<volatile int *>(hw) : 0;
    if (hw) cudaFreeHost(hw);
    cudaFree(mem);
    if (e != cudaSuccess) return cuda_fail_msg(e, "ofv_queue_selftest");
    *error_word = err;
    if (host_word != err)
        return fail_msg(OFV_ERR_CUDA, "ofv_queue_selftest: host word %d, device word %d", host_word, err);
    return err ? fail_msg(OFV_ERR_TIMEOUT, "ofv_queue_selftest: wait expired as intended (unit %d)", err - 1)
               : OFV_OK;
}

}  // extern "C"
