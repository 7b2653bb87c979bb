// The handle behind the C ABI (private to the library).
#pragma once
#include <cuda_runtime.h>

#include <map>
#include <string>
#include <vector>

#include "../../include/ofv.h"
#include "k_block.cuh"

namespace ofv {

constexpr int kMaxLevels = 16;
constexpr int kMaxBatch = kMaxPairsPerLaunch;
constexpr int kGroupStreams = 3;                  // groups of a sequence in flight
constexpr int kGroupEvents = 8;                    // event ring (power of 2, > kGroupStreams + 1)
constexpr int kMaxSlots = kGroupStreams * kMaxBatch + 1;  // pyramid slots
constexpr int kHostRing = kGroupStreams + 1;  // device ring slots of the host-memory sequence pipeline

struct ProfRec {
    int cls;
    cudaEvent_t e0, e1;
    double bytes;
};

// Configuration the batched entry point's autotuner picked for one batch
// signature (sizes and parameters).
struct BatchTune {
    int schedule;     // 0: stage-major over all pairs, else pairs in groups of this many
    int ctas_per_sm;  // persistent CTAs per SM
    int shape;        // block kernel tile shape (0 default, 1 alternative)
    double ms;        // measured duration of the persistent launch
};

// Record a failure for ofv_last_error() (thread-local) and return st.
ofv_status fail_msg(ofv_status st, const char *fmt, ...);
ofv_status cuda_fail_msg(cudaError_t e, const char *where);

inline size_t align_up(size_t v, size_t a) { return (v + a - 1) / a * a; }
inline int store_bytes(int st) { return st == OFV_STORE_F32 ? 4 : 2; }
inline int input_bytes(int in) { return in == OFV_IN_U8 ? 1 : (in == OFV_IN_U16 ? 2 : 4); }

}  // namespace ofv

struct ofv_handle {
    int H, W;
    ofv_params p;
    int L;
    int B;         // pairs per launch in sequences
    int nslots;    // pyramid slots (nstreams B + 1)
    int nstreams;  // consecutive groups of a sequence run on this many streams
    int Hs[ofv::kMaxLevels], Ws[ofv::kMaxLevels], pitch[ofv::kMaxLevels];
    int vpitch;
    int device;
    void *arena;
    size_t arena_bytes;
    void *lvl[ofv::kMaxSlots][ofv::kMaxLevels];
    float2 *vbuf[2 * ofv::kGroupStreams * ofv::kMaxBatch];  // per group stream, two ping-pong fields per pair
    float *w25;
    float *tmp[ofv::kGroupStreams * ofv::kMaxFramesPerLaunch];  // pre-filter input, per group stream and frame
    // group streams of the sequence entry points, and a ring of events:
    // gev[g % kGroupEvents][0] = pyramids of group g built, [1] = group g done
    cudaStream_t gs[ofv::kGroupStreams];
    cudaEvent_t gev[ofv::kGroupEvents][2];
    cudaEvent_t gstart;
    ofv::PlainBufs plain;
    // host-pointer entry point staging (allocated on first use)
    void *stage;
    size_t stage_bytes;
    // slots of I1 and I2 of the last computed pair
    int last_s1, last_s2;
    // kernel timing
    bool prof;
    std::vector<ofv::ProfRec> recs;
    std::vector<cudaEvent_t> pool;
    size_t pool_next;
    // batched entry point: grow-only workspace and autotuner cache
    void *batch_arena;
    size_t batch_bytes;
    std::map<std::string, ofv::BatchTune> tune;
    ofv::BatchTune last_tune;
    int last_tuned;  // 1 if the last batched call ran the autotuner
    std::map<std::string, std::vector<CUtensorMap>> batch_maps;  // tensor maps per batch layout
    // reverse mode: grow-only workspace (stage fields, sums, gradients)
    void *bw_arena;
    size_t bw_bytes;
    // strip-decomposed field (ofv_compute_strips): grow-only workspace of
    // every strip's pyramids and fields
    void *strip_arena;
    size_t strip_bytes;
    // TMA tensor maps of every (slot, level) image for the block kernel's
    // staged box, and the word a kernel sets when a TMA wait expires
    // (page-locked host memory mapped into the device)
    CUtensorMap tmap[ofv::kMaxSlots][ofv::kMaxLevels];
    int tma_ok[ofv::kMaxLevels];
    int *tma_err_h, *tma_err_d;
    // host-memory sequence pipeline: copy streams, ring events, device ring
    cudaStream_t hs_stream[2];            // [0] host-to-device, [1] device-to-host
    cudaEvent_t hs_ev[ofv::kHostRing][3];  // per ring slot: frames in, fields ready, fields out
    int hs_ready;
    void *hs_stage;
    size_t hs_bytes;
    // region mask per level (dense rows of Ws[l] bytes, 0 / 1), allocated on
    // first use; applied while mask_on
    uint8_t *mask_lvl[ofv::kMaxLevels];
    void *mask_arena;
    int mask_on;
    // batched entry point: word a persistent launch sets when a dependency
    // wait expires (page-locked, mapped), and the layouts whose schedule and
    // tensor maps are in the batch arena
    int *qerr_h, *qerr_d;
    std::string batch_sched_key, batch_maps_key;
};

// A recorded CUDA graph (ofv_graph_create, ofv_graph_create_batched).  A
// batched graph owns the arena its launches read (pyramids, fields and the
// batch descriptors); a single-pair graph uses the handle's workspace.
struct ofv_graph {
    ofv_handle *h;
    cudaGraph_t graph;
    cudaGraphExec_t exec;
    void *arena;
};

namespace ofv {
// Device allocation of the library's workspaces: cudaMalloc, unless a
// failure was scheduled by ofv_debug_fail_alloc (then
// cudaErrorMemoryAllocation and nothing allocated).
cudaError_t dev_alloc(void **p, size_t bytes);
// Steps 1-2 into the handle's pyramid slots (defined with the C ABI).
ofv_status handle_pyramids(ofv_handle *h, const void *const *frames, const int *slots, int nf, cudaStream_t s);
// Tensor map of a level image with the block kernel's TMA box.
bool encode_block_map(CUtensorMap *m, const void *base, int W, int H, int pitch, int store, int kr, int shape = 0);
// Tile shape of the block kernel that params select: 0 (default) or 1 (the
// alternative edge), -1 when tile_edge is not one of the radius's edges on
// the fused block path.  The Gaussian window and the increment form run the
// default shape whatever the edge asked for.
inline int tile_shape_of(const ofv_params &p)
{
    if (p.tile_edge == 0) return 0;
    if (p.path != OFV_PATH_FUSED || !block_supports(p.kernel_radius)) return -1;
    if (p.tile_edge == block_tile_edge(p.kernel_radius, 0)) return 0;
    if (p.tile_edge != block_tile_edge(p.kernel_radius, 1)) return -1;
    // the estimator variants are built with the default shape only
    return p.window == OFV_WINDOW_GAUSS || p.increment_form ? 0 : 1;
}
// True once a kernel of this handle recorded an expired TMA wait.
inline bool tma_expired(const ofv_handle *h)
{
    return h->tma_err_h && *static_cast<volatile int *>(h->tma_err_h) != 0;
}
}  // namespace ofv
