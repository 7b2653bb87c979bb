// Host launcher of the block-tiled iteration kernel.
#include <cstring>

#include "k_block.cuh"

namespace ofv {

extern template cudaError_t launch_block_t<float, false>(const BlockParams &, int, int, cudaStream_t, int, int);
extern template cudaError_t launch_block_t<float, true>(const BlockParams &, int, int, cudaStream_t, int, int);
extern template cudaError_t launch_block_t<__half, false>(const BlockParams &, int, int, cudaStream_t, int, int);
extern template cudaError_t launch_block_t<__half, true>(const BlockParams &, int, int, cudaStream_t, int, int);
extern template cudaError_t launch_block_t<__nv_bfloat16, false>(const BlockParams &, int, int, cudaStream_t, int, int);
extern template cudaError_t launch_block_t<__nv_bfloat16, true>(const BlockParams &, int, int, cudaStream_t, int, int);

bool block_supports(int kr) { return kr >= 1 && kr <= kBlockMaxKR; }

// The solve's reciprocal on its own, for its error test.
__global__ void k_recip(const float *x, float *y, int n)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) y[i] = recip_newton(x[i]);
}

cudaError_t launch_recip(const float *x, float *y, int n, cudaStream_t s)
{
    if (n < 0) return cudaErrorInvalidValue;
    if (n == 0) return cudaSuccess;
    k_recip<<<(n + 255) / 256, 256, 0, s>>>(x, y, n);
    return cudaGetLastError();
}

cudaError_t launch_iter_block(const IterArgs *a, int npairs, int store, int mode, cudaStream_t s,
                              const CUtensorMap *const *tm, int *err, int by0, int nby, int shape)
{
    if (npairs < 1 || npairs > kBlockMaxBatch || !block_supports(a[0].kr)) return cudaErrorInvalidValue;
    BlockParams p;
    memset(&p, 0, sizeof p);
    for (int k = 0; k < npairs; ++k) p.a[k] = a[k];
    p.mode = mode;
    p.err = err;
    p.by0 = by0;
    p.use_tma = 0;
    if (tm) {
        p.use_tma = 1;
        for (int k = 0; k < npairs; ++k) {
            if (!tm[2 * k] || !tm[2 * k + 1]) {
                p.use_tma = 0;
                break;
            }
            p.tm[k][0] = *tm[2 * k];
            p.tm[k][1] = *tm[2 * k + 1];
        }
    }
    // the kernels with variant code only when a variant is on (uniform per launch)
    const bool var = a[0].inc || a[0].gauss || a[0].mask || a[0].s_out;
    // the variant kernels have the default tile shape only; tensor maps made
    // for another shape's box would not match theirs
    if (var && shape != 0) p.use_tma = 0;
    switch (store) {
    case ST_F16: return var ? launch_block_t<__half, true>(p, a[0].kr, npairs, s, nby, var ? 0 : shape)
                            : launch_block_t<__half, false>(p, a[0].kr, npairs, s, nby, var ? 0 : shape);
    case ST_BF16: return var ? launch_block_t<__nv_bfloat16, true>(p, a[0].kr, npairs, s, nby, var ? 0 : shape)
                             : launch_block_t<__nv_bfloat16, false>(p, a[0].kr, npairs, s, nby, var ? 0 : shape);
    default: return var ? launch_block_t<float, true>(p, a[0].kr, npairs, s, nby, var ? 0 : shape)
                        : launch_block_t<float, false>(p, a[0].kr, npairs, s, nby, var ? 0 : shape);
    }
}

namespace {
template <typename T, int KS>
void box_ks(int *cols, int *rows)
{
    *cols = StageShape<T, KS>::SP;
    *rows = StageShape<T, KS>::SHB;
}

template <typename T>
void box_of(int kr, int shape, int *cols, int *rows)
{
    *cols = *rows = 0;
    if (kr < 1 || kr > kBlockMaxKR || shape < 0 || shape > 1) return;
    switch (kr + 16 * shape) {
#define OFV_BOX_CASE(K) \
    case K: box_ks<T, K>(cols, rows); return;
    OFV_BOX_CASE(1) OFV_BOX_CASE(2) OFV_BOX_CASE(3) OFV_BOX_CASE(4) OFV_BOX_CASE(5)
    OFV_BOX_CASE(6) OFV_BOX_CASE(7) OFV_BOX_CASE(8) OFV_BOX_CASE(9) OFV_BOX_CASE(10)
    OFV_BOX_CASE(17) OFV_BOX_CASE(18) OFV_BOX_CASE(19) OFV_BOX_CASE(20) OFV_BOX_CASE(21)
    OFV_BOX_CASE(22) OFV_BOX_CASE(23) OFV_BOX_CASE(24) OFV_BOX_CASE(25) OFV_BOX_CASE(26)
#undef OFV_BOX_CASE
    default: return;
    }
}
}  // namespace

void block_stage_box(int store, int kr, int *cols, int *rows, int shape)
{
    switch (store) {
    case ST_F16: box_of<__half>(kr, shape, cols, rows); break;
    case ST_BF16: box_of<__nv_bfloat16>(kr, shape, cols, rows); break;
    default: box_of<float>(kr, shape, cols, rows); break;
    }
}

}  // namespace ofv
