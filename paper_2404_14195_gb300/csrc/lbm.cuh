// lbm.cuh — argument block and launchers of the meshless LBM kernels.
#pragma once
#include "internal.cuh"

namespace rbf {

// population layouts (see pop_at in lbm.cu)
enum { LBM_LAYOUT_PAIRS = 0, LBM_LAYOUT_NODES = 1 };
// values per node record in the node layout: q rounded up to a multiple of 4
__host__ __device__ constexpr int lbm_rec_len(int q) { return (q + 3) & ~3; }

template <typename T>
struct LbmArgs {
    int64_t n, npad;
    int n_l;
    int layout;            // LBM_LAYOUT_PAIRS or LBM_LAYOUT_NODES
    const int32_t *idx;    // SELL [slice][j][lane]
    const T *w;            // SELL [slice][pair][j][lane][2]
    const uint32_t *mask;  // unknown populations of wall nodes (bit k)
    const T *fin;          // f~_post: pairs layout rest [npad], pairs [(q-1)/2][npad][2];
                           // node layout [npad][lbm_rec_len(q)]
    T *fout;
    T tp_inv, tm_inv;      // 1/tau+, 1/tau-
    T gx, gy, gz;          // g_lb
    // refined FP32 (RBF_FP32R): the residual r added to every post-collision
    // population (same layout as fout), else null; FP32 only
    const T *radd = nullptr;
};

const int *host_velocity_set(int q);
double host_lattice_weight(int q, int k);

// schedules of the fused step (same arithmetic, different thread mapping):
// on the pairs layout, node per thread with 256 / 128 threads per block and
// pair per warp with the stencil loop unrolled 5 / 3 / 6 / 2 deep; on the node
// layout, node per thread with 256 threads, registers as needed or capped for
// five blocks per SM
enum {
    LBM_NODE_PER_THREAD = 0, LBM_PAIR_PER_WARP = 1, LBM_NODE_PER_THREAD_128 = 2,
    LBM_PAIR_PER_WARP_U3 = 3, LBM_PAIR_PER_WARP_U6 = 4, LBM_PAIR_PER_WARP_U2 = 5,
    LBM_RECORD_PER_THREAD = 6, LBM_RECORD_PER_THREAD_OCC = 7,
    // node layout, node per thread, 64-register kernel in blocks of 128 / 64 threads (finer
    // blocks spread the nodes more evenly over the SMs in a one-wave launch)
    LBM_RECORD_PER_THREAD_128 = 8, LBM_RECORD_PER_THREAD_64 = 9,
    // as 6, launched as a programmatic dependent launch: the next step's blocks are
    // scheduled while this step drains and wait on the hardware grid dependency
    LBM_RECORD_PER_THREAD_PDL = 10, LBM_N_SCHEDULES = 11
};
__host__ __device__ constexpr int lbm_layout_of(int schedule) {
    return schedule >= LBM_RECORD_PER_THREAD ? LBM_LAYOUT_NODES : LBM_LAYOUT_PAIRS;
}
template <typename T>
cudaError_t lbm_launch_step(const LbmArgs<T> &a, int q, cudaStream_t st, int variant = LBM_PAIR_PER_WARP);
// populations from layout `from` (src) to layout `to` (dst, a different buffer)
template <typename T>
cudaError_t lbm_launch_relayout(int64_t npad, int q, int from, const T *src, int to, T *dst, cudaStream_t st);
cudaError_t lbm_launch_pack_f32(int64_t nc, int q, int n_l, const double *w, float *ws, cudaStream_t st);
cudaError_t lbm_launch_pack_f64(int64_t nc, int q, int n_l, const double *w, double *ws, cudaStream_t st);
template <typename T>
cudaError_t lbm_launch_init(const LbmArgs<T> &a, int q, cudaStream_t st);
cudaError_t lbm_launch_masks(int64_t n, int q, const uint8_t *type, const double *nrm, uint32_t *mask, cudaStream_t st);
// solid-check unknown-population masks (departure point inside the sphere array)
cudaError_t lbm_launch_masks_solid(int64_t n, int q, const uint8_t *type, const double *xyz, const double c[3], double r,
                                  double dx, uint32_t *mask, cudaStream_t st);
// out[perm[i]] = in[i]
cudaError_t launch_scatter_u32(int64_t n, const int32_t *perm, const uint32_t *in, uint32_t *out, cudaStream_t st);
template <typename T>
cudaError_t lbm_launch_export(int64_t n, int64_t npad, int layout, int q, const T *f, const int32_t *perm, double *out,
                              cudaStream_t st);
template <typename T>
cudaError_t lbm_launch_import(int64_t n, int64_t npad, int layout, int q, T *f, const int32_t *perm, const double *in,
                              cudaStream_t st);
template <typename T>
cudaError_t lbm_launch_macro(int64_t n, int64_t npad, int layout, int q, const T *f, const double g[3], double *out,
                             cudaStream_t st);
// refined FP32 state f = base (FP64) + delta (FP32), elementwise over `tot` stored
// values (either layout, padding included): base += delta; r = fl(fnew - base) and
// delta = r; out = base + delta
cudaError_t lbm_launch_refine_fold(int64_t tot, double *base, const float *delta, cudaStream_t st);
cudaError_t lbm_launch_refine_residual(int64_t tot, const double *fnew, const double *base, float *r, float *delta,
                                       cudaStream_t st);
cudaError_t lbm_launch_refine_combine(int64_t tot, const double *base, const float *delta, double *out,
                                      cudaStream_t st);

}  // namespace rbf
