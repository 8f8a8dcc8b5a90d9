// lbm.cuh — argument block and launchers of the meshless LBM kernels.
#pragma once
#include "internal.cuh"

namespace rbf {

template <typename T>
struct LbmArgs {
    int64_t n, npad;
    int n_l;
    const int32_t *idx;    // SELL [slice][j][lane]
    const T *w;            // SELL [slice][pair][j][lane][2]
    const uint32_t *mask;  // unknown populations of wall nodes (bit k)
    const T *fin;          // f~_post: rest [npad], pairs [(q-1)/2][npad][2]
    T *fout;
    T tp_inv, tm_inv;      // 1/tau+, 1/tau-
    T gx, gy, gz;          // g_lb
};

const int *host_velocity_set(int q);
double host_lattice_weight(int q, int k);

// schedules of the fused step (same arithmetic, different thread mapping):
// node per thread with 256 / 128 threads per block; pair per warp with the
// stencil loop unrolled 5 / 3 / 6 / 2 deep
enum {
    LBM_NODE_PER_THREAD = 0, LBM_PAIR_PER_WARP = 1, LBM_NODE_PER_THREAD_128 = 2,
    LBM_PAIR_PER_WARP_U3 = 3, LBM_PAIR_PER_WARP_U6 = 4, LBM_PAIR_PER_WARP_U2 = 5, LBM_N_SCHEDULES = 6
};
template <typename T>
cudaError_t lbm_launch_step(const LbmArgs<T> &a, int q, cudaStream_t st, int variant = LBM_PAIR_PER_WARP);
cudaError_t lbm_launch_pack_f32(int64_t nc, int q, int n_l, const double *w, float *ws, cudaStream_t st);
cudaError_t lbm_launch_pack_f64(int64_t nc, int q, int n_l, const double *w, double *ws, cudaStream_t st);
template <typename T>
cudaError_t lbm_launch_init(const LbmArgs<T> &a, int q, cudaStream_t st);
cudaError_t lbm_launch_masks(int64_t n, int q, const uint8_t *type, const double *nrm, uint32_t *mask, cudaStream_t st);
template <typename T>
cudaError_t lbm_launch_export(int64_t n, int64_t npad, int q, const T *f, const int32_t *perm, double *out, cudaStream_t st);
template <typename T>
cudaError_t lbm_launch_import(int64_t n, int64_t npad, int q, T *f, const int32_t *perm, const double *in, cudaStream_t st);
template <typename T>
cudaError_t lbm_launch_macro(int64_t n, int64_t npad, int q, const T *f, const double g[3], double *out, cudaStream_t st);

}  // namespace rbf
