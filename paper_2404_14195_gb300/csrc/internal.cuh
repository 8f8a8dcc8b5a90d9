// internal.cuh — shared device helpers and the launchers each .cu file exports
// to the host orchestration in api.cu.  Nothing here is part of the public ABI.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#define RBF_SLICE 32          // SELL-C slice height: one warp, one node per lane
#define RBF_MAX_NL 64         // largest stencil
#define RBF_MAX_NP 35         // monomials for m <= 4
#define RBF_MAX_NS (RBF_MAX_NL + RBF_MAX_NP)
#define RBF_MAX_OPS 32        // right-hand sides per saddle system

namespace rbf {

// Displacement to the nearest periodic image, cell side 1.  Exact for |d| <= 1.
__device__ __forceinline__ double mimg(double d) { return d - rint(d); }

// Squared distance without contraction, so that neighbour ordering is bitwise
// reproducible (the kNN tie-break compares these values exactly).
__device__ __forceinline__ double dist2_nofma(double dx, double dy, double dz) {
    return __dadd_rn(__dadd_rn(__dmul_rn(dx, dx), __dmul_rn(dy, dy)), __dmul_rn(dz, dz));
}

// Index of SELL-C element (slice s, operator o, stencil column j, lane l) in an
// array with n_ops operators and n_l columns per slice.
__host__ __device__ __forceinline__ int64_t sell_at(int64_t s, int o, int j, int lane, int n_ops, int n_l) {
    return (((s * n_ops + o) * (int64_t)n_l + j) << 5) + lane;
}

// Operator kinds of the weight solver: L applied at y = x_c + off.
enum OpKind { OP_INTERP = 0, OP_DX = 1, OP_DY = 2, OP_DZ = 3, OP_LAP = 4 };
struct OpSpec {
    int kind;
    double off[3];
};

// Records a CUDA event pair around each kernel launch (eager launches only) and
// the kernel class of each pair, for per-launch device timing.
struct LaunchRecorder {
    cudaEvent_t *ev = nullptr;  // 2 * cap events
    int *cls = nullptr;         // cap classes
    int cap = 0, count = 0;
    void begin(cudaStream_t st, int c) {
        if (count < cap) { cudaEventRecord(ev[2 * count], st); cls[count] = c; }
    }
    void end(cudaStream_t st) {
        if (count < cap) { cudaEventRecord(ev[2 * count + 1], st); ++count; }
    }
};

// ---- launchers (all asynchronous on `st`; they return cudaGetLastError()) ----
// knn.cu
cudaError_t launch_morton_keys(int64_t n, const double *xyz, uint64_t *keys, int32_t *vals, int64_t npow,
                               cudaStream_t st);
cudaError_t launch_bitonic_sort(uint64_t *keys, int32_t *vals, int64_t npow, cudaStream_t st, int64_t *launches);
cudaError_t launch_gather_nodes(int64_t n, const int32_t *perm, const double *xyz, const uint8_t *type,
                                const double *nrm, double *xyz_s, uint8_t *type_s, double *nrm_s,
                                int32_t *iperm, cudaStream_t st);
cudaError_t launch_scan_i32(const int32_t *in, int32_t *out, int64_t n, int32_t *tmp, int64_t tmp_len,
                            cudaStream_t st, int64_t *launches);
int64_t scan_tmp_len(int64_t n);
cudaError_t launch_cell_count(int64_t n, const double *xyz, int G, int32_t *cell_of, int32_t *count,
                              cudaStream_t st);
cudaError_t launch_cell_fill(int64_t n, const int32_t *cell_of, const int32_t *start, int32_t *fill,
                             int32_t *items, cudaStream_t st);
cudaError_t launch_flag_compact(int64_t n, const uint8_t *type, uint8_t want, const int32_t *scan,
                                int32_t *list, cudaStream_t st);
cudaError_t launch_type_flags(int64_t n, const uint8_t *type, uint8_t want, int32_t *flags, cudaStream_t st);
// kNN of nq query points (qxyz, or the nodes qnode[] when qxyz == NULL) among the
// sorted nodes; results sorted by (d^2, orig index); fluid_only skips wall nodes.
// out row stride `ld`, first column `col0`.
cudaError_t launch_knn(int64_t nq, const double *qxyz, const int32_t *qnode, const double *xyz,
                       const int32_t *perm, const uint8_t *type, int fluid_only, int G,
                       const int32_t *cell_start, const int32_t *cell_items, int n_l, int32_t *out,
                       int ld, int col0, int32_t *status, cudaStream_t st);

// weights.cu
cudaError_t launch_weights(int64_t nc, const double *xyz, const double *cxyz, const int32_t *cnode,
                           int centre_is_node, int n_l, const int32_t *idx, int k, int m, int n_ops,
                           const OpSpec *ops, int refine, double *w, double *delta, int32_t *n_sing,
                           cudaStream_t st);

// one entry of a multi-set weight launch: nc centres, centre c = node cnode[c] of
// xyz with stencil idx[c * n_l ..] -> w[(c * n_ops + o) * n_l + j], delta[c]
struct WeightJob {
    int64_t nc;
    const double *xyz;
    const int32_t *cnode;
    int n_l;
    const int32_t *idx;
    double *w;
    double *delta;
};
cudaError_t launch_weights_multi(int njobs, const WeightJob *jobs_dev, const int64_t *prefix_dev, int64_t ntot,
                                 int max_n_l, int k, int m, int n_ops, const OpSpec *ops, int refine, int32_t *n_sing,
                                 cudaStream_t st);

// pack.cu (in weights.cu): FP64 row weights [c][o][j] -> SELL T [s][o][j][lane]
cudaError_t launch_pack_f32(int64_t nc, int n_ops, int o0, int n_out, int n_l, const double *w, float *ws,
                            cudaStream_t st);
cudaError_t launch_pack_f64(int64_t nc, int n_ops, int o0, int n_out, int n_l, const double *w, double *ws,
                            cudaStream_t st);
cudaError_t launch_pack_idx(int64_t nc, int n_l, const int32_t *idx, int32_t *is, cudaStream_t st);
// FP32 copies of weight rows with each row's exact sum kept (values returned as
// doubles); wall normal-derivative rows [nb][n_l] in FP64
cudaError_t launch_round_rows_f32(int64_t nrows, int n_l, const double *w, double *out, cudaStream_t st);
cudaError_t launch_normal_rows(int64_t nb, int n_l, const int32_t *wall, const double *nrm, const double *wg,
                               double *out, cudaStream_t st);
// wall normal-derivative weights n . (wx, wy, wz) -> SELL T
cudaError_t launch_pack_normal_f32(int64_t nb, int n_l, const int32_t *wall, const double *nrm,
                                   const double *wg, float *ws, cudaStream_t st);
cudaError_t launch_pack_normal_f64(int64_t nb, int n_l, const int32_t *wall, const double *nrm,
                                   const double *wg, double *ws, cudaStream_t st);

// reduce.cu
cudaError_t launch_min_f64(const double *in, int64_t n, double *partial, double *out, cudaStream_t st);
cudaError_t launch_sum_f64(const double *in, int64_t n, int stride, int ncomp, double *partial, double *out,
                           cudaStream_t st);

}  // namespace rbf
