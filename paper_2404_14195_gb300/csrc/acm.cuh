// acm.cuh — argument block and launchers of the ACM step kernels.
#pragma once
#include "internal.cuh"

namespace rbf {

template <typename T>
struct AcmArgs {
    int64_t n, nb;
    int n_l;
    const int32_t *idx;   // SELL [slice][j][lane], all nodes
    const T *w;           // SELL [slice][4][j][lane]: d/dx, d/dy, d/dz, Laplacian
    const uint8_t *type;  // 0 fluid, 1 wall
    const int32_t *wall;  // wall node indices (nb)
    const int32_t *idxb;  // SELL over wall nodes: Neumann stencils
    const T *wn;          // SELL over wall nodes: normal-derivative weights
    T *u, *v, *w_, *p;    // velocity and pressure
    T *us, *vs, *ws;      // intermediate velocity v'
    // compensated state (null unless the context runs RBF_FP32C): low words of
    // u, v, w, p, u', v', w'; a field's value is then hi + lo
    T *ul, *vl, *wl, *pl, *usl, *vsl, *wsl;
    unsigned long long *vmax;  // 2 ping-pong slots of max |v| (double bits)
    T dt, nu, gx, gy, gz, rho;
    double beta, vref;
};

// (hi, lo) += d for a value carried as the unevaluated sum hi + lo.  The rounding
// error of hi + d (Knuth's TwoSum) joins lo and the pair is renormalised
// (Dekker's Fast2Sum), so increments far below one ulp of hi still accumulate
// instead of rounding away.  Explicit round-to-nearest adds keep the compiler
// from contracting them with the product that formed d.
__device__ __forceinline__ float add_rn(float a, float b) { return __fadd_rn(a, b); }
__device__ __forceinline__ float sub_rn(float a, float b) { return __fsub_rn(a, b); }
__device__ __forceinline__ double add_rn(double a, double b) { return __dadd_rn(a, b); }
__device__ __forceinline__ double sub_rn(double a, double b) { return __dsub_rn(a, b); }
template <typename T>
__device__ __forceinline__ void comp_add(T &hi, T &lo, T d) {
    const T s = add_rn(hi, d);
    const T bb = sub_rn(s, hi);
    const T err = add_rn(sub_rn(hi, sub_rn(s, bb)), sub_rn(d, bb));
    const T l = add_rn(lo, err);
    hi = add_rn(s, l);
    lo = sub_rn(l, sub_rn(hi, s));
}

// Sum over the G consecutive lanes that share a node (G = 1: the value itself).
template <typename T, int G>
__device__ __forceinline__ T group_sum(T v) {
#pragma unroll
    for (int off = G >> 1; off > 0; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
    return v;
}

// schedule code of the ACM sweeps: threads per block (64, 128, 256) + 1000 x
// lanes per node (0 for one lane, 2 or 4)
inline bool acm_code_ok(int code) {
    const int block = code % 1000, group = code / 1000;
    return code > 0 && (block == 64 || block == 128 || block == 256) && (group == 0 || group == 2 || group == 4);
}

template <typename T>
cudaError_t acm_launch_step(const AcmArgs<T> &a, int n_p, int parity, cudaStream_t st, int64_t *launches,
                            LaunchRecorder *rec = nullptr, int code = 256);
template <typename T>
cudaError_t acm_launch_vmax(const AcmArgs<T> &a, int slot, cudaStream_t st);
template <typename T>
cudaError_t acm_launch_predict_only(const AcmArgs<T> &a, cudaStream_t st);

}  // namespace rbf
