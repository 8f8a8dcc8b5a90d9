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
    unsigned long long *vmax;  // 2 ping-pong slots of max |v| (double bits)
    T dt, nu, gx, gy, gz, rho;
    double beta, vref;
};

template <typename T>
cudaError_t acm_launch_step(const AcmArgs<T> &a, int n_p, int parity, cudaStream_t st, int64_t *launches,
                            LaunchRecorder *rec = nullptr, int block = 256);
template <typename T>
cudaError_t acm_launch_vmax(const AcmArgs<T> &a, int slot, cudaStream_t st);
template <typename T>
cudaError_t acm_launch_predict_only(const AcmArgs<T> &a, cudaStream_t st);

}  // namespace rbf
