// ctx.cuh — the device-resident state of one case (struct rbf_ctx) and the RAII
// device array used by the host orchestration.  Private to the library.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include <string>

#include "rbfgb.h"
#include "internal.cuh"
#include "lbm.cuh"

namespace rbf {

template <typename T>
struct DevArr {
    T *p = nullptr;
    size_t n = 0;
    DevArr() = default;
    DevArr(const DevArr &) = delete;
    DevArr &operator=(const DevArr &) = delete;
    ~DevArr() { release(); }
    void release() {
        if (p) cudaFree(p);
        p = nullptr;
        n = 0;
    }
    cudaError_t alloc(size_t m) {
        release();
        if (m == 0) return cudaSuccess;
        cudaError_t e = cudaMalloc((void **)&p, m * sizeof(T));
        if (e == cudaSuccess) n = m; else p = nullptr;
        return e;
    }
    cudaError_t zero(cudaStream_t st) { return n ? cudaMemsetAsync(p, 0, n * sizeof(T), st) : cudaSuccess; }
    void swap(DevArr &o) {
        T *tp = p; p = o.p; o.p = tp;
        size_t tn = n; n = o.n; o.n = tn;
    }
};

}  // namespace rbf

struct rbf_ctx {
    template <typename T> using DevArr = rbf::DevArr<T>;
    int device = 0;
    cudaStream_t st = nullptr;
    bool own_stream = false;
    std::string err;
    int64_t launches = 0;
    // nodes (device arrays in Morton order)
    int64_t n = 0, npad = 0, nb = 0, nf = 0;
    DevArr<double> xyz, nrm;
    DevArr<uint8_t> type;
    DevArr<int32_t> perm, iperm, wall, iota;
    bool has_sphere = false;
    double c[3] = {0.5, 0.5, 0.5}, r = 0.0;
    // stencils
    int G = 0, n_l = 0;
    DevArr<int32_t> cstart, citems, idx, idxb, idxw, idx_sell, idxb_sell;
    // weights
    bool weights_ok = false;
    int solver = -1, q = 0, phs_k = 0, mono_m = 0, n_ops = 0;
    double dx = 0.0, h_min = 0.0;
    int lbm_rule = 0;  // unknown populations at wall nodes: 0 e_k . n > 0, 1 departure point in the solid
    DevArr<double> w64, wgb64, wgw64, delta;
    DevArr<float> ws32, wn32;
    DevArr<double> ws64, wn64;
    DevArr<uint32_t> mask;
    // fields
    bool inited = false;
    int prec = RBF_FP64;
    rbf_params prm{};
    double dt = 0.0, vref = 0.0, beta = 10.0, rho = 1.0;
    int n_p = 3, parity = 0;
    DevArr<float> a32[10];
    DevArr<float> l32[10];   // RBF_FP32C: low words of a32 (allocated only in that mode)
    DevArr<double> a64[10];
    DevArr<unsigned long long> vmax;
    double tp = 0.8, tm = 1.125, gl[3] = {0, 0, 0}, lbm_dt = 0.0;
    DevArr<float> f32[2];
    DevArr<double> f64[2];
    int cur = 0;
    // RBF_FP32R (LBM): f = f64[0] (FP64 base) + f32[cur] (FP32 correction); f64[1] is
    // scratch; rr the FP32 residual of the last refresh; a refresh every refine_m
    // steps, refine_phase steps since the last one
    DevArr<float> rr;
    int refine_m = 64, refine_phase = 0;
    // probes
    int m_p = 0;
    int64_t np_fluid = 0;
    DevArr<double> pxyz, pw;
    DevArr<int32_t> pidx;
    double *static_flux = nullptr;  // device address of rbf_permeability_static's file-scope scratch
    // scratch
    DevArr<double> partial, scal, mac, stage;  // stage: host <-> device field transfers
    DevArr<int32_t> status;
    // graph of `gsteps` steps
    cudaGraphExec_t gexec = nullptr;
    int gsteps = 0, gparity = -1, gcur = -1, gprec = -1, gvariant = -1, gphase = -1;
    int variant = rbf::LBM_PAIR_PER_WARP;  // schedule of the fused LBM step
    int lbm_layout = rbf::LBM_LAYOUT_PAIRS;  // layout of f32 / f64 (follows the schedule)
    int acm_code = 256;               // ACM sweeps: threads per block + 1000 x lanes per node (0: one)
    int persist_block = 256;          // threads per block of the persistent ACM driver
    int persist_cluster = 0;          // > 0: run it as one cluster of that many CTAs (8 or 16)
    int persist_group = 1;            // lanes per node of its sweeps (1, 2, 4, 8)
    double persist_ms = 0.0;          // device time of its last launch
    uint64_t wait_ns = 2000000000ull; // wall-clock limit of one grid-barrier wait of that driver
    int gblock = -1;
    cudaEvent_t ev0 = nullptr, ev1 = nullptr;
    double last_ms = 0.0;
    int64_t last_steps = 0;
    int64_t last_kernel_launches = 0;
};

