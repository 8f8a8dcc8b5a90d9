// lbm.cu — meshless lattice Boltzmann step, TRT collision (MLBM section).
//
// The paper's step is COLLIDE over all nodes, then STREAM: each population is
// interpolated (RBF-FD, L = 1) from the post-collision field at its departure
// point x_i - dx e_k (Eq. LBM_streaming), wall nodes replace the populations
// whose departure point lies in the solid (e_k . n > 0) by the opposite streamed
// population (Eq. interpolated_bounceback_mlbm), and moments follow (Eq.
// macro_var).  Here one kernel per step does, for each node, stream -> bounce-back
// -> moments -> TRT collision (Eqs. LBM_collision, feq, force_lbm) and writes the
// next post-collision populations, so the state between launches is f_post and
// each population is read and written once per step.
//
// Populations are stored shifted, f~_k = f_k - omega_k (the rho = 1, v = 0
// equilibrium).  Interpolation weights sum to one, so streaming commutes with the
// shift; collision only sees f - f_eq differences.  At the paper's low Mach
// numbers (g_lb ~ 1e-9) the shift keeps the FP32 populations' significant bits on
// the deviations instead of on omega_k.
//
// Layout: f~ SoA [q][n_pad]; stencil indices SELL [slice][j][lane]; weights SELL
// [slice][k-1][j][lane] (k = 1..q-1), one node per lane.
#include "lbm.cuh"

namespace rbf {

// Velocity sets in the paper's convention: odd k listed, e_k = -e_{k-1} for even k.
// D3Q15 as tabulated in the MLBM section; D3Q19 with the textbook weights.
__constant__ int c_e15[15][3] = {{0, 0, 0},  {1, 0, 0},  {-1, 0, 0}, {0, 1, 0},   {0, -1, 0},
                                 {0, 0, 1},  {0, 0, -1}, {1, 1, 1},  {-1, -1, -1}, {1, 1, -1},
                                 {-1, -1, 1}, {1, -1, 1}, {-1, 1, -1}, {1, -1, -1}, {-1, 1, 1}};
__constant__ int c_e19[19][3] = {{0, 0, 0},  {1, 0, 0},  {-1, 0, 0}, {0, 1, 0},  {0, -1, 0}, {0, 0, 1},  {0, 0, -1},
                                 {1, 1, 0},  {-1, -1, 0}, {1, -1, 0}, {-1, 1, 0}, {1, 0, 1},  {-1, 0, -1},
                                 {1, 0, -1}, {-1, 0, 1}, {0, 1, 1},  {0, -1, -1}, {0, 1, -1}, {0, -1, 1}};

template <int Q> struct VSet;
template <> struct VSet<19> {
    static __host__ __device__ constexpr double w(int k) { return k == 0 ? 1.0 / 3.0 : (k <= 6 ? 1.0 / 18.0 : 1.0 / 36.0); }
    static __device__ __forceinline__ int e(int k, int a) { return c_e19[k][a]; }
};
template <> struct VSet<15> {
    static __host__ __device__ constexpr double w(int k) { return k == 0 ? 2.0 / 9.0 : (k <= 6 ? 1.0 / 9.0 : 1.0 / 72.0); }
    static __device__ __forceinline__ int e(int k, int a) { return c_e15[k][a]; }
};

const int *host_velocity_set(int q) {
    static const int e15[15][3] = {{0, 0, 0},  {1, 0, 0},  {-1, 0, 0}, {0, 1, 0},   {0, -1, 0},
                                   {0, 0, 1},  {0, 0, -1}, {1, 1, 1},  {-1, -1, -1}, {1, 1, -1},
                                   {-1, -1, 1}, {1, -1, 1}, {-1, 1, -1}, {1, -1, -1}, {-1, 1, 1}};
    static const int e19[19][3] = {{0, 0, 0},  {1, 0, 0},  {-1, 0, 0}, {0, 1, 0},  {0, -1, 0}, {0, 0, 1},  {0, 0, -1},
                                   {1, 1, 0},  {-1, -1, 0}, {1, -1, 0}, {-1, 1, 0}, {1, 0, 1},  {-1, 0, -1},
                                   {1, 0, -1}, {-1, 0, 1}, {0, 1, 1},  {0, -1, -1}, {0, 1, -1}, {0, -1, 1}};
    return q == 15 ? &e15[0][0] : (q == 19 ? &e19[0][0] : nullptr);
}
double host_lattice_weight(int q, int k) { return q == 15 ? VSet<15>::w(k) : VSet<19>::w(k); }

// opposite of k: k+1 for odd k, k-1 for even k >= 2, 0 for 0
__host__ __device__ constexpr int opp(int k) { return k == 0 ? 0 : ((k & 1) ? k + 1 : k - 1); }

// unknown-population masks of the wall nodes: bit k set when e_k . n > 0
template <int Q>
__global__ void k_lbm_masks(int64_t n, const uint8_t *__restrict__ type, const double *__restrict__ nrm, uint32_t *mask) {
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n) return;
    uint32_t m = 0;
    if (type[i]) {
        for (int k = 1; k < Q; ++k) {
            double en = __dadd_rn(__dadd_rn(__dmul_rn((double)VSet<Q>::e(k, 0), nrm[3 * i]),
                                            __dmul_rn((double)VSet<Q>::e(k, 1), nrm[3 * i + 1])),
                                  __dmul_rn((double)VSet<Q>::e(k, 2), nrm[3 * i + 2]));
            if (en > 0.0) m |= 1u << k;
        }
    }
    mask[i] = m;
}

// TRT collision of one node in shifted variables; f[] in, f[] out (post-collision)
template <typename T, int Q>
__device__ __forceinline__ void trt_collide(T (&f)[Q], T tp_inv, T tm_inv, T gx, T gy, T gz) {
    T drho = 0, mx = 0, my = 0, mz = 0;
#pragma unroll
    for (int k = 0; k < Q; ++k) {
        drho += f[k];
        mx += (T)VSet<Q>::e(k, 0) * f[k];
        my += (T)VSet<Q>::e(k, 1) * f[k];
        mz += (T)VSet<Q>::e(k, 2) * f[k];
    }
    const T rho = (T)1 + drho;
    const T vx = mx / rho, vy = my / rho, vz = mz / rho;
    const T vv = vx * vx + vy * vy + vz * vz;
    const T base = rho * ((T)-1.5 * vv);
    {   // rest population: symmetric only, no force
        const T w0 = (T)VSet<Q>::w(0);
        const T feq0 = w0 * (drho + base);
        f[0] = f[0] - (f[0] - feq0) * tp_inv;
    }
#pragma unroll
    for (int k = 1; k < Q; k += 2) {
        const T wk = (T)VSet<Q>::w(k);
        const T ex = (T)VSet<Q>::e(k, 0), ey = (T)VSet<Q>::e(k, 1), ez = (T)VSet<Q>::e(k, 2);
        const T eu = ex * vx + ey * vy + ez * vz;
        const T eqp = wk * (drho + base + rho * ((T)4.5 * eu * eu));  // symmetric part of f~_eq
        const T eqm = wk * rho * ((T)3 * eu);                          // antisymmetric part
        const T fp = (T)0.5 * (f[k] + f[k + 1]);
        const T fm = (T)0.5 * (f[k] - f[k + 1]);
        const T dp = (fp - eqp) * tp_inv;
        const T dm = (fm - eqm) * tm_inv;
        const T F = wk * (T)3 * rho * (ex * gx + ey * gy + ez * gz);
        f[k] = f[k] - dp - dm + F;
        f[k + 1] = f[k + 1] - dp + dm - F;
    }
}

template <typename T, int Q>
__global__ void __launch_bounds__(256) k_lbm_step(LbmArgs<T> a) {
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= a.n) return;
    const int64_t s = i >> 5;
    const int lane = (int)(i & 31);
    const int n_l = a.n_l;
    const int64_t np = a.npad;
    const int32_t *__restrict__ ip = a.idx + ((s * n_l) << 5) + lane;
    const T *__restrict__ wp = a.w + ((s * (Q - 1) * (int64_t)n_l) << 5) + lane;
    const T *__restrict__ fin = a.fin;
    T f[Q];
#pragma unroll
    for (int k = 0; k < Q; ++k) f[k] = (T)0;
    for (int j = 0; j < n_l; ++j) {
        const int q = __ldg(ip + (j << 5));
#pragma unroll
        for (int k = 1; k < Q; ++k) f[k] += __ldg(wp + (((k - 1) * n_l + j) << 5)) * fin[k * np + q];
    }
    f[0] = fin[i];
    const uint32_t m = a.mask[i];
    if (m) {
#pragma unroll
        for (int k = 1; k < Q; ++k)
            if (m & (1u << k)) f[k] = f[opp(k)];
    }
    trt_collide<T, Q>(f, a.tp_inv, a.tm_inv, a.gx, a.gy, a.gz);
#pragma unroll
    for (int k = 0; k < Q; ++k) a.fout[k * np + i] = f[k];
}

// initial state: the collision of f_eq(rho = 1, v = 0) is f_eq + F_k, i.e.
// f~_post = 3 omega_k rho e_k . g (MLBM section's initial condition)
template <typename T, int Q>
__global__ void k_lbm_init(LbmArgs<T> a) {
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= a.npad) return;
    T f[Q];
#pragma unroll
    for (int k = 0; k < Q; ++k) f[k] = (T)0;
    trt_collide<T, Q>(f, a.tp_inv, a.tm_inv, a.gx, a.gy, a.gz);
#pragma unroll
    for (int k = 0; k < Q; ++k) a.fout[k * a.npad + i] = i < a.n ? f[k] : (T)0;
}

// populations <-> FP64 unshifted, caller's order (perm: sorted -> caller)
template <typename T, int Q>
__global__ void k_lbm_export(int64_t n, int64_t npad, const T *__restrict__ f, const int32_t *__restrict__ perm, double *out) {
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n) return;
    int64_t o = perm[i];
#pragma unroll
    for (int k = 0; k < Q; ++k) out[k * n + o] = (double)f[k * npad + i] + VSet<Q>::w(k);
}
template <typename T, int Q>
__global__ void k_lbm_import(int64_t n, int64_t npad, T *f, const int32_t *__restrict__ perm, const double *in) {
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n) return;
    int64_t o = perm[i];
#pragma unroll
    for (int k = 0; k < Q; ++k) f[k * npad + i] = (T)(in[k * n + o] - VSet<Q>::w(k));
}

// macroscopic fields from the post-collision state: rho is unchanged by the
// collision, the momentum gained rho g_lb, so v_lb = sum f e / rho - g_lb.
// out (sorted order) = (vx, vy, vz, rho - 1) in lattice units, FP64.
template <typename T, int Q>
__global__ void k_lbm_macro(int64_t n, int64_t npad, const T *__restrict__ f, double gx, double gy, double gz, double *out) {
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n) return;
    double d = 0, mx = 0, my = 0, mz = 0;
#pragma unroll
    for (int k = 0; k < Q; ++k) {
        double fk = (double)f[k * npad + i];
        d += fk;
        mx += VSet<Q>::e(k, 0) * fk; my += VSet<Q>::e(k, 1) * fk; mz += VSet<Q>::e(k, 2) * fk;
    }
    double rho = 1.0 + d;
    out[4 * i] = mx / rho - gx;
    out[4 * i + 1] = my / rho - gy;
    out[4 * i + 2] = mz / rho - gz;
    out[4 * i + 3] = d;
}

template <typename T>
cudaError_t lbm_launch_step(const LbmArgs<T> &a, int q, cudaStream_t st) {
    unsigned g = (unsigned)((a.n + 255) / 256);
    if (q == 19) k_lbm_step<T, 19><<<g, 256, 0, st>>>(a);
    else if (q == 15) k_lbm_step<T, 15><<<g, 256, 0, st>>>(a);
    else return cudaErrorInvalidValue;
    return cudaGetLastError();
}

template <typename T>
cudaError_t lbm_launch_init(const LbmArgs<T> &a, int q, cudaStream_t st) {
    unsigned g = (unsigned)((a.npad + 255) / 256);
    if (q == 19) k_lbm_init<T, 19><<<g, 256, 0, st>>>(a);
    else if (q == 15) k_lbm_init<T, 15><<<g, 256, 0, st>>>(a);
    else return cudaErrorInvalidValue;
    return cudaGetLastError();
}

cudaError_t lbm_launch_masks(int64_t n, int q, const uint8_t *type, const double *nrm, uint32_t *mask, cudaStream_t st) {
    unsigned g = (unsigned)((n + 255) / 256);
    if (q == 19) k_lbm_masks<19><<<g, 256, 0, st>>>(n, type, nrm, mask);
    else if (q == 15) k_lbm_masks<15><<<g, 256, 0, st>>>(n, type, nrm, mask);
    else return cudaErrorInvalidValue;
    return cudaGetLastError();
}

template <typename T>
cudaError_t lbm_launch_export(int64_t n, int64_t npad, int q, const T *f, const int32_t *perm, double *out, cudaStream_t st) {
    unsigned g = (unsigned)((n + 255) / 256);
    if (q == 19) k_lbm_export<T, 19><<<g, 256, 0, st>>>(n, npad, f, perm, out);
    else k_lbm_export<T, 15><<<g, 256, 0, st>>>(n, npad, f, perm, out);
    return cudaGetLastError();
}
template <typename T>
cudaError_t lbm_launch_import(int64_t n, int64_t npad, int q, T *f, const int32_t *perm, const double *in, cudaStream_t st) {
    unsigned g = (unsigned)((n + 255) / 256);
    if (q == 19) k_lbm_import<T, 19><<<g, 256, 0, st>>>(n, npad, f, perm, in);
    else k_lbm_import<T, 15><<<g, 256, 0, st>>>(n, npad, f, perm, in);
    return cudaGetLastError();
}
template <typename T>
cudaError_t lbm_launch_macro(int64_t n, int64_t npad, int q, const T *f, const double g[3], double *out, cudaStream_t st) {
    unsigned gr = (unsigned)((n + 255) / 256);
    if (q == 19) k_lbm_macro<T, 19><<<gr, 256, 0, st>>>(n, npad, f, g[0], g[1], g[2], out);
    else k_lbm_macro<T, 15><<<gr, 256, 0, st>>>(n, npad, f, g[0], g[1], g[2], out);
    return cudaGetLastError();
}

#define RBF_LBM_INST(T)                                                                                         \
    template cudaError_t lbm_launch_step<T>(const LbmArgs<T> &, int, cudaStream_t);                             \
    template cudaError_t lbm_launch_init<T>(const LbmArgs<T> &, int, cudaStream_t);                             \
    template cudaError_t lbm_launch_export<T>(int64_t, int64_t, int, const T *, const int32_t *, double *,      \
                                              cudaStream_t);                                                    \
    template cudaError_t lbm_launch_import<T>(int64_t, int64_t, int, T *, const int32_t *, const double *,      \
                                              cudaStream_t);                                                    \
    template cudaError_t lbm_launch_macro<T>(int64_t, int64_t, int, const T *, const double *, double *, cudaStream_t);
RBF_LBM_INST(float)
RBF_LBM_INST(double)

}  // namespace rbf
