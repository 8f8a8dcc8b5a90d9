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
// Layout: f~ rest population [n_pad], then the (q-1)/2 opposite pairs
// interleaved [pair][n_pad][2]; stencil indices SELL [slice][j][lane]; weights
// SELL [slice][pair][j][lane][2], one node per lane.
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

// Population k of node i.  Pairs layout: the rest population in [0, npad),
// then the opposite pairs (k, k') = (2p+1, 2p+2) interleaved, pair p at
// npad + 2 (p npad + i) + {0, 1}.  Node layout: the q populations of node i in
// one record of lbm_rec_len(q) values at i lbm_rec_len(q) (padding zero), so a
// neighbour's populations arrive in a few 16-byte loads.
__host__ __device__ __forceinline__ int64_t pop_at(int k, int64_t i, int64_t npad, int layout, int q) {
    if (layout == LBM_LAYOUT_NODES) return i * lbm_rec_len(q) + k;
    return k == 0 ? i : npad + 2 * ((int64_t)((k - 1) >> 1) * npad + i) + ((k - 1) & 1);
}

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

// Solid-check rule of the touching-limit study: at a wall node x, bit k is set
// when the departure point x + dx e_k' = x - dx e_k lies inside the solid, i.e.
// closer than r to the nearest centre of the periodic sphere array.  Products and
// sums in round-to-nearest without contraction, so the decision is the same
// as an FP64 evaluation in this order.
template <int Q>
__global__ void k_lbm_masks_solid(int64_t n, const uint8_t *__restrict__ type, const double *__restrict__ xyz,
                                  double c0, double c1, double c2, double r, double dx, uint32_t *mask) {
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n) return;
    uint32_t m = 0;
    if (type[i]) {
        const double c[3] = {c0, c1, c2};
        const double r2 = __dmul_rn(r, r);
        for (int k = 1; k < Q; ++k) {
            double d[3];
            for (int a = 0; a < 3; ++a) {
                const double p = __dsub_rn(xyz[3 * i + a], __dmul_rn(dx, (double)VSet<Q>::e(k, a)));
                const double v = __dsub_rn(p, c[a]);
                d[a] = __dsub_rn(v, rint(v));
            }
            const double s = __dadd_rn(__dadd_rn(__dmul_rn(d[0], d[0]), __dmul_rn(d[1], d[1])), __dmul_rn(d[2], d[2]));
            if (s < r2) m |= 1u << k;
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

template <typename T> struct Vec2;
template <> struct Vec2<float> { using type = float2; };
template <> struct Vec2<double> { using type = double2; };

// One thread per node: all q populations of the node in registers.  RA: add the
// residual a.radd to the post-collision populations (refined FP32).
template <typename T, int Q, bool RA = false>
__global__ void __launch_bounds__(256) k_lbm_step(LbmArgs<T> a) {
    using V = typename Vec2<T>::type;
    constexpr int NP = (Q - 1) / 2;
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= a.n) return;
    const int64_t s = i >> 5;
    const int lane = (int)(i & 31);
    const int n_l = a.n_l;
    const int64_t np = a.npad;
    const int32_t *__restrict__ ip = a.idx + ((s * n_l) << 5) + lane;
    const V *__restrict__ wp = reinterpret_cast<const V *>(a.w) + ((s * NP * (int64_t)n_l) << 5) + lane;
    const V *__restrict__ fp2 = reinterpret_cast<const V *>(a.fin + np);
    T f[Q];
#pragma unroll
    for (int k = 0; k < Q; ++k) f[k] = (T)0;
    for (int j = 0; j < n_l; ++j) {
        const int q = __ldg(ip + (j << 5));
#pragma unroll
        for (int p = 0; p < NP; ++p) {
            const V w2 = __ldcs(wp + ((p * n_l + j) << 5));
            const V g2 = __ldg(fp2 + p * np + q);
            f[2 * p + 1] += w2.x * g2.x;
            f[2 * p + 2] += w2.y * g2.y;
        }
    }
    f[0] = a.fin[i];
    const uint32_t m = a.mask[i];
    if (m) {
#pragma unroll
        for (int k = 1; k < Q; ++k)
            if (m & (1u << k)) f[k] = f[opp(k)];
    }
    trt_collide<T, Q>(f, a.tp_inv, a.tm_inv, a.gx, a.gy, a.gz);
    if constexpr (RA) {
        f[0] += a.radd[i];
        const V *__restrict__ r2 = reinterpret_cast<const V *>(a.radd + np);
#pragma unroll
        for (int p = 0; p < NP; ++p) {
            const V r = r2[p * np + i];
            f[2 * p + 1] += r.x;
            f[2 * p + 2] += r.y;
        }
    }
    a.fout[i] = f[0];
    V *__restrict__ op2 = reinterpret_cast<V *>(a.fout + np);
#pragma unroll
    for (int p = 0; p < NP; ++p) {
        V o;
        o.x = f[2 * p + 1];
        o.y = f[2 * p + 2];
        op2[p * np + i] = o;
    }
}

template <typename T> struct Vec16;  // 16-byte vector of T
template <> struct Vec16<float> {
    using type = float4;
    static constexpr int n = 4;
    static __device__ __forceinline__ void get(const float4 &v, float *d) { d[0] = v.x; d[1] = v.y; d[2] = v.z; d[3] = v.w; }
    static __device__ __forceinline__ float4 make(const float *d) { return make_float4(d[0], d[1], d[2], d[3]); }
};
template <> struct Vec16<double> {
    using type = double2;
    static constexpr int n = 2;
    static __device__ __forceinline__ void get(const double2 &v, double *d) { d[0] = v.x; d[1] = v.y; }
    static __device__ __forceinline__ double2 make(const double *d) { return make_double2(d[0], d[1]); }
};

// One thread per node on the node layout: each stencil column costs one index
// load, (q-1)/2 coalesced 8-byte weight loads and lbm_rec_len(q) / 4 16-byte
// loads of the neighbour's record (FP32 D3Q19: 5, against 9 pair gathers on the
// pairs layout).  MINB: blocks of 256 threads the compiler must fit on one SM,
// i.e. a register cap (FP32: 4 -> 64 registers, no spills; 5 -> 48 registers, a
// few spills, more warps in flight).  Same arithmetic, in the same order, as
// k_lbm_step.  PDL: launched as a programmatic dependent of the previous kernel in
// the stream; every block first lets the next step's grid be scheduled, then waits
// until the previous grid has completed and its writes are visible, before it
// touches global memory.
template <typename T, int Q, int MINB, bool RA = false, bool PDL = false>
__global__ void __launch_bounds__(256, MINB) k_lbm_step_records(LbmArgs<T> a) {
    using V = typename Vec2<T>::type;
    using W = Vec16<T>;
    using V16 = typename W::type;
    constexpr int NP = (Q - 1) / 2;
    constexpr int RL = lbm_rec_len(Q);
    constexpr int NV = RL / W::n;
    if constexpr (PDL) {
        asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
        asm volatile("griddepcontrol.wait;" ::: "memory");
    }
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= a.n) return;
    const int64_t s = i >> 5;
    const int lane = (int)(i & 31);
    const int n_l = a.n_l;
    const int32_t *__restrict__ ip = a.idx + ((s * n_l) << 5) + lane;
    const V *__restrict__ wp = reinterpret_cast<const V *>(a.w) + ((s * NP * (int64_t)n_l) << 5) + lane;
    const V16 *__restrict__ rec = reinterpret_cast<const V16 *>(a.fin);
    T f[Q];
#pragma unroll
    for (int k = 0; k < Q; ++k) f[k] = (T)0;
#pragma unroll 1
    for (int j = 0; j < n_l; ++j) {  // not unrolled: keeps the register cap without spills
        const int q = __ldg(ip + (j << 5));
        T g[RL];
#pragma unroll
        for (int v = 0; v < NV; ++v) W::get(__ldg(rec + (int64_t)q * NV + v), g + v * W::n);
#pragma unroll
        for (int p = 0; p < NP; ++p) {
            const V w2 = __ldcs(wp + ((p * n_l + j) << 5));
            f[2 * p + 1] += w2.x * g[2 * p + 1];
            f[2 * p + 2] += w2.y * g[2 * p + 2];
        }
    }
    f[0] = a.fin[i * RL];
    const uint32_t m = a.mask[i];
    if (m) {
#pragma unroll
        for (int k = 1; k < Q; ++k)
            if (m & (1u << k)) f[k] = f[opp(k)];
    }
    trt_collide<T, Q>(f, a.tp_inv, a.tm_inv, a.gx, a.gy, a.gz);
    T o[RL];
#pragma unroll
    for (int k = 0; k < Q; ++k) o[k] = f[k];
#pragma unroll
    for (int k = Q; k < RL; ++k) o[k] = (T)0;
    if constexpr (RA) {
        const V16 *__restrict__ rr = reinterpret_cast<const V16 *>(a.radd) + i * NV;
#pragma unroll
        for (int v = 0; v < NV; ++v) {
            T r[W::n];
            W::get(rr[v], r);
#pragma unroll
            for (int t = 0; t < W::n; ++t) o[v * W::n + t] += r[t];
        }
    }
    V16 *__restrict__ out = reinterpret_cast<V16 *>(a.fout) + i * NV;
#pragma unroll
    for (int v = 0; v < NV; ++v) out[v] = W::make(o + v * W::n);
}

// Pair-per-warp variant.  A block owns one SELL slice (32 nodes, one per lane)
// and has (q-1)/2 warps; warp w handles the opposite pair (k, k') = (2w+1, 2w+2)
// of every node, so the streaming of a pair, its bounce-back (which only swaps
// within the pair) and its TRT update (which only couples the pair) stay in one
// thread.  The moments are the only coupling between pairs: each warp writes its
// partial (rho, momentum) to shared memory and every thread sums the partials in
// the same order.  Warp 0 also carries the rest population.  The slice's stencil
// indices are staged in shared memory once per block.  Pairs are interleaved in
// memory (populations and weights), so each stencil column costs one 8-byte
// gather and one 256-byte coalesced weight row per warp; the loop is unrolled U
// deep to keep U such requests in flight per thread.
template <typename T, int Q, int U, bool RA = false>
__global__ void __launch_bounds__(32 * ((Q - 1) / 2), sizeof(T) == 4 ? 5 : 2) k_lbm_step_pairs(LbmArgs<T> a) {
    using V = typename Vec2<T>::type;
    constexpr int NP = (Q - 1) / 2;
    __shared__ int32_t sidx[RBF_MAX_NL][32];
    __shared__ T part[NP][4][32];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int k = 2 * w + 1, kb = k + 1;
    const int64_t s = blockIdx.x;
    const int64_t i = (s << 5) + lane;
    const bool live = i < a.n;
    const int n_l = a.n_l;
    const int64_t np = a.npad;
    {
        const int32_t *__restrict__ src = a.idx + ((s * n_l) << 5);
        for (int t = threadIdx.x; t < (n_l << 5); t += blockDim.x) sidx[t >> 5][t & 31] = __ldg(src + t);
    }
    __syncthreads();
    const V *__restrict__ wp = reinterpret_cast<const V *>(a.w) + (((s * NP + w) * (int64_t)n_l) << 5) + lane;
    const V *__restrict__ fp2 = reinterpret_cast<const V *>(a.fin + np) + (int64_t)w * np;
    T ak = 0, ab = 0, f0 = 0;
    if (live) {
        int j = 0;
        for (; j + U <= n_l; j += U) {
            int q[U];
            V w2[U], g2[U];
#pragma unroll
            for (int u = 0; u < U; ++u) q[u] = sidx[j + u][lane];
#pragma unroll
            for (int u = 0; u < U; ++u) w2[u] = __ldcs(wp + ((j + u) << 5));
#pragma unroll
            for (int u = 0; u < U; ++u) g2[u] = __ldg(fp2 + q[u]);
#pragma unroll
            for (int u = 0; u < U; ++u) {
                ak += w2[u].x * g2[u].x;
                ab += w2[u].y * g2[u].y;
            }
        }
        for (; j < n_l; ++j) {
            const V w1 = __ldcs(wp + (j << 5));
            const V g1 = __ldg(fp2 + sidx[j][lane]);
            ak += w1.x * g1.x;
            ab += w1.y * g1.y;
        }
        const uint32_t m = a.mask[i];
        if (m & (1u << k)) ak = ab;
        else if (m & (1u << kb)) ab = ak;
        if (w == 0) f0 = a.fin[i];
    }
    const T ex = (T)VSet<Q>::e(k, 0), ey = (T)VSet<Q>::e(k, 1), ez = (T)VSet<Q>::e(k, 2);
    const T dif = ak - ab;
    part[w][0][lane] = ak + ab + f0;
    part[w][1][lane] = ex * dif;
    part[w][2][lane] = ey * dif;
    part[w][3][lane] = ez * dif;
    __syncthreads();
    T drho = 0, mx = 0, my = 0, mz = 0;
#pragma unroll
    for (int t = 0; t < NP; ++t) {
        drho += part[t][0][lane];
        mx += part[t][1][lane];
        my += part[t][2][lane];
        mz += part[t][3][lane];
    }
    if (!live) return;
    const T rho = (T)1 + drho;
    const T vx = mx / rho, vy = my / rho, vz = mz / rho;
    const T vv = vx * vx + vy * vy + vz * vz;
    const T base = rho * ((T)-1.5 * vv);
    const T tp_inv = a.tp_inv, tm_inv = a.tm_inv;
    const T wk = (T)VSet<Q>::w(k);
    const T eu = ex * vx + ey * vy + ez * vz;
    const T eqp = wk * (drho + base + rho * ((T)4.5 * eu * eu));
    const T eqm = wk * rho * ((T)3 * eu);
    const T fp = (T)0.5 * (ak + ab), fm = (T)0.5 * (ak - ab);
    const T dp = (fp - eqp) * tp_inv, dm = (fm - eqm) * tm_inv;
    const T F = wk * (T)3 * rho * (ex * a.gx + ey * a.gy + ez * a.gz);
    V o;
    o.x = ak - dp - dm + F;
    o.y = ab - dp + dm - F;
    if constexpr (RA) {
        const V r = reinterpret_cast<const V *>(a.radd + np)[(int64_t)w * np + i];
        o.x += r.x;
        o.y += r.y;
    }
    reinterpret_cast<V *>(a.fout + np)[(int64_t)w * np + i] = o;
    if (w == 0) {
        const T feq0 = (T)VSet<Q>::w(0) * (drho + base);
        T f0n = f0 - (f0 - feq0) * tp_inv;
        if constexpr (RA) f0n += a.radd[i];
        a.fout[i] = f0n;
    }
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
    for (int k = 0; k < Q; ++k) a.fout[pop_at(k, i, a.npad, a.layout, Q)] = i < a.n ? f[k] : (T)0;
    if (a.layout == LBM_LAYOUT_NODES)
        for (int k = Q; k < lbm_rec_len(Q); ++k) a.fout[i * lbm_rec_len(Q) + k] = (T)0;
}

// populations <-> FP64 unshifted, caller's order (perm: sorted -> caller)
template <typename T, int Q>
__global__ void k_lbm_export(int64_t n, int64_t npad, int layout, const T *__restrict__ f,
                             const int32_t *__restrict__ perm, double *out) {
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n) return;
    int64_t o = perm[i];
#pragma unroll
    for (int k = 0; k < Q; ++k) out[k * n + o] = (double)f[pop_at(k, i, npad, layout, Q)] + VSet<Q>::w(k);
}
template <typename T, int Q>
__global__ void k_lbm_import(int64_t n, int64_t npad, int layout, T *f, const int32_t *__restrict__ perm,
                             const double *in) {
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n) return;
    int64_t o = perm[i];
#pragma unroll
    for (int k = 0; k < Q; ++k) f[pop_at(k, i, npad, layout, Q)] = (T)(in[k * n + o] - VSet<Q>::w(k));
}
template <typename T, int Q>
__global__ void k_lbm_relayout(int64_t npad, int from, const T *__restrict__ src, int to, T *dst) {
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= npad) return;
#pragma unroll
    for (int k = 0; k < Q; ++k) dst[pop_at(k, i, npad, to, Q)] = src[pop_at(k, i, npad, from, Q)];
    if (to == LBM_LAYOUT_NODES)
        for (int k = Q; k < lbm_rec_len(Q); ++k) dst[i * lbm_rec_len(Q) + k] = (T)0;
}

// macroscopic fields from the post-collision state: rho is unchanged by the
// collision, the momentum gained rho g_lb, so v_lb = sum f e / rho - g_lb.
// out (sorted order) = (vx, vy, vz, rho - 1) in lattice units, FP64.
template <typename T, int Q>
__global__ void k_lbm_macro(int64_t n, int64_t npad, int layout, const T *__restrict__ f, double gx, double gy, double gz,
                            double *out) {
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n) return;
    double d = 0, mx = 0, my = 0, mz = 0;
#pragma unroll
    for (int k = 0; k < Q; ++k) {
        double fk = (double)f[pop_at(k, i, npad, layout, Q)];
        d += fk;
        mx += VSet<Q>::e(k, 0) * fk; my += VSet<Q>::e(k, 1) * fk; mz += VSet<Q>::e(k, 2) * fk;
    }
    double rho = 1.0 + d;
    out[4 * i] = mx / rho - gx;
    out[4 * i + 1] = my / rho - gy;
    out[4 * i + 2] = mz / rho - gz;
    out[4 * i + 3] = d;
}

// FP64 row weights w[c][k-1][j] -> paired SELL [slice][pair][j][lane][2] in T
template <typename T>
__global__ void k_pack_pairs(int64_t nc, int npair, int n_l, const double *__restrict__ w, T *ws) {
    int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    int64_t npad = (nc + 31) & ~31LL;
    if (t >= npad * n_l) return;
    int64_t c = t / n_l;
    int j = (int)(t - c * n_l);
    int64_t s = c >> 5;
    int lane = (int)(c & 31);
    for (int p = 0; p < npair; ++p) {
        int64_t e = ((((s * npair + p) * (int64_t)n_l + j) << 5) + lane) * 2;
        ws[e] = c < nc ? (T)w[(c * 2 * npair + 2 * p) * n_l + j] : (T)0;
        ws[e + 1] = c < nc ? (T)w[(c * 2 * npair + 2 * p + 1) * n_l + j] : (T)0;
    }
}

cudaError_t lbm_launch_pack_f32(int64_t nc, int q, int n_l, const double *w, float *ws, cudaStream_t st) {
    int64_t tot = ((nc + 31) & ~31LL) * n_l;
    if (tot == 0) return cudaSuccess;
    k_pack_pairs<float><<<(unsigned)((tot + 255) / 256), 256, 0, st>>>(nc, (q - 1) / 2, n_l, w, ws);
    return cudaGetLastError();
}
cudaError_t lbm_launch_pack_f64(int64_t nc, int q, int n_l, const double *w, double *ws, cudaStream_t st) {
    int64_t tot = ((nc + 31) & ~31LL) * n_l;
    if (tot == 0) return cudaSuccess;
    k_pack_pairs<double><<<(unsigned)((tot + 255) / 256), 256, 0, st>>>(nc, (q - 1) / 2, n_l, w, ws);
    return cudaGetLastError();
}

template <typename T, int Q, bool RA>
static cudaError_t launch_step_q(const LbmArgs<T> &a, cudaStream_t st, int code) {
    constexpr int NP = (Q - 1) / 2;
    const unsigned slices = (unsigned)(a.npad >> 5);
    switch (code) {
    case LBM_NODE_PER_THREAD: k_lbm_step<T, Q, RA><<<(unsigned)((a.n + 255) / 256), 256, 0, st>>>(a); break;
    case LBM_NODE_PER_THREAD_128: k_lbm_step<T, Q, RA><<<(unsigned)((a.n + 127) / 128), 128, 0, st>>>(a); break;
    case LBM_PAIR_PER_WARP: k_lbm_step_pairs<T, Q, 5, RA><<<slices, 32 * NP, 0, st>>>(a); break;
    case LBM_PAIR_PER_WARP_U3: k_lbm_step_pairs<T, Q, 3, RA><<<slices, 32 * NP, 0, st>>>(a); break;
    case LBM_PAIR_PER_WARP_U6: k_lbm_step_pairs<T, Q, 6, RA><<<slices, 32 * NP, 0, st>>>(a); break;
    case LBM_PAIR_PER_WARP_U2: k_lbm_step_pairs<T, Q, 2, RA><<<slices, 32 * NP, 0, st>>>(a); break;
    // register caps: FP32 64 / 48 (4 / 5 blocks per SM); FP64 128 / 80 (2 / 3 blocks)
    case LBM_RECORD_PER_THREAD:
        k_lbm_step_records<T, Q, sizeof(T) == 4 ? 4 : 2, RA><<<(unsigned)((a.n + 255) / 256), 256, 0, st>>>(a);
        break;
    case LBM_RECORD_PER_THREAD_OCC:
        k_lbm_step_records<T, Q, sizeof(T) == 4 ? 5 : 3, RA><<<(unsigned)((a.n + 255) / 256), 256, 0, st>>>(a);
        break;
    case LBM_RECORD_PER_THREAD_128:
        k_lbm_step_records<T, Q, sizeof(T) == 4 ? 4 : 2, RA><<<(unsigned)((a.n + 127) / 128), 128, 0, st>>>(a);
        break;
    case LBM_RECORD_PER_THREAD_64:
        k_lbm_step_records<T, Q, sizeof(T) == 4 ? 4 : 2, RA><<<(unsigned)((a.n + 63) / 64), 64, 0, st>>>(a);
        break;
    case LBM_RECORD_PER_THREAD_PDL: {
        cudaLaunchConfig_t cfg = {};
        cfg.gridDim = dim3((unsigned)((a.n + 255) / 256));
        cfg.blockDim = dim3(256);
        cfg.stream = st;
        cudaLaunchAttribute at[1];
        at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
        at[0].val.programmaticStreamSerializationAllowed = 1;
        cfg.attrs = at;
        cfg.numAttrs = 1;
        const cudaError_t e = cudaLaunchKernelEx(&cfg, k_lbm_step_records<T, Q, sizeof(T) == 4 ? 4 : 2, RA, true>, a);
        if (e != cudaSuccess) return e;
        break;
    }
    default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

template <typename T>
cudaError_t lbm_launch_step(const LbmArgs<T> &a, int q, cudaStream_t st, int code) {
    if (code < 0 || code >= LBM_N_SCHEDULES || lbm_layout_of(code) != a.layout) return cudaErrorInvalidValue;
    if (a.radd) {  // the residual addend: refined FP32 only
        if constexpr (sizeof(T) == 4) {
            if (q == 19) return launch_step_q<T, 19, true>(a, st, code);
            if (q == 15) return launch_step_q<T, 15, true>(a, st, code);
        }
        return cudaErrorInvalidValue;
    }
    if (q == 19) return launch_step_q<T, 19, false>(a, st, code);
    if (q == 15) return launch_step_q<T, 15, false>(a, st, code);
    return cudaErrorInvalidValue;
}

// ---- refined FP32: f = base (FP64) + delta (FP32) -------------------------------
__global__ void k_refine_fold(int64_t tot, double *__restrict__ base, const float *__restrict__ delta) {
    int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (e < tot) base[e] += (double)delta[e];
}
__global__ void k_refine_residual(int64_t tot, const double *__restrict__ fnew, const double *__restrict__ base,
                                  float *__restrict__ r, float *__restrict__ delta) {
    int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (e >= tot) return;
    const float v = (float)(fnew[e] - base[e]);
    r[e] = v;
    delta[e] = v;
}
__global__ void k_refine_combine(int64_t tot, const double *__restrict__ base, const float *__restrict__ delta,
                                 double *__restrict__ out) {
    int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (e < tot) out[e] = base[e] + (double)delta[e];
}
cudaError_t lbm_launch_refine_fold(int64_t tot, double *base, const float *delta, cudaStream_t st) {
    if (tot == 0) return cudaSuccess;
    k_refine_fold<<<(unsigned)((tot + 255) / 256), 256, 0, st>>>(tot, base, delta);
    return cudaGetLastError();
}
cudaError_t lbm_launch_refine_residual(int64_t tot, const double *fnew, const double *base, float *r, float *delta,
                                       cudaStream_t st) {
    if (tot == 0) return cudaSuccess;
    k_refine_residual<<<(unsigned)((tot + 255) / 256), 256, 0, st>>>(tot, fnew, base, r, delta);
    return cudaGetLastError();
}
cudaError_t lbm_launch_refine_combine(int64_t tot, const double *base, const float *delta, double *out,
                                      cudaStream_t st) {
    if (tot == 0) return cudaSuccess;
    k_refine_combine<<<(unsigned)((tot + 255) / 256), 256, 0, st>>>(tot, base, delta, out);
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

cudaError_t lbm_launch_masks_solid(int64_t n, int q, const uint8_t *type, const double *xyz, const double c[3], double r,
                                  double dx, uint32_t *mask, cudaStream_t st) {
    unsigned g = (unsigned)((n + 255) / 256);
    if (q == 19) k_lbm_masks_solid<19><<<g, 256, 0, st>>>(n, type, xyz, c[0], c[1], c[2], r, dx, mask);
    else if (q == 15) k_lbm_masks_solid<15><<<g, 256, 0, st>>>(n, type, xyz, c[0], c[1], c[2], r, dx, mask);
    else return cudaErrorInvalidValue;
    return cudaGetLastError();
}

__global__ void k_scatter_u32(int64_t n, const int32_t *__restrict__ perm, const uint32_t *__restrict__ in,
                              uint32_t *out) {
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i < n) out[perm[i]] = in[i];
}
cudaError_t launch_scatter_u32(int64_t n, const int32_t *perm, const uint32_t *in, uint32_t *out, cudaStream_t st) {
    if (n == 0) return cudaSuccess;
    k_scatter_u32<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(n, perm, in, out);
    return cudaGetLastError();
}

template <typename T>
cudaError_t lbm_launch_export(int64_t n, int64_t npad, int layout, int q, const T *f, const int32_t *perm, double *out,
                              cudaStream_t st) {
    unsigned g = (unsigned)((n + 255) / 256);
    if (q == 19) k_lbm_export<T, 19><<<g, 256, 0, st>>>(n, npad, layout, f, perm, out);
    else k_lbm_export<T, 15><<<g, 256, 0, st>>>(n, npad, layout, f, perm, out);
    return cudaGetLastError();
}
template <typename T>
cudaError_t lbm_launch_import(int64_t n, int64_t npad, int layout, int q, T *f, const int32_t *perm, const double *in,
                              cudaStream_t st) {
    unsigned g = (unsigned)((n + 255) / 256);
    if (q == 19) k_lbm_import<T, 19><<<g, 256, 0, st>>>(n, npad, layout, f, perm, in);
    else k_lbm_import<T, 15><<<g, 256, 0, st>>>(n, npad, layout, f, perm, in);
    return cudaGetLastError();
}
template <typename T>
cudaError_t lbm_launch_relayout(int64_t npad, int q, int from, const T *src, int to, T *dst, cudaStream_t st) {
    unsigned g = (unsigned)((npad + 255) / 256);
    if (q == 19) k_lbm_relayout<T, 19><<<g, 256, 0, st>>>(npad, from, src, to, dst);
    else if (q == 15) k_lbm_relayout<T, 15><<<g, 256, 0, st>>>(npad, from, src, to, dst);
    else return cudaErrorInvalidValue;
    return cudaGetLastError();
}
template <typename T>
cudaError_t lbm_launch_macro(int64_t n, int64_t npad, int layout, int q, const T *f, const double g[3], double *out,
                             cudaStream_t st) {
    unsigned gr = (unsigned)((n + 255) / 256);
    if (q == 19) k_lbm_macro<T, 19><<<gr, 256, 0, st>>>(n, npad, layout, f, g[0], g[1], g[2], out);
    else k_lbm_macro<T, 15><<<gr, 256, 0, st>>>(n, npad, layout, f, g[0], g[1], g[2], out);
    return cudaGetLastError();
}

#define RBF_LBM_INST(T)                                                                                         \
    template cudaError_t lbm_launch_step<T>(const LbmArgs<T> &, int, cudaStream_t, int);                        \
    template cudaError_t lbm_launch_init<T>(const LbmArgs<T> &, int, cudaStream_t);                             \
    template cudaError_t lbm_launch_export<T>(int64_t, int64_t, int, int, const T *, const int32_t *, double *, \
                                              cudaStream_t);                                                    \
    template cudaError_t lbm_launch_import<T>(int64_t, int64_t, int, int, T *, const int32_t *, const double *, \
                                              cudaStream_t);                                                    \
    template cudaError_t lbm_launch_relayout<T>(int64_t, int, int, const T *, int, T *, cudaStream_t);          \
    template cudaError_t lbm_launch_macro<T>(int64_t, int64_t, int, int, const T *, const double *, double *,   \
                                             cudaStream_t);
RBF_LBM_INST(float)
RBF_LBM_INST(double)

}  // namespace rbf
