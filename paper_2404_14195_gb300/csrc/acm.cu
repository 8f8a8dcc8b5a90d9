// acm.cu — explicit artificial-compressibility Navier-Stokes step (MNS section,
// Eqs. MNS_intermediate, MNS_pressure, MNS_velocity, MNS_C; MNS algorithm of the
// appendix), on SELL-C slices of 32 Morton-ordered nodes with one or G lanes per
// node.
//
// Per step:   predict  v' = v + dt (nu lap v - (v . grad) v + g)   fluid; v' = 0 walls
//             n_p x {  pressure  p -= dt C^2 rho div v            fluid
//                      wall p from n . grad p = 0 on the Neumann stencil
//                      correct   v = v' - dt/rho grad p           fluid; 0 walls
//                                C = beta max(max |v|, v_ref)  }
// Stencil gathers read u, v, w, p at the neighbour indices; weights and stencil
// indices stream from HBM as SELL slices [slice][operator][j][lane] (coalesced
// 128-byte rows) with evict-first loads, which leave L2 to the gathered fields.
// max |v| is reduced per block with warp shuffles and merged with one 64-bit
// atomicMax per block into one of two ping-pong slots (non-negative IEEE values
// order like their bit patterns), which the next pressure sweep reads.
//
// Compensated FP32 (CP = true): u, v, w, p and v' are carried as float pairs
// hi + lo.  Gathers and all stencil arithmetic read the hi words only; every
// update of a field adds its increment to the pair with comp_add, so the slow
// late-time changes of a near-steady field, far below one float ulp of the
// field, are not rounded away (the explicit update otherwise stalls short of
// the steady state).  Wall values are exact zeros in both words.
#include "acm.cuh"

namespace rbf {

// Thread -> (node, stencil lanes): each warp is one unit of 32 / G nodes of a
// slice; unit `sub` of slice s holds the slice's nodes sub (32 / G) .. + 32 / G - 1,
// node nl of the unit on lanes G (nl mod 32 / G) .. + G - 1, and lane g of a node's
// group takes the stencil columns j = g, g + G, ...; the partial sums meet in
// group_sum and the group's first lane (g = 0) writes.  G = 1 is one node per
// thread.  No lane returns before the shuffles.
template <int G>
struct NodeMap {
    int64_t t, s, i;
    int nl, g;
    __device__ __forceinline__ NodeMap() {
        t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
        const int64_t unit = t >> 5;
        const int lane = (int)(t & 31);
        s = unit / G;
        nl = (int)(unit % G) * (32 / G) + lane / G;
        g = lane % G;
        i = (s << 5) + nl;
    }
};

template <typename T, bool CP, int G>
__global__ void __launch_bounds__(256) k_acm_predict(AcmArgs<T> a) {
    const NodeMap<G> m;
    const int64_t i = m.i;
    const bool valid = i < a.n;
    const bool fluid = valid && !a.type[i];
    T gu[4] = {0, 0, 0, 0}, gv[4] = {0, 0, 0, 0}, gw[4] = {0, 0, 0, 0};
    if (fluid) {
        const int n_l = a.n_l;
        const int32_t *__restrict__ ip = a.idx + ((m.s * n_l) << 5) + m.nl;
        const T *__restrict__ wp = a.w + ((m.s * 4 * (int64_t)n_l) << 5) + m.nl;
#pragma unroll 5
        for (int j = m.g; j < n_l; j += G) {
            int q = __ldcs(ip + (j << 5));
            T wx = __ldcs(wp + (j << 5)), wy = __ldcs(wp + ((n_l + j) << 5));
            T wz = __ldcs(wp + ((2 * n_l + j) << 5)), wl = __ldcs(wp + ((3 * n_l + j) << 5));
            T uq = a.u[q], vq = a.v[q], wq = a.w_[q];
            gu[0] += wx * uq; gu[1] += wy * uq; gu[2] += wz * uq; gu[3] += wl * uq;
            gv[0] += wx * vq; gv[1] += wy * vq; gv[2] += wz * vq; gv[3] += wl * vq;
            gw[0] += wx * wq; gw[1] += wy * wq; gw[2] += wz * wq; gw[3] += wl * wq;
        }
    }
    if constexpr (G > 1) {
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            gu[k] = group_sum<T, G>(gu[k]);
            gv[k] = group_sum<T, G>(gv[k]);
            gw[k] = group_sum<T, G>(gw[k]);
        }
    }
    if (!valid || m.g != 0) return;
    if (!fluid) {
        a.us[i] = (T)0; a.vs[i] = (T)0; a.ws[i] = (T)0;
        if constexpr (CP) { a.usl[i] = (T)0; a.vsl[i] = (T)0; a.wsl[i] = (T)0; }
        return;
    }
    T ui = a.u[i], vi = a.v[i], wi = a.w_[i];
    T adv_u = ui * gu[0] + vi * gu[1] + wi * gu[2];
    T adv_v = ui * gv[0] + vi * gv[1] + wi * gv[2];
    T adv_w = ui * gw[0] + vi * gw[1] + wi * gw[2];
    if constexpr (CP) {
        T h = ui, l = a.ul[i];
        comp_add(h, l, a.dt * (a.nu * gu[3] - adv_u + a.gx));
        a.us[i] = h; a.usl[i] = l;
        h = vi; l = a.vl[i];
        comp_add(h, l, a.dt * (a.nu * gv[3] - adv_v + a.gy));
        a.vs[i] = h; a.vsl[i] = l;
        h = wi; l = a.wl[i];
        comp_add(h, l, a.dt * (a.nu * gw[3] - adv_w + a.gz));
        a.ws[i] = h; a.wsl[i] = l;
    } else {
        a.us[i] = ui + a.dt * (a.nu * gu[3] - adv_u + a.gx);
        a.vs[i] = vi + a.dt * (a.nu * gv[3] - adv_v + a.gy);
        a.ws[i] = wi + a.dt * (a.nu * gw[3] - adv_w + a.gz);
    }
}

// speed of sound of Eq. MNS_C from the max |v| stored (as double bits) in a slot
__device__ __forceinline__ double acm_C(const unsigned long long *slot, double beta, double vref) {
    double vmax = __longlong_as_double((long long)*slot);
    return beta * (vmax > vref ? vmax : vref);
}

template <typename T, bool CP, int G>
__global__ void __launch_bounds__(256) k_acm_pressure(AcmArgs<T> a, const T *__restrict__ u, const T *__restrict__ v,
                                                     const T *__restrict__ w, int read_slot, int zero_slot) {
    const NodeMap<G> m;
    const int64_t i = m.i;
    if (m.t == 0) a.vmax[zero_slot] = 0ULL;
    const bool fluid = i < a.n && !a.type[i];
    T div = 0;
    if (fluid) {
        const int n_l = a.n_l;
        const int32_t *__restrict__ ip = a.idx + ((m.s * n_l) << 5) + m.nl;
        const T *__restrict__ wp = a.w + ((m.s * 4 * (int64_t)n_l) << 5) + m.nl;
#pragma unroll 5
        for (int j = m.g; j < n_l; j += G) {
            int q = __ldcs(ip + (j << 5));
            T wx = __ldcs(wp + (j << 5)), wy = __ldcs(wp + ((n_l + j) << 5)), wz = __ldcs(wp + ((2 * n_l + j) << 5));
            div += wx * u[q] + wy * v[q] + wz * w[q];
        }
    }
    if constexpr (G > 1) div = group_sum<T, G>(div);
    if (!fluid || m.g != 0) return;
    const double C = acm_C(a.vmax + read_slot, a.beta, a.vref);
    const T Ct = (T)C;
    if constexpr (CP) {
        T h = a.p[i], l = a.pl[i];
        comp_add(h, l, -(a.dt * Ct * Ct * a.rho * div));
        a.p[i] = h; a.pl[i] = l;
    } else {
        a.p[i] = a.p[i] - a.dt * Ct * Ct * a.rho * div;
    }
}

// wall pressure from the Neumann condition, on the wall nodes' own stencils
// {b, nearest fluid nodes}: p_b = -sum_{j>=1} w^n_j p_j / w^n_0
template <typename T, bool CP, int G>
__global__ void __launch_bounds__(256) k_acm_wall_pressure(AcmArgs<T> a) {
    const NodeMap<G> m;
    const int64_t b = m.i;
    const bool valid = b < a.nb;
    const int n_l = a.n_l;
    const int32_t *__restrict__ ip = a.idxb + ((m.s * n_l) << 5) + m.nl;
    const T *__restrict__ wp = a.wn + ((m.s * n_l) << 5) + m.nl;
    T acc = 0;
    if (valid) {
#pragma unroll 4
        for (int j = 1 + m.g; j < n_l; j += G) acc += __ldcs(wp + (j << 5)) * a.p[__ldcs(ip + (j << 5))];
    }
    if constexpr (G > 1) acc = group_sum<T, G>(acc);
    if (!valid || m.g != 0) return;
    const int32_t wb = a.wall[b];
    a.p[wb] = -acc / __ldcs(wp);
    if constexpr (CP) a.pl[wb] = (T)0;
}

template <typename T, bool CP, int G>
__global__ void __launch_bounds__(256) k_acm_correct(AcmArgs<T> a, int write_slot) {
    __shared__ double red[8];
    const NodeMap<G> m;
    const int64_t i = m.i;
    const bool valid = i < a.n;
    const bool fluid = valid && !a.type[i];
    T gx = 0, gy = 0, gz = 0;
    if (fluid) {
        const int n_l = a.n_l;
        const int32_t *__restrict__ ip = a.idx + ((m.s * n_l) << 5) + m.nl;
        const T *__restrict__ wp = a.w + ((m.s * 4 * (int64_t)n_l) << 5) + m.nl;
#pragma unroll 5
        for (int j = m.g; j < n_l; j += G) {
            T pq = a.p[__ldcs(ip + (j << 5))];
            gx += __ldcs(wp + (j << 5)) * pq;
            gy += __ldcs(wp + ((n_l + j) << 5)) * pq;
            gz += __ldcs(wp + ((2 * n_l + j) << 5)) * pq;
        }
    }
    if constexpr (G > 1) {
        gx = group_sum<T, G>(gx);
        gy = group_sum<T, G>(gy);
        gz = group_sum<T, G>(gz);
    }
    double speed = 0.0;
    if (valid && m.g == 0) {
        if (!fluid) {
            a.u[i] = (T)0; a.v[i] = (T)0; a.w_[i] = (T)0;
            if constexpr (CP) { a.ul[i] = (T)0; a.vl[i] = (T)0; a.wl[i] = (T)0; }
        } else {
            const T f = a.dt / a.rho;
            T un, vn, wn;
            if constexpr (CP) {
                T l = a.usl[i];
                un = a.us[i]; comp_add(un, l, -(f * gx)); a.ul[i] = l;
                l = a.vsl[i];
                vn = a.vs[i]; comp_add(vn, l, -(f * gy)); a.vl[i] = l;
                l = a.wsl[i];
                wn = a.ws[i]; comp_add(wn, l, -(f * gz)); a.wl[i] = l;
            } else {
                un = a.us[i] - f * gx; vn = a.vs[i] - f * gy; wn = a.ws[i] - f * gz;
            }
            a.u[i] = un; a.v[i] = vn; a.w_[i] = wn;
            speed = (double)sqrt(un * un + vn * vn + wn * wn);
        }
    }
    for (int off = 16; off > 0; off >>= 1) speed = fmax(speed, __shfl_xor_sync(0xffffffffu, speed, off));
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = speed;
    __syncthreads();
    if (threadIdx.x < 32) {
        double v = threadIdx.x < (blockDim.x >> 5) ? red[threadIdx.x] : 0.0;
        for (int off = 16; off > 0; off >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, off));
        if (threadIdx.x == 0 && v > 0.0) atomicMax(a.vmax + write_slot, (unsigned long long)__double_as_longlong(v));
    }
}

// max |v| of the current field into a slot (initial C)
template <typename T>
__global__ void k_acm_vmax(AcmArgs<T> a, int slot) {
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    double sp = 0.0;
    if (i < a.n) sp = (double)sqrt(a.u[i] * a.u[i] + a.v[i] * a.v[i] + a.w_[i] * a.w_[i]);
    for (int off = 16; off > 0; off >>= 1) sp = fmax(sp, __shfl_xor_sync(0xffffffffu, sp, off));
    if ((threadIdx.x & 31) == 0 && sp > 0.0) atomicMax(a.vmax + slot, (unsigned long long)__double_as_longlong(sp));
}

// Iteration g of the run (counted over all steps) writes max |v| into slot g % 2;
// the pressure sweep of iteration g reads slot (g + 1) % 2 (the previous
// iteration's) and clears slot g % 2 for its own correction sweep.  The grids
// cover every slice with G warps per slice.
template <typename T, bool CP, int G>
cudaError_t acm_launch_step_g(const AcmArgs<T> &a, int n_p, int parity, cudaStream_t st, int64_t *launches,
                              LaunchRecorder *rec, int block) {
    const int64_t threads = ((a.n + 31) >> 5) * 32 * G, threads_b = ((a.nb + 31) >> 5) * 32 * G;
    const unsigned gb = (unsigned)((threads + block - 1) / block);
    const unsigned gw = (unsigned)((threads_b + 255) / 256);
    if (rec) rec->begin(st, 0);
    k_acm_predict<T, CP, G><<<gb, block, 0, st>>>(a);
    if (rec) rec->end(st);
    ++*launches;
    for (int it = 0; it < n_p; ++it) {
        const T *u = it == 0 ? a.us : a.u;
        const T *v = it == 0 ? a.vs : a.v;
        const T *w = it == 0 ? a.ws : a.w_;
        const int g = (parity + it) & 1;
        if (rec) rec->begin(st, 1);
        k_acm_pressure<T, CP, G><<<gb, block, 0, st>>>(a, u, v, w, g ^ 1, g);
        if (rec) rec->end(st);
        ++*launches;
        if (a.nb > 0) {
            if (rec) rec->begin(st, 2);
            k_acm_wall_pressure<T, CP, G><<<gw, 256, 0, st>>>(a);
            if (rec) rec->end(st);
            ++*launches;
        }
        if (rec) rec->begin(st, 3);
        k_acm_correct<T, CP, G><<<gb, block, 0, st>>>(a, g);
        if (rec) rec->end(st);
        ++*launches;
    }
    return cudaGetLastError();
}

template <typename T, bool CP>
cudaError_t acm_launch_step_cp(const AcmArgs<T> &a, int n_p, int parity, cudaStream_t st, int64_t *launches,
                               LaunchRecorder *rec, int block, int group) {
    switch (group) {
    case 1: return acm_launch_step_g<T, CP, 1>(a, n_p, parity, st, launches, rec, block);
    case 2: return acm_launch_step_g<T, CP, 2>(a, n_p, parity, st, launches, rec, block);
    case 4: return acm_launch_step_g<T, CP, 4>(a, n_p, parity, st, launches, rec, block);
    default: return cudaErrorInvalidValue;
    }
}

// the compensated kernels run when the low words are present; code = threads per
// block (64, 128, 256) + 1000 x lanes per node (0 or 1: one, 2, 4)
template <typename T>
cudaError_t acm_launch_step(const AcmArgs<T> &a, int n_p, int parity, cudaStream_t st, int64_t *launches,
                            LaunchRecorder *rec, int code) {
    if (!acm_code_ok(code)) return cudaErrorInvalidValue;
    const int block = code % 1000, group = code / 1000 ? code / 1000 : 1;
    const bool cp = a.ul && a.vl && a.wl && a.pl && a.usl && a.vsl && a.wsl;
    if (!cp && (a.ul || a.vl || a.wl || a.pl || a.usl || a.vsl || a.wsl)) return cudaErrorInvalidValue;
    return cp ? acm_launch_step_cp<T, true>(a, n_p, parity, st, launches, rec, block, group)
              : acm_launch_step_cp<T, false>(a, n_p, parity, st, launches, rec, block, group);
}

template <typename T>
cudaError_t acm_launch_vmax(const AcmArgs<T> &a, int slot, cudaStream_t st) {
    cudaError_t e = cudaMemsetAsync(a.vmax + slot, 0, sizeof(unsigned long long), st);
    if (e != cudaSuccess) return e;
    k_acm_vmax<T><<<(unsigned)((a.n + 255) / 256), 256, 0, st>>>(a, slot);
    return cudaGetLastError();
}

template <typename T>
cudaError_t acm_launch_predict_only(const AcmArgs<T> &a, cudaStream_t st) {
    if (a.ul) {
        k_acm_predict<T, true, 1><<<(unsigned)((a.n + 255) / 256), 256, 0, st>>>(a);
        return cudaGetLastError();
    }
    k_acm_predict<T, false, 1><<<(unsigned)((a.n + 255) / 256), 256, 0, st>>>(a);
    return cudaGetLastError();
}

template cudaError_t acm_launch_step<float>(const AcmArgs<float> &, int, int, cudaStream_t, int64_t *, LaunchRecorder *, int);
template cudaError_t acm_launch_step<double>(const AcmArgs<double> &, int, int, cudaStream_t, int64_t *, LaunchRecorder *, int);
template cudaError_t acm_launch_vmax<float>(const AcmArgs<float> &, int, cudaStream_t);
template cudaError_t acm_launch_vmax<double>(const AcmArgs<double> &, int, cudaStream_t);
template cudaError_t acm_launch_predict_only<float>(const AcmArgs<float> &, cudaStream_t);
template cudaError_t acm_launch_predict_only<double>(const AcmArgs<double> &, cudaStream_t);

}  // namespace rbf
