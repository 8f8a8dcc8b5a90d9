// acm_persist.cu — the ACM steady driver as one persistent kernel over any number
// of cells (MNS algorithm of the appendix, repeated until each cell's stopping
// criterion holds).
//
// One cooperative launch; every block loops over steps and, inside a step, over
// the phases  predict -> n_p x (pressure, wall pressure, correction),  each phase
// a grid-stride loop over 32-node SELL slices of all cells still running (warp =
// slice, lane = node), separated by a software grid barrier.  Every check_every
// steps the blocks reduce, per cell, |v - v_prev|^2 and |v|^2 in FP64, block 0
// turns them into residuals and sets the cell's done flag; converged cells drop
// out of the loop while the others continue.  The arithmetic of each phase is
// that of the multi-launch kernels in acm.cu (same operations, same order).
//
// The grid barrier is a counter plus a generation word; waiting blocks give up
// after a wall-clock limit (PersistCtl::wait_ns, 2 s by default), raise an error
// flag and leave the loop, so a launch whose blocks are not co-resident ends with
// RBF_ETIMEOUT instead of hanging.  Every wait also ends as soon as another block
// has raised the flag.  The cooperative launch itself guarantees co-residency.
//
// CP = true is the compensated FP32 state of acm.cu (hi + lo pairs, comp_add
// updates, gathers of the hi words); its residual differences include the low
// words.
#include <cstring>

#include "acm_persist.cuh"
#include "acm.cuh"
#include "tc.cuh"

namespace rbf {

namespace {

// returns false (and raises *err) if the other blocks did not arrive within
// wait_ns nanoseconds, or if another block has raised *err
__device__ bool grid_barrier(unsigned *count, unsigned *gen, unsigned nblocks, int32_t *err, uint64_t wait_ns) {
    __shared__ int ok;
    __syncthreads();
    if (threadIdx.x == 0) {
        ok = 1;
        volatile unsigned *vgen = gen;
        const unsigned g = *vgen;
        __threadfence();
        if (atomicAdd(count, 1u) == nblocks - 1) {
            atomicExch(count, 0u);
            __threadfence();
            atomicAdd(gen, 1u);
        } else {
            const uint64_t t0 = tc::globaltimer_ns();
            while (*vgen == g) {
                if (*(volatile int32_t *)err) { ok = 0; break; }
                if (tc::globaltimer_ns() - t0 > wait_ns) {
                    atomicExch(err, 2);
                    ok = 0;
                    break;
                }
            }
        }
        __threadfence();
    }
    __syncthreads();
    return ok != 0;
}

__device__ __forceinline__ double slot_C(const unsigned long long *slot, double beta, double vref) {
    const double vmax = __longlong_as_double((long long)*(volatile unsigned long long *)slot);
    return beta * (vmax > vref ? vmax : vref);
}

// The phases work on units of 32 / G nodes of one slice: unit `sub` of slice ls
// holds nodes sub (32 / G) .. (sub + 1) (32 / G) - 1, node nl of the unit on lanes
// G (nl mod 32/G) .. + G - 1, each lane taking the stencil columns j = g, g + G, ...
// (g = lane mod G); the group's partial sums are combined with shuffles and the
// first lane of the group (the lead) writes.  G = 1 is one node per lane.  Every
// lane reaches the shuffles (no early return before them).
template <typename T, bool CP, int G>
__device__ void phase_predict(const CellDesc<T> &c, int64_t ls, int sub, int lane, bool snapshot) {
    const int nl = sub * (32 / G) + lane / G, g = lane % G;
    const int64_t i = (ls << 5) + nl;
    const bool valid = i < c.n;
    const bool fluid = valid && !c.type[i];
    T ui = 0, vi = 0, wi = 0;
    if (valid) { ui = c.u[i]; vi = c.v[i]; wi = c.w_[i]; }
    T gu[4] = {0, 0, 0, 0}, gv[4] = {0, 0, 0, 0}, gw[4] = {0, 0, 0, 0};
    if (fluid) {
        const int n_l = c.n_l;
        const int32_t *__restrict__ ip = c.idx + ((ls * n_l) << 5) + nl;
        const T *__restrict__ wp = c.w + ((ls * 4 * (int64_t)n_l) << 5) + nl;
#pragma unroll 5
        for (int j = g; j < n_l; j += G) {
            const int q = __ldcs(ip + (j << 5));
            const T wx = __ldcs(wp + (j << 5)), wy = __ldcs(wp + ((n_l + j) << 5));
            const T wz = __ldcs(wp + ((2 * n_l + j) << 5)), wl = __ldcs(wp + ((3 * n_l + j) << 5));
            const T uq = c.u[q], vq = c.v[q], wq = c.w_[q];
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
    if (!valid || g != 0) return;
    if (snapshot) {
        c.uo[i] = ui; c.vo[i] = vi; c.wo[i] = wi;
        if constexpr (CP) { c.uol[i] = c.ul[i]; c.vol[i] = c.vl[i]; c.wol[i] = c.wl[i]; }
    }
    if (!fluid) {
        c.us[i] = (T)0; c.vs[i] = (T)0; c.ws[i] = (T)0;
        if constexpr (CP) { c.usl[i] = (T)0; c.vsl[i] = (T)0; c.wsl[i] = (T)0; }
        return;
    }
    const T adv_u = ui * gu[0] + vi * gu[1] + wi * gu[2];
    const T adv_v = ui * gv[0] + vi * gv[1] + wi * gv[2];
    const T adv_w = ui * gw[0] + vi * gw[1] + wi * gw[2];
    if constexpr (CP) {
        T h = ui, l = c.ul[i];
        comp_add(h, l, c.dt * (c.nu * gu[3] - adv_u + c.gx));
        c.us[i] = h; c.usl[i] = l;
        h = vi; l = c.vl[i];
        comp_add(h, l, c.dt * (c.nu * gv[3] - adv_v + c.gy));
        c.vs[i] = h; c.vsl[i] = l;
        h = wi; l = c.wl[i];
        comp_add(h, l, c.dt * (c.nu * gw[3] - adv_w + c.gz));
        c.ws[i] = h; c.wsl[i] = l;
    } else {
        c.us[i] = ui + c.dt * (c.nu * gu[3] - adv_u + c.gx);
        c.vs[i] = vi + c.dt * (c.nu * gv[3] - adv_v + c.gy);
        c.ws[i] = wi + c.dt * (c.nu * gw[3] - adv_w + c.gz);
    }
}

template <typename T, bool CP, int G>
__device__ void phase_pressure(const CellDesc<T> &c, int64_t ls, int sub, int lane, bool first, int gslot) {
    const int nl = sub * (32 / G) + lane / G, g = lane % G;
    const int64_t i = (ls << 5) + nl;
    const bool fluid = i < c.n && !c.type[i];
    const T *u = first ? c.us : c.u;
    const T *v = first ? c.vs : c.v;
    const T *w = first ? c.ws : c.w_;
    T div = 0;
    if (fluid) {
        const int n_l = c.n_l;
        const int32_t *__restrict__ ip = c.idx + ((ls * n_l) << 5) + nl;
        const T *__restrict__ wp = c.w + ((ls * 4 * (int64_t)n_l) << 5) + nl;
#pragma unroll 5
        for (int j = g; j < n_l; j += G) {
            const int q = __ldcs(ip + (j << 5));
            div += __ldcs(wp + (j << 5)) * u[q] + __ldcs(wp + ((n_l + j) << 5)) * v[q] +
                   __ldcs(wp + ((2 * n_l + j) << 5)) * w[q];
        }
    }
    if constexpr (G > 1) div = group_sum<T, G>(div);
    if (!fluid || g != 0) return;
    const double C = slot_C(c.vmax + (gslot ^ 1), c.beta, c.vref);
    const T Ct = (T)C;
    if constexpr (CP) {
        T h = c.p[i], l = c.pl[i];
        comp_add(h, l, -(c.dt * Ct * Ct * c.rho * div));
        c.p[i] = h; c.pl[i] = l;
    } else {
        c.p[i] = c.p[i] - c.dt * Ct * Ct * c.rho * div;
    }
}

template <typename T, bool CP, int G>
__device__ void phase_wall(const CellDesc<T> &c, int64_t ls, int sub, int lane) {
    const int nl = sub * (32 / G) + lane / G, g = lane % G;
    const int64_t b = (ls << 5) + nl;
    const bool valid = b < c.nb;
    const int n_l = c.n_l;
    T acc = 0;
    if (valid) {
        const int32_t *__restrict__ ip = c.idxb + ((ls * n_l) << 5) + nl;
        const T *__restrict__ wp = c.wn + ((ls * n_l) << 5) + nl;
#pragma unroll 4
        for (int j = 1 + g; j < n_l; j += G) acc += __ldcs(wp + (j << 5)) * c.p[__ldcs(ip + (j << 5))];
    }
    if constexpr (G > 1) acc = group_sum<T, G>(acc);
    if (!valid || g != 0) return;
    const int32_t wb = c.wall[b];
    c.p[wb] = -acc / __ldcs(c.wn + ((ls * n_l) << 5) + nl);
    if constexpr (CP) c.pl[wb] = (T)0;
}

// returns |v| of the node (lead lane of a fluid node), 0 otherwise
template <typename T, bool CP, int G>
__device__ double phase_correct(const CellDesc<T> &c, int64_t ls, int sub, int lane) {
    const int nl = sub * (32 / G) + lane / G, g = lane % G;
    const int64_t i = (ls << 5) + nl;
    const bool valid = i < c.n;
    const bool fluid = valid && !c.type[i];
    T gx = 0, gy = 0, gz = 0;
    if (fluid) {
        const int n_l = c.n_l;
        const int32_t *__restrict__ ip = c.idx + ((ls * n_l) << 5) + nl;
        const T *__restrict__ wp = c.w + ((ls * 4 * (int64_t)n_l) << 5) + nl;
#pragma unroll 5
        for (int j = g; j < n_l; j += G) {
            const T pq = c.p[__ldcs(ip + (j << 5))];
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
    if (!valid || g != 0) return 0.0;
    if (!fluid) {
        c.u[i] = (T)0; c.v[i] = (T)0; c.w_[i] = (T)0;
        if constexpr (CP) { c.ul[i] = (T)0; c.vl[i] = (T)0; c.wl[i] = (T)0; }
        return 0.0;
    }
    const T f = c.dt / c.rho;
    T un, vn, wn;
    if constexpr (CP) {
        T l = c.usl[i];
        un = c.us[i]; comp_add(un, l, -(f * gx)); c.ul[i] = l;
        l = c.vsl[i];
        vn = c.vs[i]; comp_add(vn, l, -(f * gy)); c.vl[i] = l;
        l = c.wsl[i];
        wn = c.ws[i]; comp_add(wn, l, -(f * gz)); c.wl[i] = l;
    } else {
        un = c.us[i] - f * gx; vn = c.vs[i] - f * gy; wn = c.ws[i] - f * gz;
    }
    c.u[i] = un; c.v[i] = vn; c.w_[i] = wn;
    return (double)sqrt(un * un + vn * vn + wn * wn);
}

// every thread of every CTA of the cluster arrives (release) and waits (acquire):
// the hardware barrier of a thread-block cluster, no spinning on memory
__device__ __forceinline__ void cluster_barrier() {
    asm volatile("barrier.cluster.arrive.release.aligned;\n\tbarrier.cluster.wait.acquire.aligned;" ::: "memory");
}

// CL = false: a cooperative grid synchronised by grid_barrier (any number of
// co-resident blocks); CL = true: one thread-block cluster (8 or 16 CTAs)
// synchronised by the cluster's hardware barrier, for small cells where the
// software barrier's latency dominates a step.  Every block of a cluster takes the
// same branches at every barrier (the done flags change only before a barrier and
// the cluster barrier cannot time out), so none is left waiting.
template <typename T, bool CP, bool CL, int G>
__global__ void __launch_bounds__(256) k_acm_persistent(const CellDesc<T> *__restrict__ cells, PersistCtl ctl) {
    __shared__ double racc[PERSIST_MAX_CELLS][2];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int wpb = blockDim.x >> 5;
    const int64_t wstride = (int64_t)gridDim.x * wpb;
    const int64_t w0 = (int64_t)blockIdx.x * wpb + warp;
    const unsigned nblocks = gridDim.x;
    auto grid_barrier = [&](unsigned *count, unsigned *gen, unsigned nb, int32_t *err) -> bool {
        if constexpr (CL) {
            cluster_barrier();
            return true;
        } else {
            return rbf::grid_barrier(count, gen, nb, err, ctl.wait_ns);
        }
    };
    for (int64_t step = 0; step < ctl.max_steps; ++step) {
        // every block sees the same done flags here (they change only before a barrier)
        bool any = false;
        for (int c = 0; c < ctl.ncells; ++c) any |= !((volatile int32_t *)ctl.done)[c];
        if (!any || (!CL && *(volatile int32_t *)ctl.err)) break;
        const bool check = ((step + 1) % ctl.check_every == 0) || (step + 1 == ctl.max_steps);
        for (int64_t s = w0; s < ctl.nslices * G; s += wstride) {
            const int2 sl = ctl.slices[s / G];
            if (ctl.done[sl.x]) continue;
            phase_predict<T, CP, G>(cells[sl.x], sl.y, (int)(s % G), lane, check);
        }
        if (!grid_barrier(ctl.bar_count, ctl.bar_gen, nblocks, ctl.err)) break;
        bool broke = false;
        for (int it = 0; it < ctl.n_p && !broke; ++it) {
            // slot parity of iteration `it` of this step for each cell: (parity0 + n_p * step + it) & 1
            if (blockIdx.x == 0)
                for (int ci = threadIdx.x; ci < ctl.ncells; ci += blockDim.x) {
                    if (ctl.done[ci]) continue;
                    const CellDesc<T> &c = cells[ci];
                    const int g = (int)((c.parity0 + (int64_t)ctl.n_p * step + it) & 1);
                    c.vmax[g] = 0ULL;
                }
            for (int64_t s = w0; s < ctl.nslices * G; s += wstride) {
                const int2 sl = ctl.slices[s / G];
                if (ctl.done[sl.x]) continue;
                const CellDesc<T> &c = cells[sl.x];
                phase_pressure<T, CP, G>(c, sl.y, (int)(s % G), lane, it == 0,
                                         (int)((c.parity0 + (int64_t)ctl.n_p * step + it) & 1));
            }
            if (!grid_barrier(ctl.bar_count, ctl.bar_gen, nblocks, ctl.err)) { broke = true; break; }
            for (int64_t s = w0; s < ctl.nwslices * G; s += wstride) {
                const int2 sl = ctl.wslices[s / G];
                if (ctl.done[sl.x]) continue;
                phase_wall<T, CP, G>(cells[sl.x], sl.y, (int)(s % G), lane);
            }
            if (!grid_barrier(ctl.bar_count, ctl.bar_gen, nblocks, ctl.err)) { broke = true; break; }
            for (int64_t s = w0; s < ctl.nslices * G; s += wstride) {
                const int2 sl = ctl.slices[s / G];
                if (ctl.done[sl.x]) continue;
                const CellDesc<T> &c = cells[sl.x];
                double sp = phase_correct<T, CP, G>(c, sl.y, (int)(s % G), lane);
                for (int off = 16; off > 0; off >>= 1) sp = fmax(sp, __shfl_xor_sync(0xffffffffu, sp, off));
                if (lane == 0 && sp > 0.0) {
                    const int g = (int)((c.parity0 + (int64_t)ctl.n_p * step + it) & 1);
                    atomicMax(c.vmax + g, (unsigned long long)__double_as_longlong(sp));
                }
            }
            if (!grid_barrier(ctl.bar_count, ctl.bar_gen, nblocks, ctl.err)) { broke = true; break; }
        }
        if (broke) break;
        if (check) {
            for (int t = threadIdx.x; t < 2 * ctl.ncells; t += blockDim.x) racc[t >> 1][t & 1] = 0.0;
            __syncthreads();
            for (int64_t s = w0; s < ctl.nslices; s += wstride) {
                const int2 sl = ctl.slices[s];
                if (ctl.done[sl.x]) continue;
                const CellDesc<T> &c = cells[sl.x];
                const int64_t i = ((int64_t)sl.y << 5) + lane;
                double d2 = 0.0, v2 = 0.0;
                if (i < c.n && !c.type[i]) {
                    double a = (double)c.u[i] - (double)c.uo[i], b = (double)c.v[i] - (double)c.vo[i];
                    double e = (double)c.w_[i] - (double)c.wo[i];
                    double uu = c.u[i], vv = c.v[i], ww = c.w_[i];
                    if constexpr (CP) {
                        a += (double)c.ul[i] - (double)c.uol[i];
                        b += (double)c.vl[i] - (double)c.vol[i];
                        e += (double)c.wl[i] - (double)c.wol[i];
                        uu += c.ul[i]; vv += c.vl[i]; ww += c.wl[i];
                    }
                    d2 = a * a + b * b + e * e;
                    v2 = uu * uu + vv * vv + ww * ww;
                }
                for (int off = 16; off > 0; off >>= 1) {
                    d2 += __shfl_xor_sync(0xffffffffu, d2, off);
                    v2 += __shfl_xor_sync(0xffffffffu, v2, off);
                }
                if (lane == 0) {
                    atomicAdd(&racc[sl.x][0], d2);
                    atomicAdd(&racc[sl.x][1], v2);
                }
            }
            __syncthreads();
            for (int t = threadIdx.x; t < 2 * ctl.ncells; t += blockDim.x)
                ctl.partial[(int64_t)blockIdx.x * 2 * PERSIST_MAX_CELLS + t] = racc[t >> 1][t & 1];
            if (!grid_barrier(ctl.bar_count, ctl.bar_gen, nblocks, ctl.err)) break;
            if (blockIdx.x == 0) {
                for (int c = threadIdx.x; c < ctl.ncells; c += blockDim.x) {
                    if (ctl.done[c]) continue;
                    double d2 = 0.0, v2 = 0.0;
                    for (unsigned b = 0; b < nblocks; ++b) {
                        d2 += ctl.partial[(int64_t)b * 2 * PERSIST_MAX_CELLS + 2 * c];
                        v2 += ctl.partial[(int64_t)b * 2 * PERSIST_MAX_CELLS + 2 * c + 1];
                    }
                    // a non-finite value anywhere in the cell's velocity makes d2 or v2
                    // non-finite (a NaN fails every comparison, so test before dividing)
                    const bool bad = !isfinite(d2) || !isfinite(v2);
                    const double res = bad ? (double)NAN : (v2 > 0.0 ? sqrt(d2) / sqrt(v2) : 0.0);
                    ctl.resid[c] = res;
                    ctl.steps[c] = step + 1;
                    if (bad) ctl.done[c] = 3;
                    else if (v2 > 0.0 && res < ctl.tol) ctl.done[c] = 1;
                }
            }
            if (!grid_barrier(ctl.bar_count, ctl.bar_gen, nblocks, ctl.err)) break;
        } else if (blockIdx.x == 0) {
            for (int c = threadIdx.x; c < ctl.ncells; c += blockDim.x)
                if (!ctl.done[c]) ctl.steps[c] = step + 1;
        }
    }
}

}  // namespace

bool persist_block_ok(int block) { return block == 32 || block == 64 || block == 128 || block == 256; }

namespace {
template <typename T, bool CP>
const void *grid_kernel(int group) {
    switch (group) {
    case 1: return (const void *)k_acm_persistent<T, CP, false, 1>;
    case 2: return (const void *)k_acm_persistent<T, CP, false, 2>;
    case 4: return (const void *)k_acm_persistent<T, CP, false, 4>;
    case 8: return (const void *)k_acm_persistent<T, CP, false, 8>;
    default: return nullptr;
    }
}
}  // namespace

template <typename T>
cudaError_t acm_launch_persistent(const CellDesc<T> *cells_dev, const PersistCtl &ctl, int nblocks, int block,
                                  int group, bool cp, cudaStream_t st) {
    const void *fn = cp ? grid_kernel<T, true>(group) : grid_kernel<T, false>(group);
    if (!persist_block_ok(block) || nblocks < 1 || !fn) return cudaErrorInvalidValue;
    void *args[] = {(void *)&cells_dev, (void *)&ctl};
    return cudaLaunchCooperativeKernel(fn, dim3(nblocks), dim3(block), args, 0, st);
}

namespace {
template <typename T, bool CP>
cudaError_t launch_cluster_T(const CellDesc<T> *cells_dev, const PersistCtl &ctl, int csize, cudaStream_t st,
                             int *max_clusters) {
    auto kern = k_acm_persistent<T, CP, true, 1>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
    if (e != cudaSuccess) return e;
    cudaLaunchConfig_t cfg;
    std::memset(&cfg, 0, sizeof(cfg));
    cfg.gridDim = dim3(csize);
    cfg.blockDim = dim3(256);
    cfg.stream = st;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeClusterDimension;
    at[0].val.clusterDim.x = csize;
    at[0].val.clusterDim.y = 1;
    at[0].val.clusterDim.z = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    if (max_clusters) return cudaOccupancyMaxActiveClusters(max_clusters, kern, &cfg);
    return cudaLaunchKernelEx(&cfg, kern, cells_dev, ctl);
}
}  // namespace

template <typename T>
cudaError_t acm_launch_persistent_cluster(const CellDesc<T> *cells_dev, const PersistCtl &ctl, int csize, bool cp,
                                          cudaStream_t st) {
    if (csize != 8 && csize != 16) return cudaErrorInvalidValue;
    return cp ? launch_cluster_T<T, true>(cells_dev, ctl, csize, st, nullptr)
              : launch_cluster_T<T, false>(cells_dev, ctl, csize, st, nullptr);
}

template <typename T>
cudaError_t acm_persistent_cluster_ok(int csize, bool cp, bool *ok) {
    *ok = false;
    if (csize != 8 && csize != 16) return cudaErrorInvalidValue;
    int n = 0;
    cudaError_t e = cp ? launch_cluster_T<T, true>(nullptr, PersistCtl{}, csize, nullptr, &n)
                       : launch_cluster_T<T, false>(nullptr, PersistCtl{}, csize, nullptr, &n);
    if (e != cudaSuccess) {
        cudaGetLastError();  // an unsupported size is an answer, not an error
        return cudaSuccess;
    }
    *ok = n >= 1;
    return cudaSuccess;
}

template <typename T>
cudaError_t acm_persistent_max_blocks(int *blocks, int block, int group, bool cp) {
    const void *fn = cp ? grid_kernel<T, true>(group) : grid_kernel<T, false>(group);
    if (!persist_block_ok(block) || !fn) return cudaErrorInvalidValue;
    int dev = 0, sms = 0, per = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, fn, block, 0);
    *blocks = sms * per;
    return e;
}

template cudaError_t acm_launch_persistent<float>(const CellDesc<float> *, const PersistCtl &, int, int, int, bool, cudaStream_t);
template cudaError_t acm_launch_persistent<double>(const CellDesc<double> *, const PersistCtl &, int, int, int, bool, cudaStream_t);
template cudaError_t acm_persistent_max_blocks<float>(int *, int, int, bool);
template cudaError_t acm_persistent_max_blocks<double>(int *, int, int, bool);
template cudaError_t acm_launch_persistent_cluster<float>(const CellDesc<float> *, const PersistCtl &, int, bool, cudaStream_t);
template cudaError_t acm_launch_persistent_cluster<double>(const CellDesc<double> *, const PersistCtl &, int, bool, cudaStream_t);
template cudaError_t acm_persistent_cluster_ok<float>(int, bool, bool *);
template cudaError_t acm_persistent_cluster_ok<double>(int, bool, bool *);

}  // namespace rbf
