// knn.cu — Morton ordering of the node cloud and periodic k-nearest-neighbour
// stencils (meshless discretisation section: S_i holds the N_L nodes closest to
// x_i; periodicity through the nearest image, case definition section).
//
// Nodes are sorted along a 3-D Morton curve (21 bits per axis) so that the nodes
// of one warp are close in space and the stencil gathers of the step kernels hit
// the same cache lines.  Neighbour search uses a uniform periodic cell grid and
// expanding Chebyshev rings; candidates are ranked by (squared distance computed
// without FMA, caller's node index), which makes the stencils bitwise
// reproducible and independent of the internal order.
#include "internal.cuh"

namespace rbf {

// ---- Morton keys ---------------------------------------------------------
__device__ __forceinline__ uint64_t spread21(uint64_t v) {
    v &= 0x1fffffULL;
    v = (v | (v << 32)) & 0x1f00000000ffffULL;
    v = (v | (v << 16)) & 0x1f0000ff0000ffULL;
    v = (v | (v << 8)) & 0x100f00f00f00f00fULL;
    v = (v | (v << 4)) & 0x10c30c30c30c30c3ULL;
    v = (v | (v << 2)) & 0x1249249249249249ULL;
    return v;
}

__device__ __forceinline__ uint64_t quant21(double x) {
    double s = x * 2097152.0;
    if (!(s >= 0.0)) s = 0.0;
    if (s > 2097151.0) s = 2097151.0;
    return (uint64_t)s;
}

__global__ void k_morton(int64_t n, const double *__restrict__ xyz, uint64_t *keys, int32_t *vals,
                         int64_t npow) {
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= npow) return;
    if (i < n) {
        uint64_t x = quant21(xyz[3 * i]), y = quant21(xyz[3 * i + 1]), z = quant21(xyz[3 * i + 2]);
        keys[i] = (spread21(x) << 2) | (spread21(y) << 1) | spread21(z);
        vals[i] = (int32_t)i;
    } else {
        keys[i] = ~0ULL;
        vals[i] = INT32_MAX;
    }
}

cudaError_t launch_morton_keys(int64_t n, const double *xyz, uint64_t *keys, int32_t *vals, int64_t npow,
                               cudaStream_t st) {
    k_morton<<<(unsigned)((npow + 255) / 256), 256, 0, st>>>(n, xyz, keys, vals, npow);
    return cudaGetLastError();
}

// ---- bitonic sort of (key, val) pairs, ascending by (key, val) -------------
__device__ __forceinline__ bool pair_gt(uint64_t ka, int32_t va, uint64_t kb, int32_t vb) {
    return ka > kb || (ka == kb && va > vb);
}

__global__ void k_bitonic_global(uint64_t *keys, int32_t *vals, int64_t npow, int64_t j, int64_t k) {
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= npow) return;
    int64_t p = i ^ j;
    if (p <= i) return;
    bool up = (i & k) == 0;
    uint64_t ki = keys[i], kp = keys[p];
    int32_t vi = vals[i], vp = vals[p];
    if (pair_gt(ki, vi, kp, vp) == up) {
        keys[i] = kp; keys[p] = ki;
        vals[i] = vp; vals[p] = vi;
    }
}

// all steps with j < 1024 of stage k, in shared memory (2048 elements per block)
__global__ void k_bitonic_shared(uint64_t *keys, int32_t *vals, int64_t npow, int64_t k, int64_t jmax) {
    __shared__ uint64_t sk[2048];
    __shared__ int32_t sv[2048];
    int64_t base = blockIdx.x * 2048LL;
    for (int t = threadIdx.x; t < 2048; t += blockDim.x) {
        sk[t] = keys[base + t];
        sv[t] = vals[base + t];
    }
    __syncthreads();
    for (int64_t j = jmax; j > 0; j >>= 1) {
        for (int t = threadIdx.x; t < 2048; t += blockDim.x) {
            int p = t ^ (int)j;
            if (p > t) {
                int64_t gi = base + t;
                bool up = (gi & k) == 0;
                if (pair_gt(sk[t], sv[t], sk[p], sv[p]) == up) {
                    uint64_t tk = sk[t]; sk[t] = sk[p]; sk[p] = tk;
                    int32_t tv = sv[t]; sv[t] = sv[p]; sv[p] = tv;
                }
            }
        }
        __syncthreads();
    }
    for (int t = threadIdx.x; t < 2048; t += blockDim.x) {
        keys[base + t] = sk[t];
        vals[base + t] = sv[t];
    }
}

cudaError_t launch_bitonic_sort(uint64_t *keys, int32_t *vals, int64_t npow, cudaStream_t st, int64_t *launches) {
    unsigned blocks = (unsigned)((npow + 255) / 256);
    for (int64_t k = 2; k <= npow; k <<= 1) {
        int64_t j = k >> 1;
        for (; j >= 1024 || (j >= 1 && npow < 2048); j >>= 1) {
            k_bitonic_global<<<blocks, 256, 0, st>>>(keys, vals, npow, j, k);
            ++*launches;
        }
        if (j >= 1 && npow >= 2048) {
            k_bitonic_shared<<<(unsigned)(npow / 2048), 1024, 0, st>>>(keys, vals, npow, k, j);
            ++*launches;
        }
    }
    return cudaGetLastError();
}

__global__ void k_gather_nodes(int64_t n, const int32_t *__restrict__ perm, const double *__restrict__ xyz,
                               const uint8_t *__restrict__ type, const double *__restrict__ nrm, double *xyz_s,
                               uint8_t *type_s, double *nrm_s, int32_t *iperm) {
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n) return;
    int64_t o = perm[i];
    for (int a = 0; a < 3; ++a) {
        xyz_s[3 * i + a] = xyz[3 * o + a];
        nrm_s[3 * i + a] = nrm[3 * o + a];
    }
    type_s[i] = type[o];
    iperm[o] = (int32_t)i;
}

cudaError_t launch_gather_nodes(int64_t n, const int32_t *perm, const double *xyz, const uint8_t *type,
                                const double *nrm, double *xyz_s, uint8_t *type_s, double *nrm_s,
                                int32_t *iperm, cudaStream_t st) {
    k_gather_nodes<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(n, perm, xyz, type, nrm, xyz_s, type_s, nrm_s,
                                                               iperm);
    return cudaGetLastError();
}

// ---- exclusive scan of int32 (three passes, 1024 elements per block) --------
__device__ __forceinline__ int32_t warp_incl_scan(int32_t v) {
    int lane = threadIdx.x & 31;
    for (int d = 1; d < 32; d <<= 1) {
        int32_t t = __shfl_up_sync(0xffffffffu, v, d);
        if (lane >= d) v += t;
    }
    return v;
}

__global__ void k_scan_blocks(const int32_t *in, int32_t *out, int64_t n, int32_t *sums) {
    __shared__ int32_t ws[32];
    int64_t i = blockIdx.x * 1024LL + threadIdx.x;
    int32_t v = i < n ? in[i] : 0;
    int32_t inc = warp_incl_scan(v);
    int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (lane == 31) ws[w] = inc;
    __syncthreads();
    if (w == 0) {
        int32_t t = ws[lane];
        ws[lane] = warp_incl_scan(t) - t;
    }
    __syncthreads();
    int32_t ex = inc - v + ws[w];
    if (i < n) out[i] = ex;
    if (threadIdx.x == 1023) sums[blockIdx.x] = ex + v;
}

__global__ void k_scan_sums(int32_t *sums, int64_t nb) {
    __shared__ int32_t ws[32];
    __shared__ int32_t carry;
    if (threadIdx.x == 0) carry = 0;
    __syncthreads();
    for (int64_t base = 0; base < nb; base += 1024) {
        int64_t i = base + threadIdx.x;
        int32_t v = i < nb ? sums[i] : 0;
        int32_t inc = warp_incl_scan(v);
        int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
        if (lane == 31) ws[w] = inc;
        __syncthreads();
        if (w == 0) {
            int32_t t = ws[lane];
            ws[lane] = warp_incl_scan(t) - t;
        }
        __syncthreads();
        int32_t ex = inc - v + ws[w] + carry;
        __syncthreads();
        if (i < nb) sums[i] = ex;
        if (threadIdx.x == 1023) carry = ex + v;
        __syncthreads();
    }
}

__global__ void k_scan_add(int32_t *out, int64_t n, const int32_t *sums) {
    int64_t i = blockIdx.x * 1024LL + threadIdx.x;
    if (i < n) out[i] += sums[blockIdx.x];
}

int64_t scan_tmp_len(int64_t n) { return (n + 1023) / 1024 + 1; }

cudaError_t launch_scan_i32(const int32_t *in, int32_t *out, int64_t n, int32_t *tmp, int64_t tmp_len,
                            cudaStream_t st, int64_t *launches) {
    int64_t nb = (n + 1023) / 1024;
    if (nb + 1 > tmp_len) return cudaErrorInvalidValue;
    k_scan_blocks<<<(unsigned)nb, 1024, 0, st>>>(in, out, n, tmp);
    k_scan_sums<<<1, 1024, 0, st>>>(tmp, nb);
    k_scan_add<<<(unsigned)nb, 1024, 0, st>>>(out, n, tmp);
    *launches += 3;
    return cudaGetLastError();
}

// ---- cell grid -------------------------------------------------------------
__device__ __forceinline__ int cell_coord(double x, int G) {
    int c = (int)(x * G);
    return c < 0 ? 0 : (c >= G ? G - 1 : c);
}

__global__ void k_cell_count(int64_t n, const double *__restrict__ xyz, int G, int32_t *cell_of, int32_t *count) {
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n) return;
    int cx = cell_coord(xyz[3 * i], G), cy = cell_coord(xyz[3 * i + 1], G), cz = cell_coord(xyz[3 * i + 2], G);
    int32_t c = (int32_t)(((int64_t)cx * G + cy) * G + cz);
    cell_of[i] = c;
    atomicAdd(&count[c], 1);
}

cudaError_t launch_cell_count(int64_t n, const double *xyz, int G, int32_t *cell_of, int32_t *count,
                              cudaStream_t st) {
    k_cell_count<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(n, xyz, G, cell_of, count);
    return cudaGetLastError();
}

__global__ void k_cell_fill(int64_t n, const int32_t *cell_of, const int32_t *start, int32_t *fill,
                            int32_t *items) {
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n) return;
    int32_t c = cell_of[i];
    items[start[c] + atomicAdd(&fill[c], 1)] = (int32_t)i;
}

cudaError_t launch_cell_fill(int64_t n, const int32_t *cell_of, const int32_t *start, int32_t *fill,
                             int32_t *items, cudaStream_t st) {
    k_cell_fill<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(n, cell_of, start, fill, items);
    return cudaGetLastError();
}

__global__ void k_type_flags(int64_t n, const uint8_t *type, uint8_t want, int32_t *flags) {
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i < n) flags[i] = type[i] == want;
}

cudaError_t launch_type_flags(int64_t n, const uint8_t *type, uint8_t want, int32_t *flags, cudaStream_t st) {
    k_type_flags<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(n, type, want, flags);
    return cudaGetLastError();
}

__global__ void k_flag_compact(int64_t n, const uint8_t *type, uint8_t want, const int32_t *scan, int32_t *list) {
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i < n && type[i] == want) list[scan[i]] = (int32_t)i;
}

cudaError_t launch_flag_compact(int64_t n, const uint8_t *type, uint8_t want, const int32_t *scan,
                                int32_t *list, cudaStream_t st) {
    k_flag_compact<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(n, type, want, scan, list);
    return cudaGetLastError();
}

// ---- k nearest neighbours ---------------------------------------------------
// One thread per query.  The best n_l candidates are kept sorted in local memory
// by (d2, orig).  Rings of cells at Chebyshev distance r = 0, 1, ... around the
// query's cell are scanned; after ring r every unseen node is at least r*cs
// away, so the search stops once the n_l-th distance is below (r cs)^2, or when
// the whole periodic grid has been seen.
__global__ void __launch_bounds__(128) k_knn(int64_t nq, const double *__restrict__ qxyz,
                                             const int32_t *__restrict__ qnode, const double *__restrict__ xyz,
                                             const int32_t *__restrict__ perm, const uint8_t *__restrict__ type,
                                             int fluid_only, int G, const int32_t *__restrict__ cstart,
                                             const int32_t *__restrict__ citems, int n_l, int32_t *out, int ld,
                                             int col0, int32_t *status) {
    int64_t a = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (a >= nq) return;
    double bd[RBF_MAX_NL];
    int32_t bo[RBF_MAX_NL];
    int32_t bs[RBF_MAX_NL];
    int cnt = 0;
    double qx, qy, qz;
    if (qxyz) {
        qx = qxyz[3 * a]; qy = qxyz[3 * a + 1]; qz = qxyz[3 * a + 2];
    } else {
        int64_t s = qnode[a];
        qx = xyz[3 * s]; qy = xyz[3 * s + 1]; qz = xyz[3 * s + 2];
    }
    qx -= floor(qx); qy -= floor(qy); qz -= floor(qz);
    const double cs = 1.0 / G;
    int cx = cell_coord(qx, G), cy = cell_coord(qy, G), cz = cell_coord(qz, G);
    const int lo = -((G - 1) / 2), hi = G / 2;  // distinct periodic offsets
    for (int r = 0;; ++r) {
        bool any = false;
        int ax0 = max(-r, lo), ax1 = min(r, hi);
        for (int dx = ax0; dx <= ax1; ++dx)
            for (int dy = ax0; dy <= ax1; ++dy)
                for (int dz = ax0; dz <= ax1; ++dz) {
                    int m = max(abs(dx), max(abs(dy), abs(dz)));
                    if (m != r) continue;
                    any = true;
                    int ix = (cx + dx + G) % G, iy = (cy + dy + G) % G, iz = (cz + dz + G) % G;
                    int64_t c = ((int64_t)ix * G + iy) * G + iz;
                    int32_t e0 = cstart[c], e1 = cstart[c + 1];
                    for (int32_t e = e0; e < e1; ++e) {
                        int32_t s = citems[e];
                        if (fluid_only && type[s]) continue;
                        double ddx = mimg(xyz[3 * s] - qx);
                        double ddy = mimg(xyz[3 * s + 1] - qy);
                        double ddz = mimg(xyz[3 * s + 2] - qz);
                        double d2 = dist2_nofma(ddx, ddy, ddz);
                        int32_t o = perm[s];
                        if (cnt == n_l && (d2 > bd[cnt - 1] || (d2 == bd[cnt - 1] && o > bo[cnt - 1]))) continue;
                        int pos = cnt < n_l ? cnt++ : cnt - 1;
                        while (pos > 0 && (bd[pos - 1] > d2 || (bd[pos - 1] == d2 && bo[pos - 1] > o))) {
                            bd[pos] = bd[pos - 1]; bo[pos] = bo[pos - 1]; bs[pos] = bs[pos - 1];
                            --pos;
                        }
                        bd[pos] = d2; bo[pos] = o; bs[pos] = s;
                    }
                }
        if (!any) break;  // every cell seen
        double reach = r * cs;
        if (cnt == n_l && bd[n_l - 1] < reach * reach * (1.0 - 1e-12)) break;
    }
    if (cnt < n_l) {
        atomicExch(status, 1);
        for (int t = cnt; t < n_l; ++t) bs[t] = cnt > 0 ? bs[0] : 0;  // flagged: never used
    }
    for (int t = 0; t < n_l; ++t) out[a * ld + col0 + t] = bs[t];
}

cudaError_t launch_knn(int64_t nq, const double *qxyz, const int32_t *qnode, const double *xyz,
                       const int32_t *perm, const uint8_t *type, int fluid_only, int G,
                       const int32_t *cell_start, const int32_t *cell_items, int n_l, int32_t *out, int ld,
                       int col0, int32_t *status, cudaStream_t st) {
    if (nq <= 0) return cudaSuccess;
    k_knn<<<(unsigned)((nq + 127) / 128), 128, 0, st>>>(nq, qxyz, qnode, xyz, perm, type, fluid_only, G,
                                                        cell_start, cell_items, n_l, out, ld, col0, status);
    return cudaGetLastError();
}

}  // namespace rbf
