// weights.cu — RBF-FD stencil weights, batched: one warp per stencil.
//
// For every centre x_c with stencil S (N_L nodes) the warp assembles the saddle
// system of Eq. augmentedSystem in shared memory, FP64:
//   A_jl = |xi_j - xi_l|^k      (PHS r^k, Eq. rbfScaling: xi = (x - x_c) / delta)
//   P_jl = p_l(xi_j)            (monomials of degree <= m, graded lexicographic)
//   M = [[A, P], [P^T, 0]]
// factors it by LU with partial pivoting (warp-parallel rank-1 updates), and
// solves the right-hand sides of up to RBF_MAX_OPS operators L (Eq.
// operatorApprox) together, the warp's lanes spread over (row, operator) pairs:
//   b_j = (L Phi_j)(y), c_l = (L p_l)(y),  y = x_c + off
// followed by one step of iterative refinement whose residual is accumulated
// with the compensated dot product Dot2 (Ogita, Rump & Oishi, SIAM J. Sci.
// Comput. 26, 2005), i.e. as if in twice the working precision.  delta is the
// distance to the nearest other node (centre is a node) or to the nearest node
// (centre is a free point such as a permeability probe).
#include "internal.cuh"

namespace rbf {

__device__ __forceinline__ double ipow(double x, int e) {
    double r = 1.0;
    for (int i = 0; i < e; ++i) r *= x;
    return r;
}

// exponents (a, b, c) of the l-th monomial, graded lexicographic order
__device__ void mono_exp(int l, int *a, int *b, int *c) {
    int cnt = 0;
    for (int d = 0;; ++d)
        for (int x = d; x >= 0; --x)
            for (int y = d - x; y >= 0; --y) {
                if (cnt == l) { *a = x; *b = y; *c = d - x - y; return; }
                ++cnt;
            }
}

// L applied to the basis function centred at xi_j, at eta; s = eta - xi_j
__device__ double rbf_rhs(int kind, int k, double sx, double sy, double sz, double delta) {
    double rho = sqrt(sx * sx + sy * sy + sz * sz);
    switch (kind) {
    case OP_INTERP: return ipow(rho, k);
    case OP_DX: return (double)k * ipow(rho, k - 2) * sx / delta;
    case OP_DY: return (double)k * ipow(rho, k - 2) * sy / delta;
    case OP_DZ: return (double)k * ipow(rho, k - 2) * sz / delta;
    default: return (double)(k * (k + 1)) * ipow(rho, k - 2) / (delta * delta);
    }
}

// L applied to x^a y^b z^c at eta (scaled coordinates; derivatives in physical ones)
__device__ double mono_rhs(int kind, int a, int b, int c, double ex, double ey, double ez, double delta) {
    switch (kind) {
    case OP_INTERP: return ipow(ex, a) * ipow(ey, b) * ipow(ez, c);
    case OP_DX: return a ? (double)a * ipow(ex, a - 1) * ipow(ey, b) * ipow(ez, c) / delta : 0.0;
    case OP_DY: return b ? (double)b * ipow(ex, a) * ipow(ey, b - 1) * ipow(ez, c) / delta : 0.0;
    case OP_DZ: return c ? (double)c * ipow(ex, a) * ipow(ey, b) * ipow(ez, c - 1) / delta : 0.0;
    default: {
        double s = 0.0;
        if (a >= 2) s += (double)(a * (a - 1)) * ipow(ex, a - 2) * ipow(ey, b) * ipow(ez, c);
        if (b >= 2) s += (double)(b * (b - 1)) * ipow(ex, a) * ipow(ey, b - 2) * ipow(ez, c);
        if (c >= 2) s += (double)(c * (c - 1)) * ipow(ex, a) * ipow(ey, b) * ipow(ez, c - 2);
        return s / (delta * delta);
    }
    }
}

// Solve with the in-place LU (rows swapped as recorded in piv) for all n_rhs
// columns of the row-major [ns][n_rhs] block X at once, by the whole warp:
// forward elimination with the unit lower factor, then back substitution with
// the upper one, both column by column so that every step is one warp-wide
// update over the (row, column) pairs below (above) the pivot.  Each entry sees
// its subtractions in the order of a row-oriented substitution in the forward
// pass and in decreasing column order in the backward pass.
__device__ void lu_solve_warp(int ns, int ld, const double *M, const int *piv, double *X, int n_rhs, int lane) {
    for (int o = lane; o < n_rhs; o += 32)
        for (int c = 0; c < ns; ++c) {
            const int p = piv[c];
            if (p != c) { double t = X[c * n_rhs + o]; X[c * n_rhs + o] = X[p * n_rhs + o]; X[p * n_rhs + o] = t; }
        }
    __syncwarp();
    for (int c = 0; c < ns - 1; ++c) {
        const int cnt = (ns - c - 1) * n_rhs;
        for (int e = lane; e < cnt; e += 32) {
            const int r = c + 1 + e / n_rhs, o = e - (r - c - 1) * n_rhs;
            X[r * n_rhs + o] -= M[r * ld + c] * X[c * n_rhs + o];
        }
        __syncwarp();
    }
    for (int c = ns - 1; c >= 0; --c) {
        for (int o = lane; o < n_rhs; o += 32) X[c * n_rhs + o] /= M[c * ld + c];
        __syncwarp();
        const int cnt = c * n_rhs;
        for (int e = lane; e < cnt; e += 32) {
            const int r = e / n_rhs, o = e - r * n_rhs;
            X[r * n_rhs + o] -= M[r * ld + c] * X[c * n_rhs + o];
        }
        __syncwarp();
    }
}

struct WLayout {
    int ns, ld;      // system size, padded row stride
    int n_ops;
    size_t per_warp; // doubles per warp
};

__host__ __device__ inline WLayout wlayout(int n_l, int np, int n_ops) {
    WLayout L;
    L.ns = n_l + np;
    L.ld = L.ns | 1;  // odd stride: FP64 rows fall on different banks
    L.n_ops = n_ops;
    // M, Morig (ns x ld each), X, R, D (ns x n_ops each), xi (n_l x 3), piv (ns ints, one double each)
    L.per_warp = (size_t)2 * L.ns * L.ld + (size_t)3 * L.ns * n_ops + 3 * (size_t)n_l + L.ns;
    return L;
}

// One stencil's saddle system and its right-hand sides, by one warp; `smem_w` is
// the warp's shared-memory region (at least wlayout(n_l, np, n_ops).per_warp doubles).
__device__ void weights_one(int64_t c, double *smem_w, const double *__restrict__ xyz, const double *__restrict__ cxyz,
                            const int32_t *__restrict__ cnode, int centre_is_node, int n_l,
                            const int32_t *__restrict__ idx, int k, int np, int n_ops,
                            const OpSpec *__restrict__ ops, int refine, double *__restrict__ wout,
                            double *__restrict__ delta_out, int32_t *n_sing) {
    const int lane = threadIdx.x & 31;
    const WLayout L = wlayout(n_l, np, n_ops);
    const int ns = L.ns, ld = L.ld;
    double *M = smem_w;
    double *M0 = M + (size_t)ns * ld;
    double *X = M0 + (size_t)ns * ld;       // [r][o]
    double *R = X + (size_t)ns * n_ops;     // [r][o]
    double *D = R + (size_t)ns * n_ops;     // [r][o]
    double *xi = D + (size_t)ns * n_ops;    // [j][3]
    int *piv = (int *)(xi + 3 * n_l);

    double xc, yc, zc;
    if (cxyz) { xc = cxyz[3 * c]; yc = cxyz[3 * c + 1]; zc = cxyz[3 * c + 2]; }
    else { int64_t s = cnode[c]; xc = xyz[3 * s]; yc = xyz[3 * s + 1]; zc = xyz[3 * s + 2]; }
    for (int j = lane; j < n_l; j += 32) {
        int64_t s = idx[c * n_l + j];
        xi[3 * j] = mimg(xyz[3 * s] - xc);
        xi[3 * j + 1] = mimg(xyz[3 * s + 1] - yc);
        xi[3 * j + 2] = mimg(xyz[3 * s + 2] - zc);
    }
    __syncwarp();
    const int jd = centre_is_node ? 1 : 0;
    const double delta = sqrt(xi[3 * jd] * xi[3 * jd] + xi[3 * jd + 1] * xi[3 * jd + 1] + xi[3 * jd + 2] * xi[3 * jd + 2]);
    if (lane == 0 && delta_out) delta_out[c] = delta;
    __syncwarp();
    for (int j = lane; j < n_l; j += 32) {
        xi[3 * j] /= delta; xi[3 * j + 1] /= delta; xi[3 * j + 2] /= delta;
    }
    __syncwarp();
    // assemble
    for (int e = lane; e < ns * ns; e += 32) {
        int r = e / ns, q = e - r * ns;
        double v;
        if (r < n_l && q < n_l) {
            v = rbf_rhs(OP_INTERP, k, xi[3 * r] - xi[3 * q], xi[3 * r + 1] - xi[3 * q + 1], xi[3 * r + 2] - xi[3 * q + 2], delta);
        } else if (r < n_l) {
            int a, b, cc; mono_exp(q - n_l, &a, &b, &cc);
            v = mono_rhs(OP_INTERP, a, b, cc, xi[3 * r], xi[3 * r + 1], xi[3 * r + 2], delta);
        } else if (q < n_l) {
            int a, b, cc; mono_exp(r - n_l, &a, &b, &cc);
            v = mono_rhs(OP_INTERP, a, b, cc, xi[3 * q], xi[3 * q + 1], xi[3 * q + 2], delta);
        } else {
            v = 0.0;
        }
        M[r * ld + q] = v;
        M0[r * ld + q] = v;
    }
    __syncwarp();
    // LU with partial pivoting (rows swapped in full, multipliers stored below)
    bool singular = false;
    for (int col = 0; col < ns; ++col) {
        double best = -1.0;
        int bi = ns;
        for (int r = col + lane; r < ns; r += 32) {
            double v = fabs(M[r * ld + col]);
            if (v > best) { best = v; bi = r; }
        }
        for (int off = 16; off > 0; off >>= 1) {
            double ob = __shfl_xor_sync(0xffffffffu, best, off);
            int oi = __shfl_xor_sync(0xffffffffu, bi, off);
            if (ob > best || (ob == best && oi < bi)) { best = ob; bi = oi; }
        }
        if (!(best > 0.0)) { singular = true; break; }
        if (lane == 0) piv[col] = bi;
        if (bi != col)
            for (int q = lane; q < ns; q += 32) {
                double t = M[col * ld + q]; M[col * ld + q] = M[bi * ld + q]; M[bi * ld + q] = t;
            }
        __syncwarp();
        const double pv = M[col * ld + col];
        for (int r = col + 1 + lane; r < ns; r += 32) M[r * ld + col] /= pv;
        __syncwarp();
        const int R1 = ns - col - 1;
        for (int e = lane; e < R1 * R1; e += 32) {
            int r = col + 1 + e / R1, q = col + 1 + e % R1;
            M[r * ld + q] -= M[r * ld + col] * M[col * ld + q];
        }
        __syncwarp();
    }
    if (singular) {
        if (lane == 0) atomicAdd(n_sing, 1);
        for (int e = lane; e < n_ops * n_l; e += 32) wout[c * n_ops * n_l + e] = __longlong_as_double(0x7ff8000000000000LL);
        return;
    }
    __syncwarp();
    // right-hand sides R[r][o] (row r of operator o), warp-wide over (r, o)
    for (int e = lane; e < ns * n_ops; e += 32) {
        const int r = e / n_ops, o = e - r * n_ops;
        const OpSpec op = ops[o];
        const double ex = op.off[0] / delta, ey = op.off[1] / delta, ez = op.off[2] / delta;
        double v;
        if (r < n_l) {
            v = rbf_rhs(op.kind, k, ex - xi[3 * r], ey - xi[3 * r + 1], ez - xi[3 * r + 2], delta);
        } else {
            int a, b, cc; mono_exp(r - n_l, &a, &b, &cc);
            v = mono_rhs(op.kind, a, b, cc, ex, ey, ez, delta);
        }
        R[e] = v;
        X[e] = v;
    }
    __syncwarp();
    lu_solve_warp(ns, ld, M, piv, X, n_ops, lane);
    for (int it = 0; it < refine; ++it) {
        // D = rhs - M0 x, each entry a compensated dot product (Dot2), warp-wide over (r, o)
        for (int e = lane; e < ns * n_ops; e += 32) {
            const int r = e / n_ops, o = e - r * n_ops;
            double s = R[e], cmp = 0.0;
            for (int q = 0; q < ns; ++q) {
                const double a = M0[r * ld + q], x = X[q * n_ops + o];
                const double p = -a * x;
                const double pe = fma(-a, x, -p);  // -a x = p + pe exactly
                const double t = s + p;
                const double z = t - s;
                cmp += ((s - (t - z)) + (p - z)) + pe;
                s = t;
            }
            D[e] = s + cmp;
        }
        __syncwarp();
        lu_solve_warp(ns, ld, M, piv, D, n_ops, lane);
        for (int e = lane; e < ns * n_ops; e += 32) X[e] += D[e];
        __syncwarp();
    }
    __syncwarp();
    for (int e = lane; e < n_ops * n_l; e += 32) {
        int o = e / n_l, j = e - o * n_l;
        wout[(c * n_ops + o) * n_l + j] = X[j * n_ops + o];
    }
}

__global__ void k_weights(int64_t nc, const double *__restrict__ xyz, const double *__restrict__ cxyz,
                          const int32_t *__restrict__ cnode, int centre_is_node, int n_l,
                          const int32_t *__restrict__ idx, int k, int m, int np, int n_ops,
                          const OpSpec *__restrict__ ops, int refine, double *__restrict__ wout,
                          double *__restrict__ delta_out, int32_t *n_sing) {
    extern __shared__ double smem[];
    const int warp = threadIdx.x >> 5;
    const int64_t c = blockIdx.x * (int64_t)(blockDim.x >> 5) + warp;
    if (c >= nc) return;
    (void)m;
    weights_one(c, smem + warp * wlayout(n_l, np, n_ops).per_warp, xyz, cxyz, cnode, centre_is_node, n_l, idx, k, np,
                n_ops, ops, refine, wout, delta_out, n_sing);
}

// Many stencil sets (e.g. the nodes of many cells, each with its own N_L) in one
// launch: warp t solves centre t of the concatenation of the jobs.
__global__ void k_weights_multi(int njobs, const WeightJob *__restrict__ jobs, const int64_t *__restrict__ prefix,
                                int64_t ntot, size_t per_warp, int k, int np, int n_ops, const OpSpec *__restrict__ ops,
                                int refine, int32_t *n_sing) {
    extern __shared__ double smem[];
    const int warp = threadIdx.x >> 5;
    const int64_t t = blockIdx.x * (int64_t)(blockDim.x >> 5) + warp;
    if (t >= ntot) return;
    int j = 0;
    while (j + 1 < njobs && prefix[j + 1] <= t) ++j;
    const WeightJob jb = jobs[j];
    weights_one(t - prefix[j], smem + warp * per_warp, jb.xyz, nullptr, jb.cnode, 1, jb.n_l, jb.idx, k, np, n_ops, ops,
                refine, jb.w, jb.delta, n_sing);
}

cudaError_t launch_weights_multi(int njobs, const WeightJob *jobs_dev, const int64_t *prefix_dev, int64_t ntot,
                                 int max_n_l, int k, int m, int n_ops, const OpSpec *ops, int refine, int32_t *n_sing,
                                 cudaStream_t st) {
    if (ntot <= 0) return cudaSuccess;
    if (n_ops < 1 || n_ops > RBF_MAX_OPS || max_n_l < 2 || max_n_l > RBF_MAX_NL || m < 0 || m > 4) return cudaErrorInvalidValue;
    const int np = (m + 1) * (m + 2) * (m + 3) / 6;
    const WLayout L = wlayout(max_n_l, np, n_ops);
    const size_t per_warp_bytes = L.per_warp * sizeof(double);
    int warps = (int)((200 * 1024) / per_warp_bytes);
    if (warps > 4) warps = 4;
    if (warps < 1) return cudaErrorInvalidValue;
    const size_t smem = per_warp_bytes * warps;
    cudaError_t e = cudaFuncSetAttribute(k_weights_multi, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    k_weights_multi<<<(unsigned)((ntot + warps - 1) / warps), 32 * warps, smem, st>>>(njobs, jobs_dev, prefix_dev, ntot,
                                                                                     L.per_warp, k, np, n_ops, ops,
                                                                                     refine, n_sing);
    return cudaGetLastError();
}

cudaError_t launch_weights(int64_t nc, const double *xyz, const double *cxyz, const int32_t *cnode,
                           int centre_is_node, int n_l, const int32_t *idx, int k, int m, int n_ops,
                           const OpSpec *ops, int refine, double *w, double *delta, int32_t *n_sing,
                           cudaStream_t st) {
    if (nc <= 0) return cudaSuccess;
    if (n_ops < 1 || n_ops > RBF_MAX_OPS || n_l < 2 || n_l > RBF_MAX_NL || m < 0 || m > 4) return cudaErrorInvalidValue;
    int np = (m + 1) * (m + 2) * (m + 3) / 6;
    WLayout L = wlayout(n_l, np, n_ops);
    size_t per_warp_bytes = L.per_warp * sizeof(double);
    int warps = (int)((200 * 1024) / per_warp_bytes);
    if (warps > 4) warps = 4;
    if (warps < 1) return cudaErrorInvalidValue;
    size_t smem = per_warp_bytes * warps;
    cudaError_t e = cudaFuncSetAttribute(k_weights, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    unsigned blocks = (unsigned)((nc + warps - 1) / warps);
    k_weights<<<blocks, 32 * warps, smem, st>>>(nc, xyz, cxyz, cnode, centre_is_node, n_l, idx, k, m, np, n_ops,
                                                 ops, refine, w, delta, n_sing);
    return cudaGetLastError();
}

// ---- FP32 copies of the weights ---------------------------------------------
// Each row of n_l FP64 weights (one operator at one centre) is rounded to FP32 so
// that the exact sum of the FP32 values stays at the FP64 row sum: every weight is
// rounded to nearest, then the sum's residual is added to the smallest-magnitude
// nonzero weight, which is rounded again (its ulp bounds what is left).  Plain
// rounding leaves each row sum off by ~1e-7 of its weights' size, so constants
// are no longer reproduced (interpolation rows no longer sum to 1, derivative
// rows no longer to 0); the explicit iterations carry that error in every step
// and in the MLBM it biased the steady permeability by 2e-4 on the 150k-node cell.
// out holds the FP32 values as doubles (exactly representable), rows as in w.
__global__ void k_round_rows_f32(int64_t nrows, int n_l, const double *__restrict__ w, double *__restrict__ out) {
    int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (r >= nrows) return;
    const double *a = w + r * n_l;
    double *o = out + r * n_l;
    double s64 = 0.0, s32 = 0.0, amin = 0.0;
    int jmin = -1;
    for (int j = 0; j < n_l; ++j) {
        const float f = (float)a[j];
        s64 += a[j];
        s32 += (double)f;
        o[j] = (double)f;
        if (f != 0.0f && (jmin < 0 || fabs((double)f) < amin)) { amin = fabs((double)f); jmin = j; }
    }
    if (jmin >= 0) o[jmin] = (double)(float)(o[jmin] + (s64 - s32));
}

cudaError_t launch_round_rows_f32(int64_t nrows, int n_l, const double *w, double *out, cudaStream_t st) {
    if (nrows == 0) return cudaSuccess;
    k_round_rows_f32<<<(unsigned)((nrows + 255) / 256), 256, 0, st>>>(nrows, n_l, w, out);
    return cudaGetLastError();
}

// wall normal-derivative rows w^n_j = n_x w^x_j + n_y w^y_j + n_z w^z_j (FP64,
// [nb][n_l]) from the gradient weights of the wall nodes' Neumann stencils
__global__ void k_normal_rows(int64_t nb, int n_l, const int32_t *__restrict__ wall, const double *__restrict__ nrm,
                              const double *__restrict__ wg, double *__restrict__ out) {
    int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (t >= nb * n_l) return;
    int64_t b = t / n_l;
    int j = (int)(t - b * n_l);
    int64_t i = wall[b];
    const double *g = wg + b * 3 * n_l;
    double nx = nrm[3 * i], ny = nrm[3 * i + 1], nz = nrm[3 * i + 2];
    out[t] = __dadd_rn(__dadd_rn(__dmul_rn(nx, g[j]), __dmul_rn(ny, g[n_l + j])), __dmul_rn(nz, g[2 * n_l + j]));
}

cudaError_t launch_normal_rows(int64_t nb, int n_l, const int32_t *wall, const double *nrm, const double *wg,
                               double *out, cudaStream_t st) {
    int64_t tot = nb * n_l;
    if (tot == 0) return cudaSuccess;
    k_normal_rows<<<(unsigned)((tot + 255) / 256), 256, 0, st>>>(nb, n_l, wall, nrm, wg, out);
    return cudaGetLastError();
}

// ---- packing into SELL-C slices for the step kernels ------------------------
template <typename T>
__global__ void k_pack(int64_t nc, int n_ops, int o0, int n_out, int n_l, const double *__restrict__ w, T *ws) {
    // one thread per (centre, j); centres beyond nc (the last slice's padding) get 0
    int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    int64_t npad = (nc + 31) & ~31LL;
    if (t >= npad * n_l) return;
    int64_t c = t / n_l;
    int j = (int)(t - c * n_l);
    int64_t s = c >> 5;
    int lane = (int)(c & 31);
    for (int o = 0; o < n_out; ++o)
        ws[sell_at(s, o, j, lane, n_out, n_l)] = c < nc ? (T)w[(c * n_ops + o0 + o) * n_l + j] : (T)0;
}

cudaError_t launch_pack_f32(int64_t nc, int n_ops, int o0, int n_out, int n_l, const double *w, float *ws,
                            cudaStream_t st) {
    int64_t tot = ((nc + 31) & ~31LL) * n_l;
    if (tot == 0) return cudaSuccess;
    k_pack<float><<<(unsigned)((tot + 255) / 256), 256, 0, st>>>(nc, n_ops, o0, n_out, n_l, w, ws);
    return cudaGetLastError();
}
cudaError_t launch_pack_f64(int64_t nc, int n_ops, int o0, int n_out, int n_l, const double *w, double *ws,
                            cudaStream_t st) {
    int64_t tot = ((nc + 31) & ~31LL) * n_l;
    if (tot == 0) return cudaSuccess;
    k_pack<double><<<(unsigned)((tot + 255) / 256), 256, 0, st>>>(nc, n_ops, o0, n_out, n_l, w, ws);
    return cudaGetLastError();
}

__global__ void k_pack_idx(int64_t nc, int n_l, const int32_t *__restrict__ idx, int32_t *is) {
    int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    int64_t npad = (nc + 31) & ~31LL;
    if (t >= npad * n_l) return;
    int64_t c = t / n_l;
    int j = (int)(t - c * n_l);
    is[sell_at(c >> 5, 0, j, (int)(c & 31), 1, n_l)] = c < nc ? idx[c * n_l + j] : 0;
}

cudaError_t launch_pack_idx(int64_t nc, int n_l, const int32_t *idx, int32_t *is, cudaStream_t st) {
    int64_t tot = ((nc + 31) & ~31LL) * n_l;
    if (tot == 0) return cudaSuccess;
    k_pack_idx<<<(unsigned)((tot + 255) / 256), 256, 0, st>>>(nc, n_l, idx, is);
    return cudaGetLastError();
}

// wall normal-derivative weights w^n_j = n_x w^x_j + n_y w^y_j + n_z w^z_j (FP64),
// from the gradient weights of the wall nodes' Neumann stencils
template <typename T>
__global__ void k_pack_normal(int64_t nb, int n_l, const int32_t *__restrict__ wall, const double *__restrict__ nrm,
                              const double *__restrict__ wg, T *ws) {
    int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    int64_t npad = (nb + 31) & ~31LL;
    if (t >= npad * n_l) return;
    int64_t b = t / n_l;
    int j = (int)(t - b * n_l);
    T v = (T)0;
    if (b < nb) {
        int64_t i = wall[b];
        const double *g = wg + b * 3 * n_l;
        double nx = nrm[3 * i], ny = nrm[3 * i + 1], nz = nrm[3 * i + 2];
        v = (T)(__dadd_rn(__dadd_rn(__dmul_rn(nx, g[j]), __dmul_rn(ny, g[n_l + j])), __dmul_rn(nz, g[2 * n_l + j])));
    }
    ws[sell_at(b >> 5, 0, j, (int)(b & 31), 1, n_l)] = v;
}

cudaError_t launch_pack_normal_f32(int64_t nb, int n_l, const int32_t *wall, const double *nrm,
                                   const double *wg, float *ws, cudaStream_t st) {
    int64_t tot = ((nb + 31) & ~31LL) * n_l;
    if (tot == 0) return cudaSuccess;
    k_pack_normal<float><<<(unsigned)((tot + 255) / 256), 256, 0, st>>>(nb, n_l, wall, nrm, wg, ws);
    return cudaGetLastError();
}
cudaError_t launch_pack_normal_f64(int64_t nb, int n_l, const int32_t *wall, const double *nrm,
                                   const double *wg, double *ws, cudaStream_t st) {
    int64_t tot = ((nb + 31) & ~31LL) * n_l;
    if (tot == 0) return cudaSuccess;
    k_pack_normal<double><<<(unsigned)((tot + 255) / 256), 256, 0, st>>>(nb, n_l, wall, nrm, wg, ws);
    return cudaGetLastError();
}

}  // namespace rbf
