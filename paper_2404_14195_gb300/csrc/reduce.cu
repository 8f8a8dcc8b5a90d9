// reduce.cu — FP64 reductions and field marshalling.
//
//  * residual: |v - v_prev|_2 / |v|_2 over fluid nodes;
//  * permeability (Eq. k_definition): probe interpolation of v_x and its mean;
//  * drag (Eqs. stress_tensor_force, integration_force): sigma . n summed over
//    wall nodes with the wall nodes' gradient weights;
//  * min / sum helpers.
// Every reduction writes one FP64 partial per block and a single block adds the
// partials in a fixed order, so results are reproducible run to run.
#include "reduce.cuh"

namespace rbf {

__device__ __forceinline__ double warp_sum(double v) {
    for (int off = 16; off > 0; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
    return v;
}

// block sum of ncomp values per thread into partial[blockIdx.x * ncomp + c]
template <int NC>
__device__ __forceinline__ void block_partial(double (&v)[NC], double *partial) {
    __shared__ double red[8][NC];
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
#pragma unroll
    for (int c = 0; c < NC; ++c) v[c] = warp_sum(v[c]);
    if (lane == 0)
#pragma unroll
        for (int c = 0; c < NC; ++c) red[w][c] = v[c];
    __syncthreads();
    if (threadIdx.x < NC) {
        double s = 0.0;
        for (int t = 0; t < (int)(blockDim.x >> 5); ++t) s += red[t][threadIdx.x];
        partial[blockIdx.x * NC + threadIdx.x] = s;
    }
}

__global__ void k_final_sum(const double *partial, int64_t nb, int nc, double *out) {
    // one warp per component, strided over blocks, fixed order
    const int c = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (c >= nc) return;
    double s = 0.0;
    for (int64_t b = lane; b < nb; b += 32) s += partial[b * nc + c];
    s = warp_sum(s);
    if (lane == 0) out[c] = s;
}

static cudaError_t final_sum(const double *partial, int64_t nb, int nc, double *out, cudaStream_t st) {
    k_final_sum<<<1, 32 * nc, 0, st>>>(partial, nb, nc, out);
    return cudaGetLastError();
}

template <typename T>
__global__ void __launch_bounds__(256) k_residual(int64_t n, const uint8_t *type, const T *u, const T *v, const T *w,
                                                  const T *uo, const T *vo, const T *wo, double *partial) {
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    double acc[2] = {0.0, 0.0};
    if (i < n && !type[i]) {
        double a = (double)u[i] - (double)uo[i], b = (double)v[i] - (double)vo[i], c = (double)w[i] - (double)wo[i];
        acc[0] = a * a + b * b + c * c;
        acc[1] = (double)u[i] * u[i] + (double)v[i] * v[i] + (double)w[i] * w[i];
    }
    block_partial<2>(acc, partial);
}

template <typename T>
cudaError_t launch_residual(int64_t n, const uint8_t *type, const T *u, const T *v, const T *w, const T *uo,
                            const T *vo, const T *wo, double *partial, double *out2, cudaStream_t st) {
    int64_t nb = (n + 255) / 256;
    k_residual<T><<<(unsigned)nb, 256, 0, st>>>(n, type, u, v, w, uo, vo, wo, partial);
    return final_sum(partial, nb, 2, out2, st);
}

// probe interpolation: out_sum = sum_p sum_j w_pj vx[S_p(j)]  (vx + vxl for a
// compensated state)
template <typename T>
__global__ void __launch_bounds__(256) k_probe_sum(int64_t np, int n_l, const int32_t *idx, const double *w,
                                                   const T *vx, const T *vxl, int64_t stride, double *partial) {
    int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    double acc[1] = {0.0};
    if (p < np) {
        double s = 0.0;
        for (int j = 0; j < n_l; ++j) {
            const int64_t q = idx[p * n_l + j] * stride;
            const double v = vxl ? (double)vx[q] + (double)vxl[q] : (double)vx[q];
            s += w[p * n_l + j] * v;
        }
        acc[0] = s;
    }
    block_partial<1>(acc, partial);
}

template <typename T>
cudaError_t launch_probe_sum(int64_t np, int n_l, const int32_t *idx, const double *w, const T *vx, const T *vxl,
                             int64_t stride, double *partial, double *out, cudaStream_t st) {
    if (np == 0) return cudaMemsetAsync(out, 0, sizeof(double), st);
    int64_t nb = (np + 255) / 256;
    k_probe_sum<T><<<(unsigned)nb, 256, 0, st>>>(np, n_l, idx, w, vx, vxl, stride, partial);
    return final_sum(partial, nb, 1, out, st);
}

// sigma . n at wall nodes: sigma_ij = -p d_ij + rho nu (d_j v_i + d_i v_j).
// Velocity components and pressure are read through (pointer, stride) views and
// scaled to physical units: v = vs * vel, p = (praw - p0) * ps.  Per wall node the
// kernel adds (sigma . n, p, n): the host turns the sums into the force with the
// wall-mean pressure removed, F = sum sigma . n + pbar sum n, so that a constant
// pressure contributes nothing (the exact surface integral of a constant is zero;
// the equal-weight quadrature over scattered wall nodes is not).
template <typename T>
__global__ void __launch_bounds__(256) k_drag(int64_t nb, int n_l, const int32_t *wall, const int32_t *idx,
                                              const double *wg, const double *nrm, FieldView<T> f, double mu,
                                              double *partial) {
    int64_t b = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    double acc[7] = {0.0, 0.0, 0.0, 0.0, 0.0, 0.0, 0.0};
    if (b < nb) {
        int64_t i = wall[b];
        double G[3][3] = {{0, 0, 0}, {0, 0, 0}, {0, 0, 0}};  // G[comp][dir] = d v_comp / d x_dir
        const double *gx = wg + b * 3 * n_l, *gy = gx + n_l, *gz = gy + n_l;
        for (int j = 0; j < n_l; ++j) {
            const int64_t q = idx[i * n_l + j] * f.stride;
            double vq[3] = {(double)f.u[q], (double)f.v[q], (double)f.w[q]};
            if (f.ul) { vq[0] += (double)f.ul[q]; vq[1] += (double)f.vl[q]; vq[2] += (double)f.wl[q]; }
            vq[0] *= f.vel; vq[1] *= f.vel; vq[2] *= f.vel;
            for (int c = 0; c < 3; ++c) {
                G[c][0] += gx[j] * vq[c];
                G[c][1] += gy[j] * vq[c];
                G[c][2] += gz[j] * vq[c];
            }
        }
        double praw = (double)f.p[i * f.stride];
        if (f.pl) praw += (double)f.pl[i * f.stride];
        double p = (praw - f.p0) * f.ps;
        double n3[3] = {nrm[3 * i], nrm[3 * i + 1], nrm[3 * i + 2]};
        for (int a = 0; a < 3; ++a) {
            double s = -p * n3[a];
            for (int c = 0; c < 3; ++c) s += mu * (G[a][c] + G[c][a]) * n3[c];
            acc[a] = s;
        }
        acc[3] = p;
        acc[4] = n3[0]; acc[5] = n3[1]; acc[6] = n3[2];
    }
    block_partial<7>(acc, partial);
}

template <typename T>
cudaError_t launch_drag(int64_t nb, int n_l, const int32_t *wall, const int32_t *idx, const double *wg,
                        const double *nrm, const FieldView<T> &f, double mu, double *partial, double *out7,
                        cudaStream_t st) {
    if (nb == 0) return cudaMemsetAsync(out7, 0, 7 * sizeof(double), st);
    int64_t nbl = (nb + 255) / 256;
    k_drag<T><<<(unsigned)nbl, 256, 0, st>>>(nb, n_l, wall, idx, wg, nrm, f, mu, partial);
    return final_sum(partial, nbl, 7, out7, st);
}

__global__ void k_min(const double *in, int64_t n, double *partial) {
    __shared__ double red[8];
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    double v = i < n ? in[i] : __longlong_as_double(0x7ff0000000000000LL);
    for (int off = 16; off > 0; off >>= 1) v = fmin(v, __shfl_xor_sync(0xffffffffu, v, off));
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
    __syncthreads();
    if (threadIdx.x == 0) {
        double m = red[0];
        for (int t = 1; t < (int)(blockDim.x >> 5); ++t) m = fmin(m, red[t]);
        partial[blockIdx.x] = m;
    }
}
__global__ void k_min_final(const double *partial, int64_t nb, double *out) {
    double v = __longlong_as_double(0x7ff0000000000000LL);
    for (int64_t b = threadIdx.x; b < nb; b += 32) v = fmin(v, partial[b]);
    for (int off = 16; off > 0; off >>= 1) v = fmin(v, __shfl_xor_sync(0xffffffffu, v, off));
    if (threadIdx.x == 0) *out = v;
}
cudaError_t launch_min_f64(const double *in, int64_t n, double *partial, double *out, cudaStream_t st) {
    int64_t nb = (n + 255) / 256;
    k_min<<<(unsigned)nb, 256, 0, st>>>(in, n, partial);
    k_min_final<<<1, 32, 0, st>>>(partial, nb, out);
    return cudaGetLastError();
}

// sum of in[i * stride + c] for c < ncomp (ncomp <= 4)
__global__ void k_sum_strided(const double *in, int64_t n, int stride, int ncomp, double *partial) {
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    double acc[4] = {0, 0, 0, 0};
    if (i < n)
        for (int c = 0; c < ncomp; ++c) acc[c] = in[i * stride + c];
    block_partial<4>(acc, partial);
}
cudaError_t launch_sum_f64(const double *in, int64_t n, int stride, int ncomp, double *partial, double *out,
                           cudaStream_t st) {
    int64_t nb = (n + 255) / 256;
    k_sum_strided<<<(unsigned)nb, 256, 0, st>>>(in, n, stride, ncomp, partial);
    return final_sum(partial, nb, 4, out, st);
}

// ---- ACM fields <-> caller order, FP64 ---------------------------------------
template <typename T>
__global__ void k_acm_export(int64_t n, const int32_t *perm, const T *u, const T *v, const T *w, const T *p,
                             double *out) {
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n) return;
    int64_t o = perm[i];
    out[4 * o] = (double)u[i]; out[4 * o + 1] = (double)v[i]; out[4 * o + 2] = (double)w[i]; out[4 * o + 3] = (double)p[i];
}
template <typename T>
__global__ void k_acm_import(int64_t n, const int32_t *perm, T *u, T *v, T *w, T *p, const double *in) {
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n) return;
    int64_t o = perm[i];
    u[i] = (T)in[4 * o]; v[i] = (T)in[4 * o + 1]; w[i] = (T)in[4 * o + 2]; p[i] = (T)in[4 * o + 3];
}
template <typename T>
cudaError_t launch_acm_export(int64_t n, const int32_t *perm, const T *u, const T *v, const T *w, const T *p,
                              double *out, cudaStream_t st) {
    k_acm_export<T><<<(unsigned)((n + 255) / 256), 256, 0, st>>>(n, perm, u, v, w, p, out);
    return cudaGetLastError();
}
template <typename T>
cudaError_t launch_acm_import(int64_t n, const int32_t *perm, T *u, T *v, T *w, T *p, const double *in,
                              cudaStream_t st) {
    k_acm_import<T><<<(unsigned)((n + 255) / 256), 256, 0, st>>>(n, perm, u, v, w, p, in);
    return cudaGetLastError();
}

__global__ void k_acm_export_pair(int64_t n, const int32_t *perm, const float *u, const float *v, const float *w,
                                  const float *p, const float *ul, const float *vl, const float *wl, const float *pl,
                                  double *out) {
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n) return;
    int64_t o = perm[i];
    out[4 * o] = (double)u[i] + (double)ul[i];
    out[4 * o + 1] = (double)v[i] + (double)vl[i];
    out[4 * o + 2] = (double)w[i] + (double)wl[i];
    out[4 * o + 3] = (double)p[i] + (double)pl[i];
}
__device__ __forceinline__ void split_pair(double x, float *hi, float *lo, int64_t i) {
    const float h = (float)x;
    hi[i] = h;
    lo[i] = (float)(x - (double)h);
}
__global__ void k_acm_import_pair(int64_t n, const int32_t *perm, float *u, float *v, float *w, float *p, float *ul,
                                  float *vl, float *wl, float *pl, const double *in) {
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n) return;
    int64_t o = perm[i];
    split_pair(in[4 * o], u, ul, i);
    split_pair(in[4 * o + 1], v, vl, i);
    split_pair(in[4 * o + 2], w, wl, i);
    split_pair(in[4 * o + 3], p, pl, i);
}
cudaError_t launch_acm_export_pair(int64_t n, const int32_t *perm, const float *u, const float *v, const float *w,
                                   const float *p, const float *ul, const float *vl, const float *wl,
                                   const float *pl, double *out, cudaStream_t st) {
    k_acm_export_pair<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(n, perm, u, v, w, p, ul, vl, wl, pl, out);
    return cudaGetLastError();
}
cudaError_t launch_acm_import_pair(int64_t n, const int32_t *perm, float *u, float *v, float *w, float *p,
                                   float *ul, float *vl, float *wl, float *pl, const double *in, cudaStream_t st) {
    k_acm_import_pair<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(n, perm, u, v, w, p, ul, vl, wl, pl, in);
    return cudaGetLastError();
}

// Velocity of a context in physical units, scattered to the caller's node order:
// out[3 perm[i] + c] = scale (v_c[i stride] + lo_c[i]), lo null for a plain state.
template <typename T>
__global__ void k_velocity(int64_t n, const int32_t *perm, const T *u, const T *v, const T *w, const T *ul,
                           const T *vl, const T *wl, int64_t stride, double scale, double *out) {
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n) return;
    double x = (double)u[i * stride], y = (double)v[i * stride], z = (double)w[i * stride];
    if (ul) {
        x += (double)ul[i];
        y += (double)vl[i];
        z += (double)wl[i];
    }
    const int64_t o = 3 * (int64_t)perm[i];
    out[o] = scale * x;
    out[o + 1] = scale * y;
    out[o + 2] = scale * z;
}
template <typename T>
cudaError_t launch_velocity(int64_t n, const int32_t *perm, const T *u, const T *v, const T *w, const T *ul,
                            const T *vl, const T *wl, int64_t stride, double scale, double *out, cudaStream_t st) {
    if (n == 0) return cudaSuccess;
    k_velocity<T><<<(unsigned)((n + 255) / 256), 256, 0, st>>>(n, perm, u, v, w, ul, vl, wl, stride, scale, out);
    return cudaGetLastError();
}

// Eq. pointwise_error on [n][3] velocity fields in one node order:
// dv = |v_a - v_b|_2, delta = dv / |v_b|_2 (NaN where v_b = 0)
__global__ void k_pointwise(int64_t n, const double *va, const double *vb, double *delta, double *dv) {
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n) return;
    const double bx = vb[3 * i], by = vb[3 * i + 1], bz = vb[3 * i + 2];
    const double x = va[3 * i] - bx, y = va[3 * i + 1] - by, z = va[3 * i + 2] - bz;
    const double d = sqrt(x * x + y * y + z * z);
    const double nb = sqrt(bx * bx + by * by + bz * bz);
    dv[i] = d;
    delta[i] = nb > 0.0 ? d / nb : __longlong_as_double(0x7ff8000000000000LL);
}
cudaError_t launch_pointwise(int64_t n, const double *va, const double *vb, double *delta, double *dv,
                             cudaStream_t st) {
    if (n == 0) return cudaSuccess;
    k_pointwise<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(n, va, vb, delta, dv);
    return cudaGetLastError();
}

// LBM macro buffer (sorted, lattice units, (vx, vy, vz, rho - 1)) -> physical uvwp,
// caller order; p = ps c_s^2 (rho - <rho>) / <rho> (pressure relative to the mean
// density, in units of it)
__global__ void k_lbm_fields(int64_t n, const int32_t *perm, const double *mac, double vel, double ps,
                             const double *drho_sum, double *out) {
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n) return;
    int64_t o = perm[i];
    double mean = drho_sum[0] / (double)n;
    out[4 * o] = mac[4 * i] * vel;
    out[4 * o + 1] = mac[4 * i + 1] * vel;
    out[4 * o + 2] = mac[4 * i + 2] * vel;
    out[4 * o + 3] = (mac[4 * i + 3] - mean) / (1.0 + mean) * (1.0 / 3.0) * ps;
}
cudaError_t launch_lbm_fields(int64_t n, const int32_t *perm, const double *mac, double vel, double ps,
                              const double *drho_sum, double *out, cudaStream_t st) {
    k_lbm_fields<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(n, perm, mac, vel, ps, drho_sum, out);
    return cudaGetLastError();
}

// non-finite detector: sets *flag when any value is NaN/Inf
template <typename T>
__global__ void k_nonfinite(const T *a, int64_t n, int32_t *flag) {
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i < n && !isfinite((double)a[i])) atomicExch(flag, 1);
}
template <typename T>
cudaError_t launch_nonfinite(const T *a, int64_t n, int32_t *flag, cudaStream_t st) {
    if (n <= 0) return cudaSuccess;
    k_nonfinite<T><<<(unsigned)((n + 255) / 256), 256, 0, st>>>(a, n, flag);
    return cudaGetLastError();
}

// caller-order gathers for rbf_get_stencils / rbf_get_weights
__global__ void k_export_stencils(int64_t n, int n_l, const int32_t *perm, const int32_t *iperm,
                                  const int32_t *idx, int32_t *out) {
    int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (t >= n * n_l) return;
    int64_t o = t / n_l;
    int j = (int)(t - o * n_l);
    out[t] = perm[idx[(int64_t)iperm[o] * n_l + j]];
}
cudaError_t launch_export_stencils(int64_t n, int n_l, const int32_t *perm, const int32_t *iperm,
                                   const int32_t *idx, int32_t *out, cudaStream_t st) {
    int64_t tot = n * n_l;
    k_export_stencils<<<(unsigned)((tot + 255) / 256), 256, 0, st>>>(n, n_l, perm, iperm, idx, out);
    return cudaGetLastError();
}
// rows of w (sorted row r = node, n_ops operators) for operator op -> out[caller][j];
// rowmap (optional): caller node -> row (-1: no row, output NaN)
__global__ void k_export_weights(int64_t n, int n_l, int n_ops, int op, const int32_t *iperm, const int32_t *rowmap,
                                 const double *w, double *out) {
    int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (t >= n * n_l) return;
    int64_t o = t / n_l;
    int j = (int)(t - o * n_l);
    int64_t r = iperm[o];
    if (rowmap) r = rowmap[r];
    out[t] = r < 0 ? __longlong_as_double(0x7ff8000000000000LL) : w[(r * n_ops + op) * n_l + j];
}
cudaError_t launch_export_weights(int64_t n, int n_l, int n_ops, int op, const int32_t *iperm, const int32_t *rowmap,
                                  const double *w, double *out, cudaStream_t st) {
    int64_t tot = n * n_l;
    k_export_weights<<<(unsigned)((tot + 255) / 256), 256, 0, st>>>(n, n_l, n_ops, op, iperm, rowmap, w, out);
    return cudaGetLastError();
}

#define RBF_RED_INST(T)                                                                                         \
    template cudaError_t launch_residual<T>(int64_t, const uint8_t *, const T *, const T *, const T *, const T *, \
                                            const T *, const T *, double *, double *, cudaStream_t);            \
    template cudaError_t launch_probe_sum<T>(int64_t, int, const int32_t *, const double *, const T *, const T *, \
                                             int64_t, double *, double *, cudaStream_t);                        \
    template cudaError_t launch_drag<T>(int64_t, int, const int32_t *, const int32_t *, const double *,          \
                                        const double *, const FieldView<T> &, double, double *, double *,       \
                                        cudaStream_t);                                                          \
    template cudaError_t launch_acm_export<T>(int64_t, const int32_t *, const T *, const T *, const T *,         \
                                              const T *, double *, cudaStream_t);                               \
    template cudaError_t launch_acm_import<T>(int64_t, const int32_t *, T *, T *, T *, T *, const double *,      \
                                              cudaStream_t);                                                    \
    template cudaError_t launch_nonfinite<T>(const T *, int64_t, int32_t *, cudaStream_t);                    \
    template cudaError_t launch_velocity<T>(int64_t, const int32_t *, const T *, const T *, const T *, const T *, \
                                            const T *, const T *, int64_t, double, double *, cudaStream_t);
RBF_RED_INST(float)
RBF_RED_INST(double)

}  // namespace rbf
