// mlp.cu — the learned warm start: a Fourier-feature MLP (64 -> 128 x 4 GELU -> 16)
// trained and evaluated with hand-written BF16 tensor-core (tcgen05) GEMMs, FP32
// accumulation in tensor memory, fused epilogues, and Adam on FP32 master weights.
//
// Every layer is C = A B^T with both operands K-major BF16 (row-major with the
// reduction index contiguous):
//   forward   Z_l = H_{l-1} W_l^T           (A = activations [B][in], B = W_l [out][in])
//   backward  dH_{l-1} = dZ_l W_l           (A = dZ_l [B][out],  B = W_l^T [in][out])
//             dW_l = dZ_l^T H_{l-1}         (A = dZ_l^T [out][B], B = H_{l-1}^T [in][B]),
//             split over the batch, partials reduced in FP32
// so the epilogues also write the transposed copies the weight-gradient GEMMs
// read, and the optimizer writes W and W^T in BF16.  The network is not in the
// paper; it implements the build's warm-start design (features of position,
// radius and wall distance -> (u, v, w, p)).
#include <cuda_bf16.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <string>
#include <vector>

#include "acm.cuh"
#include "ctx.cuh"
#include "rbfgb.h"
#include "tc.cuh"

using namespace rbf;
typedef __nv_bfloat16 bf16;

namespace {

constexpr int N_IN = 64, N_H = 128, N_OUT = 4, N_OUT_PAD = 16, N_LAYERS = 5;
__host__ __device__ constexpr int fan_in(int l) { return l == 0 ? N_IN : N_H; }
__host__ __device__ constexpr int fan_out(int l) { return l == N_LAYERS - 1 ? N_OUT_PAD : N_H; }

int64_t w_off(int l) {  // offset of W_l in the packed parameter vector
    int64_t o = 0;
    for (int i = 0; i < l; ++i) o += (int64_t)fan_out(i) * fan_in(i) + fan_out(i);
    return o;
}
int64_t b_off(int l) { return w_off(l) + (int64_t)fan_out(l) * fan_in(l); }
int64_t n_params_total() { return w_off(N_LAYERS); }
__host__ __device__ constexpr int64_t w_off_c(int l) {  // w_off / b_off usable in device code
    return l == 0 ? 0 : w_off_c(l - 1) + (int64_t)fan_out(l - 1) * fan_in(l - 1) + fan_out(l - 1);
}
__host__ __device__ constexpr int64_t b_off_c(int l) { return w_off_c(l) + (int64_t)fan_out(l) * fan_in(l); }

// element offset of (r, k) in a K-major no-swizzle core-matrix operand with K columns:
// 8 x 8 blocks of 128 bytes, adjacent along K (LBO = 128 B), row groups 16 K bytes apart
__device__ __forceinline__ int cmo(int r, int k, int K) { return (((r >> 3) * (K >> 3) + (k >> 3)) << 6) + ((r & 7) << 3) + (k & 7); }

// ---- tcgen05 GEMM -------------------------------------------------------------------
enum { EP_F32 = 0, EP_FWD = 1, EP_OUT = 2, EP_BWD = 3, EP_PRED = 4 };

struct GemmArgs {
    const bf16 *A;
    int lda;
    const bf16 *B;
    int ldb;
    int M, N, K;          // M multiple of 128; N in {16, 32, 64, 128}; K multiple of 16, split by gridDim.y
    // epilogue operands
    float *out32;         // EP_F32: partials [split][M][N]; EP_PRED: [M][4]
    const float *bias;    // N
    bf16 *H, *Ht, *G;     // EP_FWD / EP_OUT / EP_BWD outputs (row-major [M][N], transposed [N][ldt], G [M][N])
    int ldt;
    const float *T;       // EP_OUT targets [M][4]
    float *loss, *db;     // accumulators
    const bf16 *Gin;      // EP_BWD: GELU'(Z) of the layer below, [M][N]
    int nvalid;
    float gscale;
    int32_t *err;
};

constexpr int SMEM_A = 16384, SMEM_B = 16384;
constexpr size_t GEMM_SMEM = 57344;  // also caps residency at 3-4 CTAs per SM (<= 512 TMEM columns)
constexpr uint64_t WAIT_NS = 1000000000ull;

// GELU in its tanh form, h = z (1 + tanh u) / 2 with u = sqrt(2/pi) (z + 0.044715 z^3),
// evaluated through the identity (1 + tanh u) / 2 = s = 1 / (1 + 2^a), a = -2u log2(e):
// one hardware base-2 exponential and one hardware reciprocal (PTX ex2.approx and
// rcp.approx, a few ulp; ~1e-6 against the tanh form, far below the BF16 resolution h is
// stored at) instead of a full-precision tanhf.  The derivative follows from
// 1 - tanh^2 u = 4 s (1 - s):
//   h' = s + 2 z s (1 - s) u' = s + h (1 - s) 2u',  2u' = 2 sqrt(2/pi) (1 + 3 * 0.044715 z^2).
// a is clamped at 126 so that 1 + 2^a stays finite (s >= 2^-126 there instead of ~0).
__device__ __forceinline__ float ex2_approx(float x) {
    float y;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}
__device__ __forceinline__ float rcp_approx(float x) {
    float y;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}
// GELU h and its derivative g from one exponential
__device__ __forceinline__ void gelu_both(float z, float &h, float &g) {
    const float zz = z * z;
    const float a = fminf(z * fmaf(0.044715f, zz, 1.0f) * -2.302208198144325f, 126.0f);
    const float s = rcp_approx(1.0f + ex2_approx(a));
    h = z * s;
    g = fmaf(h * (1.0f - s), fmaf(0.21406444881780073f, zz, 1.5957691216057308f), s);
}
__device__ __forceinline__ float gelu_f(float z) {
    float h, g;
    gelu_both(z, h, g);
    return h;
}
__device__ __forceinline__ float gelu_prime_f(float z) {
    float h, g;
    gelu_both(z, h, g);
    return g;
}

// copy rows [r0, r0 + nrows) x cols [k0, k0 + kw) of a K-major BF16 matrix into the
// no-swizzle core-matrix layout: element (r, k) at (r/8)*1024 + (k/8)*128 + (r%8)*16 + (k%8)*2
__device__ __forceinline__ void stage_tile(uint8_t *dst, const bf16 *src, int ld, int r0, int nrows, int k0, int kw) {
    const int kp_n = kw >> 3;
    for (int p = threadIdx.x; p < nrows * kp_n; p += blockDim.x) {
        const int r = p / kp_n, kp = p - r * kp_n;
        const uint4 v = *reinterpret_cast<const uint4 *>(src + (int64_t)(r0 + r) * ld + k0 + kp * 8);
        *reinterpret_cast<uint4 *>(dst + (r >> 3) * 1024 + kp * 128 + (r & 7) * 16) = v;
    }
}

template <int EP>
__global__ void __launch_bounds__(128) k_gemm(GemmArgs g) {
    extern __shared__ __align__(1024) uint8_t smem[];
    uint8_t *sA = smem;
    uint8_t *sB = smem + SMEM_A;
    uint64_t *bar = reinterpret_cast<uint64_t *>(smem + SMEM_A + SMEM_B);
    uint32_t *slot = reinterpret_cast<uint32_t *>(smem + SMEM_A + SMEM_B + 8);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int m0 = blockIdx.x * 128;
    const int kid = blockIdx.y, ksplit = gridDim.y;
    const int Kper = g.K / ksplit, k_lo = kid * Kper;
    const int N = g.N;
    const uint32_t ncols = N <= 32 ? 32u : (N <= 64 ? 64u : 128u);
    if (warp == 0) {
        tc::tmem_alloc(slot, ncols);
        tc::tmem_relinquish();
    }
    if (tid == 0) tc::mbar_init(bar, 1);
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    const uint32_t tmem = *slot;
    const uint32_t idesc = tc::idesc_bf16_f32(128, N);
    uint32_t phase = 0;
    bool ok = true;
    for (int kc = 0; kc < Kper && ok; kc += 64) {
        const int kw = min(64, Kper - kc);
        stage_tile(sA, g.A, g.lda, m0, 128, k_lo + kc, kw);
        stage_tile(sB, g.B, g.ldb, 0, N, k_lo + kc, kw);
        tc::fence_proxy_async_smem();
        __syncthreads();
        if (tid == 0) {
            tc::fence_after_sync();
            for (int kk = 0; kk < (kw >> 4); ++kk) {
                const uint64_t da = tc::smem_desc(sA + kk * 256, 128, 1024);
                const uint64_t db = tc::smem_desc(sB + kk * 256, 128, 1024);
                tc::mma_bf16(tmem, da, db, idesc, (kc > 0 || kk > 0) ? 1u : 0u);
            }
            tc::mma_commit(bar);
        }
        ok = tc::mbar_wait(bar, phase, WAIT_NS);
        phase ^= 1;
        __syncthreads();
    }
    if (!ok) {  // the MMAs did not complete in time: report, give them one more bounded wait, free TMEM
        if (tid == 0) atomicExch(g.err, 1);
        tc::mbar_wait(bar, phase ^ 1, WAIT_NS);
        tc::fence_before_sync();
        __syncthreads();
        if (warp == 0) tc::tmem_dealloc(tmem, ncols);
        return;
    }
    tc::fence_after_sync();
    const int m = m0 + warp * 32 + lane;
    const bool valid = m < g.nvalid;
    float lsum = 0.0f;
    for (int c0 = 0; c0 < N; c0 += 16) {
        float v[16];
        tc::tmem_ld16(tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)c0, v);
        if (EP == EP_F32) {
            float *o = g.out32 + ((int64_t)kid * g.M + m) * N + c0;
#pragma unroll
            for (int i = 0; i < 16; i += 4) *reinterpret_cast<float4 *>(o + i) = make_float4(v[i], v[i + 1], v[i + 2], v[i + 3]);
        } else if (EP == EP_PRED) {
            if (c0 == 0 && valid)
#pragma unroll
                for (int i = 0; i < N_OUT; ++i) g.out32[(int64_t)m * N_OUT + i] = v[i] + g.bias[i];
        } else {
            __align__(16) bf16 hv[16];
            __align__(16) bf16 gv[16];
            float colv[16];
#pragma unroll
            for (int i = 0; i < 16; ++i) {
                const int c = c0 + i;
                float h, gp = 0.0f;
                if (EP == EP_FWD) {
                    const float z = v[i] + g.bias[c];
                    gelu_both(z, h, gp);
                } else if (EP == EP_OUT) {
                    const float y = v[i] + g.bias[c];
                    float dy = 0.0f;
                    if (c < N_OUT && valid) {
                        const float e = y - g.T[(int64_t)m * N_OUT + c];
                        lsum += e * e;
                        dy = g.gscale * e;
                    }
                    h = dy;
                } else {  // EP_BWD
                    h = valid ? v[i] * __bfloat162float(g.Gin[(int64_t)m * N + c]) : 0.0f;
                }
                hv[i] = __float2bfloat16(h);
                gv[i] = __float2bfloat16(gp);
                colv[i] = __bfloat162float(hv[i]);
            }
            if (g.H) {
                uint4 *dst = reinterpret_cast<uint4 *>(g.H + (int64_t)m * N + c0);
                dst[0] = reinterpret_cast<uint4 *>(hv)[0];
                dst[1] = reinterpret_cast<uint4 *>(hv)[1];
            }
            if (g.G) {
                uint4 *dst = reinterpret_cast<uint4 *>(g.G + (int64_t)m * N + c0);
                dst[0] = reinterpret_cast<uint4 *>(gv)[0];
                dst[1] = reinterpret_cast<uint4 *>(gv)[1];
            }
            if (g.Ht)
#pragma unroll
                for (int i = 0; i < 16; ++i) g.Ht[(int64_t)(c0 + i) * g.ldt + m] = hv[i];
            if (g.db && (EP == EP_OUT || EP == EP_BWD)) {  // bias gradient: column sums over the tile's rows
#pragma unroll
                for (int i = 0; i < 16; ++i) {
                    float s = colv[i];
                    for (int off = 16; off > 0; off >>= 1) s += __shfl_xor_sync(0xffffffffu, s, off);
                    if (lane == 0 && s != 0.0f) atomicAdd(g.db + c0 + i, s);
                }
            }
        }
    }
    if (EP == EP_OUT && g.loss) {
        for (int off = 16; off > 0; off >>= 1) lsum += __shfl_xor_sync(0xffffffffu, lsum, off);
        if (lane == 0) atomicAdd(g.loss, lsum);
    }
    tc::fence_before_sync();
    __syncthreads();
    if (warp == 0) tc::tmem_dealloc(tmem, ncols);
}

cudaError_t launch_gemm(int ep, const GemmArgs &g, int ksplit, cudaStream_t st) {
    if (g.M % 128 || g.K % 16 || (g.K / ksplit) % 16 || g.K % ksplit || !(g.N == 16 || g.N == 32 || g.N == 64 || g.N == 128))
        return cudaErrorInvalidValue;
    dim3 grid(g.M / 128, ksplit);
    switch (ep) {
    case EP_F32: k_gemm<EP_F32><<<grid, 128, GEMM_SMEM, st>>>(g); break;
    case EP_FWD: k_gemm<EP_FWD><<<grid, 128, GEMM_SMEM, st>>>(g); break;
    case EP_OUT: k_gemm<EP_OUT><<<grid, 128, GEMM_SMEM, st>>>(g); break;
    case EP_BWD: k_gemm<EP_BWD><<<grid, 128, GEMM_SMEM, st>>>(g); break;
    case EP_PRED: k_gemm<EP_PRED><<<grid, 128, GEMM_SMEM, st>>>(g); break;
    default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

cudaError_t gemm_set_smem() {
    cudaError_t e = cudaSuccess;
    for (auto f : {k_gemm<EP_F32>, k_gemm<EP_FWD>, k_gemm<EP_OUT>, k_gemm<EP_BWD>, k_gemm<EP_PRED>}) {
        e = cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)GEMM_SMEM);
        if (e != cudaSuccess) return e;
    }
    return e;
}

// ---- features, targets, reductions, optimizer ------------------------------------------
__constant__ int c_waves[16][3] = {{1, 0, 0},  {0, 1, 0},  {0, 0, 1},  {1, 1, 0},   {1, -1, 0}, {1, 0, 1},
                                   {1, 0, -1}, {0, 1, 1},  {0, 1, -1}, {1, 1, 1},   {1, 1, -1}, {1, -1, 1},
                                   {1, -1, -1}, {2, 0, 0}, {0, 2, 0},  {0, 0, 2}};

__device__ __forceinline__ uint64_t splitmix64(uint64_t x) {
    uint64_t z = x + 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

// Rows b < B of X [B][64] and X^T [64][ldt]: sample s = explicit index, or the
// counter-based draw splitmix64(seed * 2^32 + step * B + b) mod n (step read from
// *step_dev so a captured graph draws a new batch each replay); targets into T.
__global__ void k_features(int B, int64_t n, const double *__restrict__ xyz, const float *__restrict__ rad,
                           const float *__restrict__ sdf, const float *__restrict__ tgt, const int64_t *__restrict__ idx,
                           uint64_t seed, const int64_t *step_dev, bf16 *X, bf16 *Xt, int ldt, float *T) {
    const int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= B) return;
    int64_t s;
    if (idx) s = idx[b];
    else {
        const uint64_t c = seed * (1ull << 32) + (uint64_t)(*step_dev) * (uint64_t)B + (uint64_t)b;
        s = (int64_t)(splitmix64(c) % (uint64_t)n);
    }
    const double x = xyz[3 * s], y = xyz[3 * s + 1], z = xyz[3 * s + 2];
    __align__(16) bf16 row[N_IN];
#pragma unroll
    for (int j = 0; j < 16; ++j) {
        double sn, cs;
        sincospi(2.0 * (c_waves[j][0] * x + c_waves[j][1] * y + c_waves[j][2] * z), &sn, &cs);
        row[2 * j] = __double2bfloat16(sn);
        row[2 * j + 1] = __double2bfloat16(cs);
    }
    row[32] = __float2bfloat16(rad[s]);
    row[33] = __float2bfloat16(sdf[s]);
#pragma unroll
    for (int j = 34; j < N_IN; ++j) row[j] = __float2bfloat16(0.0f);
    uint4 *dst = reinterpret_cast<uint4 *>(X + (int64_t)b * N_IN);
#pragma unroll
    for (int j = 0; j < N_IN / 8; ++j) dst[j] = reinterpret_cast<uint4 *>(row)[j];
    if (Xt)
#pragma unroll
        for (int j = 0; j < N_IN; ++j) Xt[(int64_t)j * ldt + b] = row[j];
    if (T && tgt)
#pragma unroll
        for (int c = 0; c < N_OUT; ++c) T[(int64_t)b * N_OUT + c] = tgt[s * N_OUT + c];
}

// out[m][n] (or out[n][m] when transposed) = sum over splits of part[k][m][n]
__global__ void k_reduce_splits(const float *__restrict__ part, int ksplit, int M, int N, float *out, int transposed) {
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= M * N) return;
    float s = 0.0f;
    for (int k = 0; k < ksplit; ++k) s += part[(int64_t)k * M * N + t];
    const int m = t / N, n = t - m * N;
    out[transposed ? n * M + m : t] = s;
}

// Adam on the packed FP32 parameters, then the BF16 copies W_l [out][in] and W_l^T [in][out]
struct BfPtrs {
    bf16 *W[N_LAYERS], *Wt[N_LAYERS];
    bf16 *Wc[N_LAYERS], *Wtc[N_LAYERS];  // core-matrix layouts (K = fan_in / fan_out) of the fused kernels
};
__global__ void k_adam(int64_t np, float *theta, const float *grad, float *m, float *v, const int64_t *t_dev, float lr,
                       float b1, float b2, float eps, int update, BfPtrs bp) {
    const int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (p >= np) return;
    float th = theta[p];
    if (update) {
        const int64_t t = *t_dev + 1;
        const float gp = grad[p];
        const float mm = b1 * m[p] + (1.0f - b1) * gp;
        const float vv = b2 * v[p] + (1.0f - b2) * gp * gp;
        m[p] = mm;
        v[p] = vv;
        const float mh = mm / (1.0f - powf(b1, (float)t));
        const float vh = vv / (1.0f - powf(b2, (float)t));
        th -= lr * mh / (sqrtf(vh) + eps);
        theta[p] = th;
    }
    int64_t o = 0;
    for (int l = 0; l < N_LAYERS; ++l) {
        const int64_t nw = (int64_t)fan_out(l) * fan_in(l);
        if (p < o + nw) {
            const int64_t q = p - o;
            const int r = (int)(q / fan_in(l)), c = (int)(q - (int64_t)r * fan_in(l));
            const bf16 hb = __float2bfloat16(th);
            bp.W[l][q] = hb;
            bp.Wt[l][(int64_t)c * fan_out(l) + r] = hb;
            bp.Wc[l][cmo(r, c, fan_in(l))] = hb;
            bp.Wtc[l][cmo(c, r, fan_out(l))] = hb;
            return;
        }
        o += nw + fan_out(l);
        if (p < o) return;  // a bias
    }
}
__global__ void k_incr(int64_t *a, int64_t *b) {
    ++*a;
    if (b) ++*b;
}

// warm start: predicted (u, v, w, p) into ACM fields of type T (sorted node order),
// zero velocity on wall nodes
template <typename T>
__global__ void k_inject(int64_t n, const float *__restrict__ pred, const uint8_t *__restrict__ type, float4 scale,
                         T *u, T *v, T *w, T *p) {
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n) return;
    const bool wall = type[i] != 0;
    u[i] = wall ? (T)0 : (T)(scale.x * pred[4 * i]);
    v[i] = wall ? (T)0 : (T)(scale.y * pred[4 * i + 1]);
    w[i] = wall ? (T)0 : (T)(scale.z * pred[4 * i + 2]);
    p[i] = (T)(scale.w * pred[4 * i + 3]);
}
// radius and signed wall distance of the context's nodes (sorted order)
__global__ void k_node_geo(int64_t n, const double *__restrict__ xyz, double cx, double cy, double cz, double r,
                           float *rad, float *sdf) {
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n) return;
    const double dx = mimg(xyz[3 * i] - cx), dy = mimg(xyz[3 * i + 1] - cy), dz = mimg(xyz[3 * i + 2] - cz);
    rad[i] = (float)r;
    sdf[i] = (float)(sqrt(dx * dx + dy * dy + dz * dz) - r);
}

// ---- fused training step -------------------------------------------------------------
// Two kernels per training step instead of one GEMM launch per layer and pass.  A CTA
// owns 128-row tiles of the batch (row = TMEM lane).
//
//  k_mlp_fwd: draws the tile's samples, computes their features, and runs the five
//    layers back to back: A operand = the tile's activations in shared memory, B =
//    the layer's weights (all five bulk-copied into shared memory once per CTA),
//    accumulator in TMEM; the epilogue (bias, GELU, GELU') writes the next layer's A
//    operand in place and keeps H_l, GELU'(Z_l) and the output error dY in global
//    memory for the backward kernel.
//  k_mlp_bwd: for l = 5..1, from the tile's rows of dZ_l and H_{l-1} in shared
//    memory: dW_l = dZ_l^T H_{l-1} (both tiles read MN-major, so no transposed copy
//    is written) and dH_{l-1} = dZ_l W_l (K-major) as two tcgen05 MMA chains (W_l^T
//    resident in shared memory), dZ_{l-1} = dH_{l-1} * GELU'(Z_{l-1}); the tile's dW
//    and db are added into the gradient with vector reductions.
//
// Operands are BF16 in the no-swizzle core-matrix layout with the whole K in one
// buffer: element (r, k) of an R x K operand at byte
// ((r/8) (K/8) + k/8) 128 + (r%8) 16 + (k%8) 2, so LBO = 128 B and SBO = 16 K B
// read K-major; the same bytes read MN-major are the R x K tile transposed.
// The rounding points are those of the per-layer path: BF16 features, activations,
// GELU' and back-propagated errors, FP32 accumulation.
constexpr int FW_WBYTES = 2 * (N_H * N_IN + 3 * N_H * N_H + N_OUT_PAD * N_H);  // W_1..W_5
constexpr int FB_WBYTES = 2 * (3 * N_H * N_H + N_H * N_OUT_PAD);               // W_2^T..W_5^T
constexpr int TILE_BYTES = 2 * 128 * 128;
// all five layers' biases, layer l at [128 l, 128 l + fan_out(l))
constexpr int FW_NBIAS = 4 * 128 + N_OUT_PAD;
// forward: weights, one activation tile per tile group (NG groups of 256 threads), biases
constexpr size_t fw_smem(int ng) { return FW_WBYTES + ng * TILE_BYTES + 4 * FW_NBIAS + 64 + 1024; }
// backward: W^T, the dZ and H tiles, per-CTA sums of db (5 layers x 4 row groups x 128),
// dW_5^T (16 x 128) and dW_1 (64 x 128) in FP32
constexpr int FB_NSUM = 5 * 4 * 128 + 16 * 128 + 64 * 128;
constexpr size_t FB_SMEM = FB_WBYTES + 2 * TILE_BYTES + 4 * FB_NSUM + 64 + 1024;

// The features X, H_l, GELU'(Z_l) and the output error dY between the fused forward
// and backward kernels (private to them): per 128-row tile, NQ chunks of 8 columns
// (NQ = columns / 8), each chunk's 128 rows contiguous at 16 bytes per row, so the 32
// lanes of a warp (32 consecutive rows of the tile) write or read 512 contiguous bytes
// per 16-byte access.  Element offset of chunk q of row r.
template <int NQ>
__device__ __forceinline__ int64_t chunk_off(int64_t r, int q) {
    return (((r >> 7) * NQ + q) * 128 + (r & 127)) * 8;
}
__device__ __forceinline__ int64_t hg_off(int64_t r, int q) { return chunk_off<N_H / 8>(r, q); }

struct FusedArgs {
    int B;                       // rows, a multiple of 128
    int64_t n;                   // samples in the data
    const double *xyz;
    const float *rad, *sdf, *tgt;
    const int64_t *idx;          // explicit sample indices, or null: counter-based draws
    uint64_t seed;
    const int64_t *step_dev;
    const bf16 *Wc[N_LAYERS];    // W_l [fan_out][fan_in], core layout, K = fan_in
    const bf16 *Wtc[N_LAYERS];   // W_l^T [fan_in][fan_out], core layout, K = fan_out (l >= 1)
    const float *theta;          // FP32 masters (biases)
    bf16 *X;                     // B x 64 in the chunked layout of chunk_off
    bf16 *H[4], *G[4];           // B x 128 in the chunked layout of hg_off
    bf16 *dY;                    // B x 16 in the chunked layout of chunk_off
    float *loss, *grad;
    float gscale;
    int32_t *err;
};

// this thread's shared-memory stores -> visible to the tensor cores, then a CTA barrier
__device__ __forceinline__ void smem_to_mma_sync() {
    tc::fence_proxy_async_smem();
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
}
// the same over the 256 threads of tile group g (named barrier 1 + g)
__device__ __forceinline__ void smem_to_mma_sync_group(int g) {
    tc::fence_proxy_async_smem();
    tc::fence_before_sync();
    asm volatile("bar.sync %0, 256;" ::"r"(1 + g) : "memory");
    tc::fence_after_sync();
}

// D (TMEM) = A B^T over K, both operands K-major in shared memory (A: K_A = K columns)
__device__ __forceinline__ void mma_chain(uint32_t d, const bf16 *A, const bf16 *Bm, int K, uint32_t idesc) {
    for (int kk = 0; kk < (K >> 4); ++kk) {
        const uint64_t da = tc::smem_desc(reinterpret_cast<const uint8_t *>(A) + kk * 256, 128, 16 * K);
        const uint64_t db = tc::smem_desc(reinterpret_cast<const uint8_t *>(Bm) + kk * 256, 128, 16 * K);
        tc::mma_bf16(d, da, db, idesc, kk > 0 ? 1u : 0u);
    }
}

// D (TMEM) = A^T B over the 128 rows of a tile: A and B are [128 rows][width] tiles
// (widths wa, wb) in the K-major core layout above, read MN-major with K = the row
// index.  Core matrices adjacent along K (8 rows) are 16 width bytes apart (LBO),
// adjacent along M / N 128 bytes (SBO); one MMA takes 16 rows.
// acc: add to the accumulator already in D instead of overwriting it.
__device__ __forceinline__ void mma_chain_rows(uint32_t d, const bf16 *A, int wa, const bf16 *Bm, int wb, uint32_t idesc,
                                               bool acc) {
    for (int kk = 0; kk < 8; ++kk) {
        const uint64_t da = tc::smem_desc(reinterpret_cast<const uint8_t *>(A) + kk * 32 * wa, 16 * wa, 128);
        const uint64_t db = tc::smem_desc(reinterpret_cast<const uint8_t *>(Bm) + kk * 32 * wb, 16 * wb, 128);
        tc::mma_bf16(d, da, db, idesc | tc::IDESC_A_MN | tc::IDESC_B_MN, (kk > 0 || acc) ? 1u : 0u);
    }
}

// Column sums over a warp's 32 rows (lane = row) of the 16 values each lane holds:
// a butterfly in which every step halves the values a lane carries (it keeps one
// half, adds its partner's copy of that half and hands over the other), 8 + 4 + 2 +
// 1 + 1 shuffles instead of 5 per value.  Returns the sum of column
// col = 8 b4 + 4 b3 + 2 b2 + b1 (bK: bit K of the lane), held by lanes 2 col + {0, 1}.
__device__ __forceinline__ float warp_colsum16(const float *v, int lane, int &col) {
    float a[8], b[4], c[2];
    bool hi = (lane & 16) != 0;
#pragma unroll
    for (int i = 0; i < 8; ++i)
        a[i] = (hi ? v[i + 8] : v[i]) + __shfl_xor_sync(0xffffffffu, hi ? v[i] : v[i + 8], 16);
    hi = (lane & 8) != 0;
#pragma unroll
    for (int i = 0; i < 4; ++i)
        b[i] = (hi ? a[i + 4] : a[i]) + __shfl_xor_sync(0xffffffffu, hi ? a[i] : a[i + 4], 8);
    hi = (lane & 4) != 0;
#pragma unroll
    for (int i = 0; i < 2; ++i)
        c[i] = (hi ? b[i + 2] : b[i]) + __shfl_xor_sync(0xffffffffu, hi ? b[i] : b[i + 2], 4);
    hi = (lane & 2) != 0;
    float d = (hi ? c[1] : c[0]) + __shfl_xor_sync(0xffffffffu, hi ? c[0] : c[1], 2);
    d += __shfl_xor_sync(0xffffffffu, d, 1);
    col = ((lane >> 4) & 1) * 8 + ((lane >> 3) & 1) * 4 + ((lane >> 2) & 1) * 2 + ((lane >> 1) & 1);
    return d;
}

// 8 BF16 values as one 16-byte word
__device__ __forceinline__ uint4 pack8(const bf16 *v) { return *reinterpret_cast<const uint4 *>(v); }

// Both kernels run 256 threads per tile: thread t serves row t % 128 of the tile (TMEM
// lane t % 128, reachable by warps w and w + 4) and half h = t / 128 of each layer's
// columns, so two warps per scheduler share the epilogue math.  The forward kernel
// runs NG such tile groups per CTA on the shared resident weights, each with its own
// activation tile, TMEM columns, mbarrier and named barrier: while one group's
// epilogue runs, the other's MMAs keep the tensor pipe busy.
template <int NG>
__global__ void __launch_bounds__(256 * NG, 1) k_mlp_fwd(FusedArgs f) {
    extern __shared__ __align__(1024) uint8_t smem[];
    bf16 *sW[N_LAYERS];
    uint8_t *p = smem;
    for (int l = 0; l < N_LAYERS; ++l) {
        sW[l] = reinterpret_cast<bf16 *>(p);
        p += 2 * fan_out(l) * fan_in(l);
    }
    const int t = threadIdx.x, warp = t >> 5, lane = t & 31;
    const int grp = t >> 8, gt = t & 255;  // tile group, thread within it
    const int row = gt & 127, half = gt >> 7;
    bf16 *act = reinterpret_cast<bf16 *>(p + grp * TILE_BYTES);
    p += NG * TILE_BYTES;
    float *sB = reinterpret_cast<float *>(p);  // the biases (FP32 masters), read by every epilogue
    p += 4 * FW_NBIAS;
    uint64_t *wbar = reinterpret_cast<uint64_t *>(p), *mbar = wbar + 1 + grp;
    uint32_t *slot = reinterpret_cast<uint32_t *>(wbar + 1 + NG);
    if (warp == 0) {
        tc::tmem_alloc(slot, 128 * NG);
        tc::tmem_relinquish();
    }
    if (t == 0) {
        tc::mbar_init(wbar, 1);
        for (int g = 0; g < NG; ++g) tc::mbar_init(wbar + 1 + g, 1);
        tc::fence_mbar_init();
    }
    for (int i = t; i < FW_NBIAS; i += blockDim.x) {
        const int l = i >> 7, c = i & 127;
        sB[i] = f.theta[b_off_c(l) + c];
    }
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    const uint32_t tmem = *slot + (uint32_t)(128 * grp), tlane = (uint32_t)((warp & 3) * 32) << 16;
    if (t == 0) {
        tc::mbar_arrive_expect_tx(wbar, FW_WBYTES);
        for (int l = 0; l < N_LAYERS; ++l) tc::bulk_copy_g2s(sW[l], f.Wc[l], 2 * fan_out(l) * fan_in(l), wbar);
    }
    bool ok = tc::mbar_wait(wbar, 0, WAIT_NS);
    uint32_t phase = 0;
    float lsum = 0.0f;
    for (int tile = blockIdx.x * NG + grp; ok && tile < (f.B >> 7); tile += gridDim.x * NG) {
        const int64_t r = (int64_t)tile * 128 + row;
        int64_t s;
        if (f.idx) s = f.idx[r];
        else {
            const uint64_t c = f.seed * (1ull << 32) + (uint64_t)(*f.step_dev) * (uint64_t)f.B + (uint64_t)r;
            s = (int64_t)(splitmix64(c) % (uint64_t)f.n);
        }
        {   // features of sample s (half h: wave vectors 8h .. 8h + 7; half 0 also r and
            // phi_sdf): the sines and cosines of k_features, evaluated in FP32 on the
            // coordinates reduced to [0, 1) (periodic, so exact up to float rounding,
            // ~1e-7, far below the BF16 resolution the features are stored at)
            const double x = f.xyz[3 * s], y = f.xyz[3 * s + 1], z = f.xyz[3 * s + 2];
            const float xf = (float)(x - floor(x)), yf = (float)(y - floor(y)), zf = (float)(z - floor(z));
            __align__(16) bf16 part[32];
#pragma unroll
            for (int jj = 0; jj < 8; ++jj) {
                const int j = 8 * half + jj;
                float sn, cs;
                sincospif(2.0f * ((float)c_waves[j][0] * xf + (float)c_waves[j][1] * yf + (float)c_waves[j][2] * zf), &sn,
                          &cs);
                part[2 * jj] = __float2bfloat16(sn);
                part[2 * jj + 1] = __float2bfloat16(cs);
            }
#pragma unroll
            for (int j = 16; j < 32; ++j) part[j] = __float2bfloat16(0.0f);
            if (half == 0) {
                part[16] = __float2bfloat16(f.rad[s]);  // columns 32, 33 of the row
                part[17] = __float2bfloat16(f.sdf[s]);
            }
            // half 0 owns columns 0..15 and 32..47 (r, phi_sdf, zeros), half 1 columns
            // 16..31 and 48..63 (zeros): each written as two 16-column pieces
            const int cA = 16 * half, cB = 32 + 16 * half;
#pragma unroll
            for (int k = 0; k < 2; ++k) {
                const uint4 wA = pack8(part + 8 * k), wB = pack8(part + 16 + 8 * k);
                *reinterpret_cast<uint4 *>(act + cmo(row, cA + 8 * k, N_IN)) = wA;
                *reinterpret_cast<uint4 *>(act + cmo(row, cB + 8 * k, N_IN)) = wB;
                *reinterpret_cast<uint4 *>(f.X + chunk_off<N_IN / 8>(r, (cA >> 3) + k)) = wA;
                *reinterpret_cast<uint4 *>(f.X + chunk_off<N_IN / 8>(r, (cB >> 3) + k)) = wB;
            }
        }
        float tg[N_OUT];
#pragma unroll
        for (int c = 0; c < N_OUT; ++c) tg[c] = half ? 0.0f : f.tgt[s * N_OUT + c];
        for (int l = 0; l < N_LAYERS && ok; ++l) {
            const int fi = fan_in(l), fo = fan_out(l);
            if (NG == 1) smem_to_mma_sync();
            else smem_to_mma_sync_group(grp);
            if (gt == 0) {
                mma_chain(tmem, act, sW[l], fi, tc::idesc_bf16_f32(128, fo));
                tc::mma_commit(mbar);
            }
            ok = tc::mbar_wait(mbar, phase, WAIT_NS);
            phase ^= 1;
            if (!ok) break;
            tc::fence_after_sync();
            const float *bias = sB + 128 * l;
            if (l < N_LAYERS - 1) {
                for (int c0 = 64 * half; c0 < 64 * half + 64; c0 += 16) {
                    float v[16];
                    tc::tmem_ld16(tmem + tlane + (uint32_t)c0, v);
#pragma unroll
                    for (int k = 0; k < 4; ++k) {  // z = accumulator + bias, the bias as four 16-byte loads
                        const float4 q = reinterpret_cast<const float4 *>(bias + c0)[k];
                        v[4 * k] += q.x; v[4 * k + 1] += q.y; v[4 * k + 2] += q.z; v[4 * k + 3] += q.w;
                    }
                    __align__(16) __nv_bfloat162 hv2[8];
                    __align__(16) __nv_bfloat162 gv2[8];
#pragma unroll
                    for (int i = 0; i < 16; i += 2) {  // pairs: one two-value conversion each
                        float h0, g0, h1, g1;
                        gelu_both(v[i], h0, g0);
                        gelu_both(v[i + 1], h1, g1);
                        hv2[i >> 1] = __floats2bfloat162_rn(h0, h1);
                        gv2[i >> 1] = __floats2bfloat162_rn(g0, g1);
                    }
                    const bf16 *hv = reinterpret_cast<const bf16 *>(hv2), *gv = reinterpret_cast<const bf16 *>(gv2);
                    *reinterpret_cast<uint4 *>(act + cmo(row, c0, N_H)) = pack8(hv);
                    *reinterpret_cast<uint4 *>(act + cmo(row, c0 + 8, N_H)) = pack8(hv + 8);
#pragma unroll
                    for (int k = 0; k < 2; ++k) {
                        *reinterpret_cast<uint4 *>(f.H[l] + hg_off(r, (c0 >> 3) + k)) = pack8(hv + 8 * k);
                        *reinterpret_cast<uint4 *>(f.G[l] + hg_off(r, (c0 >> 3) + k)) = pack8(gv + 8 * k);
                    }
                }
            } else if (half == 0) {
                float v[16];
                tc::tmem_ld16(tmem + tlane, v);
                __align__(16) bf16 dv[16];
#pragma unroll
                for (int c = 0; c < 16; ++c) {
                    float dy = 0.0f;
                    if (c < N_OUT) {
                        const float e = v[c] + bias[c] - tg[c];
                        lsum += e * e;
                        dy = f.gscale * e;
                    }
                    dv[c] = __float2bfloat16(dy);
                }
                *reinterpret_cast<uint4 *>(f.dY + chunk_off<N_OUT_PAD / 8>(r, 0)) = pack8(dv);
                *reinterpret_cast<uint4 *>(f.dY + chunk_off<N_OUT_PAD / 8>(r, 1)) = pack8(dv + 8);
            }
            tc::fence_before_sync();
        }
    }
    if (!ok) {  // a wait ran out: report, give the outstanding work one more bounded wait
        if (gt == 0) atomicExch(f.err, 1);
        tc::mbar_wait(mbar, phase, WAIT_NS);
    }
    for (int off = 16; off > 0; off >>= 1) lsum += __shfl_xor_sync(0xffffffffu, lsum, off);
    if (lane == 0 && lsum != 0.0f) atomicAdd(f.loss, lsum);
    tc::fence_before_sync();
    __syncthreads();
    if (warp == 0) tc::tmem_dealloc(*slot, 128 * NG);
}

__global__ void __launch_bounds__(256, 1) k_mlp_bwd(FusedArgs f) {
    extern __shared__ __align__(1024) uint8_t smem[];
    bf16 *sWt[N_LAYERS] = {nullptr, nullptr, nullptr, nullptr, nullptr};
    uint8_t *p = smem;
    for (int l = 1; l < N_LAYERS; ++l) {
        sWt[l] = reinterpret_cast<bf16 *>(p);
        p += 2 * fan_out(l) * fan_in(l);
    }
    bf16 *An = reinterpret_cast<bf16 *>(p);                  // dZ_l [128 rows][fan_out], K = fan_out
    bf16 *Hs = reinterpret_cast<bf16 *>(p + TILE_BYTES);     // H_{l-1} [128 rows][fan_in]
    p += 2 * TILE_BYTES;
    // this CTA's sums over its tiles, each entry owned by one thread: db_l per warp row
    // group [l][row group][column] (the lane that holds the column's warp sum), dW_5^T
    // [out][in] and dW_1 [in][out] (thread = the TMEM lane's unit)
    float *dbq = reinterpret_cast<float *>(p);
    float *dw5 = dbq + 5 * 4 * 128;
    float *dw1 = dw5 + 16 * 128;
    p += 4 * FB_NSUM;
    uint64_t *wbar = reinterpret_cast<uint64_t *>(p), *mbar = wbar + 1;
    uint32_t *slot = reinterpret_cast<uint32_t *>(wbar + 2);
    const int t = threadIdx.x, warp = t >> 5, lane = t & 31;
    const int row = t & 127, half = t >> 7, wq = warp & 3;
    // TMEM columns: 0..127 dH_{l-1} of the current layer (also dW_5^T and dW_1 of the
    // current tile, read out at once); 128 l .. 128 l + 127 for l = 1, 2, 3: dW_{l+1}
    // summed over all of this CTA's tiles, added into the gradient once at the end
    for (int e = threadIdx.x; e < FB_NSUM; e += blockDim.x) dbq[e] = 0.0f;
    if (warp == 0) {
        tc::tmem_alloc(slot, 512);
        tc::tmem_relinquish();
    }
    if (t == 0) {
        tc::mbar_init(wbar, 1);
        tc::mbar_init(mbar, 1);
        tc::fence_mbar_init();
    }
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    const uint32_t tmem = *slot, tlane = (uint32_t)(wq * 32) << 16;
    int ntiles = 0;  // tiles this CTA has finished
    if (t == 0) {
        tc::mbar_arrive_expect_tx(wbar, FB_WBYTES);
        for (int l = 1; l < N_LAYERS; ++l) tc::bulk_copy_g2s(sWt[l], f.Wtc[l], 2 * fan_out(l) * fan_in(l), wbar);
    }
    bool ok = tc::mbar_wait(wbar, 0, WAIT_NS);
    uint32_t phase = 0;
    // column sums of this thread's dz values over its warp's 32 rows, added to db_l of the
    // warp's row group (no barrier: each entry has one owner; the groups are summed at the end)
    auto colsum16 = [&](const float *dz, int c0, int l) {
        int col;
        const float sv = warp_colsum16(dz, lane, col);
        if ((lane & 1) == 0) dbq[(l * 4 + wq) * 128 + c0 + col] += sv;
    };
    // Global rows are loaded into registers while the MMAs run: this half's columns of the
    // input of layer l (H_{l-1}, X for the first layer) for the next layer's staging, and of
    // GELU'(Z_{l-2}) for the next layer's epilogue (gnext, moved into greg after this
    // layer's epilogue), so each GELU' load has a layer's MMAs and epilogue to arrive.
    uint4 hreg[8], greg[8], gnext[8];
    auto load_h = [&](int l, int64_t rr) {
        const int hw = fan_in(l) >> 1;
        if (l > 0) {
#pragma unroll
            for (int k = 0; k < 8; ++k)
                hreg[k] = *reinterpret_cast<const uint4 *>(f.H[l - 1] + hg_off(rr, ((hw * half) >> 3) + k));
        } else {  // X
#pragma unroll
            for (int k = 0; k < 4; ++k)
                hreg[k] = *reinterpret_cast<const uint4 *>(f.X + chunk_off<N_IN / 8>(rr, ((hw * half) >> 3) + k));
        }
    };
    auto store_h = [&](int l) {
        const int fi = fan_in(l), hw = fi >> 1;
#pragma unroll
        for (int k = 0; k < 8; ++k)
            if (k < (hw >> 3)) *reinterpret_cast<uint4 *>(Hs + cmo(row, hw * half + 8 * k, fi)) = hreg[k];
    };
    // GELU'(Z_{l-1}), read by the epilogue of layer l, into dst
    auto load_g = [&](uint4 (&dst)[8], int l, int64_t rr) {
#pragma unroll
        for (int k = 0; k < 8; ++k) dst[k] = *reinterpret_cast<const uint4 *>(f.G[l - 1] + hg_off(rr, 8 * half + k));
    };
    uint4 dyreg[2];  // the tile's output error row dY (half 0), fetched with the tile's H_4 rows
    auto load_dy = [&](int64_t rr) {
        if (half == 0) {
            dyreg[0] = *reinterpret_cast<const uint4 *>(f.dY + chunk_off<N_OUT_PAD / 8>(rr, 0));
            dyreg[1] = *reinterpret_cast<const uint4 *>(f.dY + chunk_off<N_OUT_PAD / 8>(rr, 1));
        }
    };
    if (blockIdx.x < (f.B >> 7)) {
        load_h(N_LAYERS - 1, (int64_t)blockIdx.x * 128 + row);
        load_dy((int64_t)blockIdx.x * 128 + row);
        load_g(greg, N_LAYERS - 1, (int64_t)blockIdx.x * 128 + row);
    }
    for (int tile = blockIdx.x; ok && tile < (f.B >> 7); tile += gridDim.x) {
        const int64_t r = (int64_t)tile * 128 + row;
        const int64_t r_next = tile + (int)gridDim.x < (f.B >> 7) ? r + (int64_t)gridDim.x * 128 : -1;
        if (half == 0) {  // dZ_5 = dY (K = 16) and its column sums (db_5)
            __align__(16) bf16 dv[16];
            *reinterpret_cast<uint4 *>(dv) = dyreg[0];
            *reinterpret_cast<uint4 *>(dv + 8) = dyreg[1];
            *reinterpret_cast<uint4 *>(An + cmo(row, 0, N_OUT_PAD)) = pack8(dv);
            *reinterpret_cast<uint4 *>(An + cmo(row, 8, N_OUT_PAD)) = pack8(dv + 8);
            float dz[16];
#pragma unroll
            for (int c = 0; c < 16; ++c) dz[c] = __bfloat162float(dv[c]);
            colsum16(dz, 0, N_LAYERS - 1);
        }
        for (int l = N_LAYERS - 1; l >= 0 && ok; --l) {
            const int fi = fan_in(l), fo = fan_out(l), hw = fi >> 1;
            store_h(l);  // the tile's rows of H_{l-1} (X for the first layer), this half's columns
            smem_to_mma_sync();
            // the MMAs below no longer need the registers: fetch the next rows behind them
            auto prefetch = [&]() {
                if (l > 0) {
                    if (l >= 2) load_g(gnext, l - 1, r);
                    load_h(l - 1, r);
                } else if (r_next >= 0) {
                    load_h(N_LAYERS - 1, r_next);
                    load_dy(r_next);
                    load_g(gnext, N_LAYERS - 1, r_next);
                }
            };
            if (l == N_LAYERS - 1) {
                // dW_5^T [128 in][16 out] = H_4^T dZ_5 into columns 0..15, read out (lane =
                // input unit) before dH_4 takes those columns
                if (t == 0) {
                    mma_chain_rows(tmem, Hs, fi, An, N_OUT_PAD, tc::idesc_bf16_f32(128, N_OUT_PAD), false);
                    tc::mma_commit(mbar);
                }
                prefetch();
                ok = tc::mbar_wait(mbar, phase, WAIT_NS);
                phase ^= 1;
                if (!ok) break;
                tc::fence_after_sync();
                if (half == 0) {
                    float v[16];
                    tc::tmem_ld16(tmem + tlane, v);
#pragma unroll
                    for (int o = 0; o < N_OUT_PAD; ++o) dw5[o * 128 + row] += v[o];
                }
                tc::fence_before_sync();
                __syncthreads();
                tc::fence_after_sync();
                if (t == 0) {  // dH_4 [128 rows][128] = dZ_5 W_5
                    mma_chain(tmem, An, sWt[l], fo, tc::idesc_bf16_f32(128, fi));
                    tc::mma_commit(mbar);
                }
            } else {
                if (t == 0) {
                    // dW_l [128 out][fan_in] = dZ_l^T H_{l-1}: the first layer's into columns
                    // 0..63 (no dH there), the others added to their per-CTA sums
                    mma_chain_rows(tmem + 128 * l, An, fo, Hs, fi, tc::idesc_bf16_f32(128, fi), l > 0 && ntiles > 0);
                    if (l > 0)  // dH_{l-1} [128 rows][fan_in] = dZ_l W_l
                        mma_chain(tmem, An, sWt[l], fo, tc::idesc_bf16_f32(128, fi));
                    tc::mma_commit(mbar);
                }
                prefetch();
            }
            ok = tc::mbar_wait(mbar, phase, WAIT_NS);
            phase ^= 1;
            if (!ok) break;
            tc::fence_after_sync();
            if (l == 0) {  // lane = output unit: row `row` of dW_1, columns of this half
                for (int c0 = hw * half; c0 < hw * half + hw; c0 += 16) {
                    float v[16];
                    tc::tmem_ld16(tmem + tlane + (uint32_t)c0, v);
#pragma unroll
                    for (int i = 0; i < 16; ++i) dw1[(c0 + i) * 128 + row] += v[i];
                }
            }
            if (l > 0) {  // dZ_{l-1} = dH_{l-1} * GELU'(Z_{l-1}); its column sums are db_{l-1}
#pragma unroll
                for (int j = 0; j < 4; ++j) {
                    const int c0 = 64 * half + 16 * j;
                    float v[16];
                    tc::tmem_ld16(tmem + tlane + (uint32_t)c0, v);
                    __align__(16) bf16 gv[16];
                    *reinterpret_cast<uint4 *>(gv) = greg[2 * j];
                    *reinterpret_cast<uint4 *>(gv + 8) = greg[2 * j + 1];
                    __align__(16) __nv_bfloat162 dv2[8];
                    float dz[16];
#pragma unroll
                    for (int i = 0; i < 16; i += 2) {  // pairs: one two-value conversion each
                        const float2 gf = __bfloat1622float2(reinterpret_cast<const __nv_bfloat162 *>(gv)[i >> 1]);
                        dv2[i >> 1] = __floats2bfloat162_rn(v[i] * gf.x, v[i + 1] * gf.y);
                        const float2 df = __bfloat1622float2(dv2[i >> 1]);
                        dz[i] = df.x;
                        dz[i + 1] = df.y;
                    }
                    const bf16 *dv = reinterpret_cast<const bf16 *>(dv2);
                    *reinterpret_cast<uint4 *>(An + cmo(row, c0, N_H)) = pack8(dv);
                    *reinterpret_cast<uint4 *>(An + cmo(row, c0 + 8, N_H)) = pack8(dv + 8);
                    colsum16(dz, c0, l - 1);
                }
            }
            if (l >= 2 || (l == 0 && r_next >= 0)) {  // GELU' of the next epilogue
#pragma unroll
                for (int k = 0; k < 8; ++k) greg[k] = gnext[k];
            }
            tc::fence_before_sync();
        }
        ++ntiles;
    }
    if (ok && ntiles > 0) {  // this CTA's sums into the gradient: dW_1, dW_5, db from shared memory,
        // dW_2 .. dW_4 (lane = output unit) from TMEM
        {
            float *gw = f.grad + w_off_c(0) + (int64_t)row * N_IN;
            for (int c0 = 32 * half; c0 < 32 * half + 32; c0 += 4)
                tc::red_add_v4(gw + c0, dw1[c0 * 128 + row], dw1[(c0 + 1) * 128 + row], dw1[(c0 + 2) * 128 + row],
                               dw1[(c0 + 3) * 128 + row]);
            if (half == 0)
                for (int o = 0; o < N_OUT_PAD; ++o) {
                    const float v = dw5[o * 128 + row];
                    if (v != 0.0f) atomicAdd(f.grad + w_off_c(N_LAYERS - 1) + o * N_H + row, v);
                }
            if (t < N_H)
                for (int l = 0; l < N_LAYERS; ++l) {  // (written before the last layer's barrier)
                    const float *q = dbq + l * 4 * 128 + t;
                    const float v = q[0] + q[128] + q[256] + q[384];
                    if (v != 0.0f && (l < N_LAYERS - 1 || t < N_OUT_PAD)) atomicAdd(f.grad + b_off_c(l) + t, v);
                }
        }
        tc::fence_after_sync();
        for (int l = 1; l < N_LAYERS - 1; ++l) {
            float *gw = f.grad + w_off_c(l) + (int64_t)row * N_H;
            for (int c0 = 64 * half; c0 < 64 * half + 64; c0 += 16) {
                float v[16];
                tc::tmem_ld16(tmem + tlane + (uint32_t)(128 * l + c0), v);
#pragma unroll
                for (int i = 0; i < 16; i += 4) tc::red_add_v4(gw + c0 + i, v[i], v[i + 1], v[i + 2], v[i + 3]);
            }
        }
    }
    if (!ok) {
        if (t == 0) atomicExch(f.err, 1);
        tc::mbar_wait(mbar, phase, WAIT_NS);
    }
    tc::fence_before_sync();
    __syncthreads();
    if (warp == 0) tc::tmem_dealloc(tmem, 512);
}

cudaError_t fused_set_smem() {
    cudaError_t e = cudaFuncSetAttribute(k_mlp_fwd<1>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)fw_smem(1));
    if (e == cudaSuccess) e = cudaFuncSetAttribute(k_mlp_fwd<2>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)fw_smem(2));
    if (e == cudaSuccess) e = cudaFuncSetAttribute(k_mlp_bwd, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)FB_SMEM);
    return e;
}

}  // namespace

// =====================================================================================
struct rbf_mlp {
    template <typename T> using DevArr = rbf::DevArr<T>;
    int device = 0;
    cudaStream_t st = nullptr;
    bool own_stream = false;
    std::string err;
    int64_t launches = 0;
    DevArr<float> theta, m, v, grad;
    DevArr<bf16> W[N_LAYERS], Wt[N_LAYERS], Wc[N_LAYERS], Wtc[N_LAYERS];
    int nsm = 0;
    bool fused = true;  // training step: fused forward and backward kernels (else one GEMM per layer and pass)
    DevArr<int64_t> counters;  // [0] Adam step t, [1] batch draw step
    // training data
    int64_t nd = 0;
    DevArr<double> dxyz;
    DevArr<float> drad, dsdf, dtgt;
    // workspace for batch B
    int B = 0;
    DevArr<bf16> X, Xt, H[4], Ht[4], G[4], dY, dYt, dZ[4], dZt[4];
    DevArr<float> T, part, loss, pred;
    DevArr<int64_t> idx;
    DevArr<int32_t> errflag;
    cudaGraphExec_t gexec = nullptr;
    int gB = -1;
    uint64_t gseed = 0;
    float glr = 0.f;
};

namespace {

int mfail(rbf_mlp *m, int code, const std::string &msg) {
    if (m) m->err = msg;
    return code;
}
#define MCK(call)                                                                                         \
    do {                                                                                                  \
        cudaError_t e_ = (call);                                                                          \
        if (e_ != cudaSuccess)                                                                            \
            return mfail(mm, e_ == cudaErrorMemoryAllocation ? RBF_ENOMEM : RBF_ECUDA,                    \
                         std::string(#call) + ": " + cudaGetErrorString(e_));                             \
    } while (0)

struct MDevGuard {
    int prev = -1;
    explicit MDevGuard(int d) {
        cudaGetDevice(&prev);
        if (prev != d) cudaSetDevice(d);
    }
    ~MDevGuard() {
        int now = -1;
        cudaGetDevice(&now);
        if (prev >= 0 && now != prev) cudaSetDevice(prev);
    }
};

BfPtrs bf_ptrs(rbf_mlp *mm) {
    BfPtrs b;
    for (int l = 0; l < N_LAYERS; ++l) {
        b.W[l] = mm->W[l].p;
        b.Wt[l] = mm->Wt[l].p;
        b.Wc[l] = mm->Wc[l].p;
        b.Wtc[l] = mm->Wtc[l].p;
    }
    return b;
}

int ensure_workspace(rbf_mlp *mm, int B) {
    if (mm->B == B) return RBF_OK;
    if (mm->gexec) {
        cudaGraphExecDestroy(mm->gexec);
        mm->gexec = nullptr;
    }
    MCK(mm->X.alloc((size_t)B * N_IN));
    MCK(mm->Xt.alloc((size_t)B * N_IN));
    for (int l = 0; l < 4; ++l) {
        MCK(mm->H[l].alloc((size_t)B * N_H));
        MCK(mm->Ht[l].alloc((size_t)B * N_H));
        MCK(mm->G[l].alloc((size_t)B * N_H));
        MCK(mm->dZ[l].alloc((size_t)B * N_H));
        MCK(mm->dZt[l].alloc((size_t)B * N_H));
    }
    MCK(mm->dY.alloc((size_t)B * N_OUT_PAD));
    MCK(mm->dYt.alloc((size_t)B * N_OUT_PAD));
    MCK(mm->T.alloc((size_t)B * N_OUT));
    MCK(mm->pred.alloc((size_t)B * N_OUT));
    MCK(mm->idx.alloc((size_t)B));
    MCK(mm->part.alloc((size_t)(B / 128) * N_H * N_H));
    mm->B = B;
    return RBF_OK;
}

GemmArgs gemm_args(const bf16 *A, int lda, const bf16 *Bm, int ldb, int M, int N, int K, int32_t *err) {
    GemmArgs g;
    std::memset(&g, 0, sizeof(g));
    g.A = A; g.lda = lda; g.B = Bm; g.ldb = ldb; g.M = M; g.N = N; g.K = K; g.err = err; g.nvalid = M;
    return g;
}

// forward of the B rows in X; train: keep activations, transposes and GELU' and
// the loss gradient (targets T); otherwise write predictions to pred
cudaError_t enqueue_forward(rbf_mlp *mm, int B, int nvalid, bool train) {
    cudaError_t e;
    const bf16 *in = mm->X.p;
    int fin = N_IN;
    for (int l = 0; l < 4; ++l) {
        GemmArgs g = gemm_args(in, fin, mm->W[l].p, fan_in(l), B, N_H, fin, mm->errflag.p);
        g.bias = mm->theta.p + b_off(l);
        g.H = mm->H[l].p;
        g.Ht = train ? mm->Ht[l].p : nullptr;
        g.G = train ? mm->G[l].p : nullptr;
        g.ldt = B;
        g.nvalid = nvalid;
        if ((e = launch_gemm(EP_FWD, g, 1, mm->st)) != cudaSuccess) return e;
        ++mm->launches;
        in = mm->H[l].p;
        fin = N_H;
    }
    GemmArgs g = gemm_args(in, N_H, mm->W[4].p, N_H, B, N_OUT_PAD, N_H, mm->errflag.p);
    g.bias = mm->theta.p + b_off(4);
    g.nvalid = nvalid;
    if (train) {
        g.T = mm->T.p;
        g.H = mm->dY.p;
        g.Ht = mm->dYt.p;
        g.ldt = B;
        g.loss = mm->loss.p;
        g.db = mm->grad.p + b_off(4);
        g.gscale = 2.0f / ((float)nvalid * N_OUT);
        e = launch_gemm(EP_OUT, g, 1, mm->st);
    } else {
        g.out32 = mm->pred.p;
        e = launch_gemm(EP_PRED, g, 1, mm->st);
    }
    ++mm->launches;
    return e;
}

// backward: gradient of the mean squared error into mm->grad (packed layout)
cudaError_t enqueue_backward(rbf_mlp *mm, int B) {
    cudaError_t e;
    const int ks = B / 128;
    // dW5^T = H4^T dY  ([128][16], split over the batch)
    {
        GemmArgs g = gemm_args(mm->Ht[3].p, B, mm->dYt.p, B, N_H, N_OUT_PAD, B, mm->errflag.p);
        g.out32 = mm->part.p;
        if ((e = launch_gemm(EP_F32, g, ks, mm->st)) != cudaSuccess) return e;
        k_reduce_splits<<<(N_H * N_OUT_PAD + 255) / 256, 256, 0, mm->st>>>(mm->part.p, ks, N_H, N_OUT_PAD,
                                                                         mm->grad.p + w_off(4), 1);
        mm->launches += 2;
    }
    // dZ4 = (dY W5) * GELU'(Z4)
    {
        GemmArgs g = gemm_args(mm->dY.p, N_OUT_PAD, mm->Wt[4].p, N_OUT_PAD, B, N_H, N_OUT_PAD, mm->errflag.p);
        g.Gin = mm->G[3].p;
        g.H = mm->dZ[3].p;
        g.Ht = mm->dZt[3].p;
        g.ldt = B;
        g.db = mm->grad.p + b_off(3);
        if ((e = launch_gemm(EP_BWD, g, 1, mm->st)) != cudaSuccess) return e;
        ++mm->launches;
    }
    for (int l = 3; l >= 0; --l) {
        // dW_l = dZ_l^T H_{l-1}
        const bf16 *Hin_t = l > 0 ? mm->Ht[l - 1].p : mm->Xt.p;
        const int fin = fan_in(l);
        GemmArgs g = gemm_args(mm->dZt[l].p, B, Hin_t, B, N_H, fin, B, mm->errflag.p);
        g.out32 = mm->part.p;
        if ((e = launch_gemm(EP_F32, g, ks, mm->st)) != cudaSuccess) return e;
        k_reduce_splits<<<(N_H * fin + 255) / 256, 256, 0, mm->st>>>(mm->part.p, ks, N_H, fin, mm->grad.p + w_off(l), 0);
        mm->launches += 2;
        if (l == 0) break;
        // dZ_{l-1} = (dZ_l W_l) * GELU'(Z_{l-1})
        GemmArgs h = gemm_args(mm->dZ[l].p, N_H, mm->Wt[l].p, N_H, B, N_H, N_H, mm->errflag.p);
        h.Gin = mm->G[l - 1].p;
        h.H = mm->dZ[l - 1].p;
        h.Ht = mm->dZt[l - 1].p;
        h.ldt = B;
        h.db = mm->grad.p + b_off(l - 1);
        if ((e = launch_gemm(EP_BWD, h, 1, mm->st)) != cudaSuccess) return e;
        ++mm->launches;
    }
    return cudaGetLastError();
}

// the fused forward and backward kernels of one training step on B rows
cudaError_t enqueue_fused(rbf_mlp *mm, int B, uint64_t seed, const int64_t *explicit_idx) {
    FusedArgs f;
    std::memset(&f, 0, sizeof(f));
    f.B = B; f.n = mm->nd; f.xyz = mm->dxyz.p; f.rad = mm->drad.p; f.sdf = mm->dsdf.p; f.tgt = mm->dtgt.p;
    f.idx = explicit_idx; f.seed = seed; f.step_dev = mm->counters.p + 1;
    for (int l = 0; l < N_LAYERS; ++l) { f.Wc[l] = mm->Wc[l].p; f.Wtc[l] = mm->Wtc[l].p; }
    f.theta = mm->theta.p; f.X = mm->X.p;
    for (int l = 0; l < 4; ++l) { f.H[l] = mm->H[l].p; f.G[l] = mm->G[l].p; }
    f.dY = mm->dY.p; f.loss = mm->loss.p; f.grad = mm->grad.p;
    f.gscale = 2.0f / ((float)B * N_OUT);
    f.err = mm->errflag.p;
    // two tile groups per forward CTA once the tiles outnumber the SMs
    const int tiles = B / 128, nsm = std::max(mm->nsm, 1);
    const unsigned grid = (unsigned)std::min(tiles, nsm);
    if (tiles > nsm) {
        k_mlp_fwd<2><<<(unsigned)std::min((tiles + 1) / 2, nsm), 512, fw_smem(2), mm->st>>>(f);
    } else {
        k_mlp_fwd<1><<<grid, 256, fw_smem(1), mm->st>>>(f);
    }
    k_mlp_bwd<<<grid, 256, FB_SMEM, mm->st>>>(f);
    mm->launches += 2;
    return cudaGetLastError();
}

cudaError_t enqueue_train_step(rbf_mlp *mm, int B, uint64_t seed, float lr, const int64_t *explicit_idx, bool update) {
    cudaError_t e;
    if ((e = cudaMemsetAsync(mm->grad.p, 0, mm->grad.n * sizeof(float), mm->st)) != cudaSuccess) return e;
    if ((e = cudaMemsetAsync(mm->loss.p, 0, sizeof(float), mm->st)) != cudaSuccess) return e;
    if (mm->fused) {
        if ((e = enqueue_fused(mm, B, seed, explicit_idx)) != cudaSuccess) return e;
    } else {
        k_features<<<(B + 127) / 128, 128, 0, mm->st>>>(B, mm->nd, mm->dxyz.p, mm->drad.p, mm->dsdf.p, mm->dtgt.p,
                                                        explicit_idx, seed, mm->counters.p + 1, mm->X.p, mm->Xt.p, B,
                                                        mm->T.p);
        ++mm->launches;
        if ((e = enqueue_forward(mm, B, B, true)) != cudaSuccess) return e;
        if ((e = enqueue_backward(mm, B)) != cudaSuccess) return e;
    }
    if (update) {
        const int64_t np = n_params_total();
        k_adam<<<(unsigned)((np + 255) / 256), 256, 0, mm->st>>>(np, mm->theta.p, mm->grad.p, mm->m.p, mm->v.p,
                                                                 mm->counters.p, lr, 0.9f, 0.999f, 1e-8f, 1, bf_ptrs(mm));
        k_incr<<<1, 1, 0, mm->st>>>(mm->counters.p, mm->counters.p + 1);
        mm->launches += 2;
    }
    return cudaGetLastError();
}

int check_err(rbf_mlp *mm) {
    int32_t f = 0;
    MCK(cudaMemcpyAsync(&f, mm->errflag.p, sizeof(int32_t), cudaMemcpyDeviceToHost, mm->st));
    MCK(cudaStreamSynchronize(mm->st));
    if (f) return mfail(mm, RBF_ETIMEOUT, "tensor-core wait exceeded its limit");
    return RBF_OK;
}

}  // namespace

extern "C" {

int64_t rbf_mlp_num_params(void) { return n_params_total(); }

int rbf_mlp_create(rbf_mlp **out, int device, void *stream) {
    if (!out) return RBF_EINVAL;
    *out = nullptr;
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || device < 0 || device >= ndev) return RBF_ECUDA;
    rbf_mlp *mm = new rbf_mlp();
    mm->device = device;
    MDevGuard dg(device);
    if (stream) mm->st = (cudaStream_t)stream;
    else {
        if (cudaStreamCreateWithFlags(&mm->st, cudaStreamNonBlocking) != cudaSuccess) { delete mm; return RBF_ECUDA; }
        mm->own_stream = true;
    }
    const int64_t np = n_params_total();
    bool ok = mm->theta.alloc(np) == cudaSuccess && mm->m.alloc(np) == cudaSuccess && mm->v.alloc(np) == cudaSuccess &&
              mm->grad.alloc(np) == cudaSuccess && mm->counters.alloc(2) == cudaSuccess &&
              mm->loss.alloc(1) == cudaSuccess && mm->errflag.alloc(1) == cudaSuccess && gemm_set_smem() == cudaSuccess &&
              fused_set_smem() == cudaSuccess &&
              cudaDeviceGetAttribute(&mm->nsm, cudaDevAttrMultiProcessorCount, device) == cudaSuccess;
    for (int l = 0; l < N_LAYERS && ok; ++l)
        ok = mm->W[l].alloc((size_t)fan_out(l) * fan_in(l)) == cudaSuccess &&
             mm->Wt[l].alloc((size_t)fan_out(l) * fan_in(l)) == cudaSuccess &&
             mm->Wc[l].alloc((size_t)fan_out(l) * fan_in(l)) == cudaSuccess &&
             mm->Wtc[l].alloc((size_t)fan_out(l) * fan_in(l)) == cudaSuccess;
    if (!ok) { rbf_mlp_destroy(mm); return RBF_ECUDA; }
    cudaMemsetAsync(mm->theta.p, 0, np * sizeof(float), mm->st);
    cudaMemsetAsync(mm->m.p, 0, np * sizeof(float), mm->st);
    cudaMemsetAsync(mm->v.p, 0, np * sizeof(float), mm->st);
    cudaMemsetAsync(mm->counters.p, 0, 2 * sizeof(int64_t), mm->st);
    cudaMemsetAsync(mm->errflag.p, 0, sizeof(int32_t), mm->st);
    if (cudaStreamSynchronize(mm->st) != cudaSuccess) { rbf_mlp_destroy(mm); return RBF_ECUDA; }
    *out = mm;
    return RBF_OK;
}

int rbf_mlp_destroy(rbf_mlp *mm) {
    if (!mm) return RBF_EINVAL;
    {
        MDevGuard dg(mm->device);
        if (mm->st) cudaStreamSynchronize(mm->st);
        if (mm->gexec) cudaGraphExecDestroy(mm->gexec);
        if (mm->own_stream && mm->st) cudaStreamDestroy(mm->st);
        delete mm;
    }
    return RBF_OK;
}

const char *rbf_mlp_last_error(const rbf_mlp *mm) { return mm ? mm->err.c_str() : "null"; }

int rbf_mlp_set_params(rbf_mlp *mm, const float *theta) {
    if (!mm || !theta) return RBF_EINVAL;
    MDevGuard dg(mm->device);
    const int64_t np = n_params_total();
    MCK(cudaMemcpyAsync(mm->theta.p, theta, np * sizeof(float), cudaMemcpyHostToDevice, mm->st));
    MCK(cudaMemsetAsync(mm->m.p, 0, np * sizeof(float), mm->st));
    MCK(cudaMemsetAsync(mm->v.p, 0, np * sizeof(float), mm->st));
    MCK(cudaMemsetAsync(mm->counters.p, 0, 2 * sizeof(int64_t), mm->st));
    k_adam<<<(unsigned)((np + 255) / 256), 256, 0, mm->st>>>(np, mm->theta.p, nullptr, nullptr, nullptr, mm->counters.p,
                                                             0.f, 0.f, 0.f, 0.f, 0, bf_ptrs(mm));
    ++mm->launches;
    MCK(cudaGetLastError());
    MCK(cudaStreamSynchronize(mm->st));
    return RBF_OK;
}

int rbf_mlp_get_params(rbf_mlp *mm, float *theta) {
    if (!mm || !theta) return RBF_EINVAL;
    MDevGuard dg(mm->device);
    MCK(cudaMemcpyAsync(theta, mm->theta.p, n_params_total() * sizeof(float), cudaMemcpyDeviceToHost, mm->st));
    MCK(cudaStreamSynchronize(mm->st));
    return RBF_OK;
}

int rbf_mlp_set_data(rbf_mlp *mm, int64_t n, const double *xyz, const float *radius, const float *sdf,
                     const float *target) {
    if (!mm || n < 1 || !xyz || !radius || !sdf || !target) return RBF_EINVAL;
    MDevGuard dg(mm->device);
    MCK(mm->dxyz.alloc(3 * n)); MCK(mm->drad.alloc(n)); MCK(mm->dsdf.alloc(n)); MCK(mm->dtgt.alloc(4 * n));
    MCK(cudaMemcpyAsync(mm->dxyz.p, xyz, 3 * n * sizeof(double), cudaMemcpyHostToDevice, mm->st));
    MCK(cudaMemcpyAsync(mm->drad.p, radius, n * sizeof(float), cudaMemcpyHostToDevice, mm->st));
    MCK(cudaMemcpyAsync(mm->dsdf.p, sdf, n * sizeof(float), cudaMemcpyHostToDevice, mm->st));
    MCK(cudaMemcpyAsync(mm->dtgt.p, target, 4 * n * sizeof(float), cudaMemcpyHostToDevice, mm->st));
    MCK(cudaStreamSynchronize(mm->st));
    mm->nd = n;
    return RBF_OK;
}

int rbf_mlp_gradient(rbf_mlp *mm, int batch, const int64_t *sample_idx, float *grad, double *loss) {
    if (!mm || !sample_idx || !grad) return RBF_EINVAL;
    if (batch < 128 || batch % 128 || batch > (1 << 22)) return mfail(mm, RBF_EINVAL, "batch must be a multiple of 128");
    if (!mm->nd) return mfail(mm, RBF_EINVAL, "rbf_mlp_gradient: set data first");
    for (int b = 0; b < batch; ++b)
        if (sample_idx[b] < 0 || sample_idx[b] >= mm->nd) return mfail(mm, RBF_EINVAL, "sample index out of range");
    MDevGuard dg(mm->device);
    int rc = ensure_workspace(mm, batch);
    if (rc) return rc;
    MCK(cudaMemcpyAsync(mm->idx.p, sample_idx, batch * sizeof(int64_t), cudaMemcpyHostToDevice, mm->st));
    MCK(enqueue_train_step(mm, batch, 0, 0.f, mm->idx.p, false));
    rc = check_err(mm);
    if (rc) return rc;
    float l = 0.f;
    MCK(cudaMemcpyAsync(grad, mm->grad.p, n_params_total() * sizeof(float), cudaMemcpyDeviceToHost, mm->st));
    MCK(cudaMemcpyAsync(&l, mm->loss.p, sizeof(float), cudaMemcpyDeviceToHost, mm->st));
    MCK(cudaStreamSynchronize(mm->st));
    if (loss) *loss = (double)l / ((double)batch * N_OUT);
    return RBF_OK;
}

int rbf_mlp_train(rbf_mlp *mm, int steps, int batch, double lr, uint64_t seed, float *loss_hist) {
    if (!mm || steps < 0) return RBF_EINVAL;
    if (batch < 128 || batch % 128 || batch > (1 << 22)) return mfail(mm, RBF_EINVAL, "batch must be a multiple of 128");
    if (!mm->nd) return mfail(mm, RBF_EINVAL, "rbf_mlp_train: set data first");
    MDevGuard dg(mm->device);
    int rc = ensure_workspace(mm, batch);
    if (rc) return rc;
    if (!mm->gexec || mm->gB != batch || mm->gseed != seed || mm->glr != (float)lr) {
        if (mm->gexec) cudaGraphExecDestroy(mm->gexec);
        mm->gexec = nullptr;
        cudaGraph_t g;
        MCK(cudaStreamBeginCapture(mm->st, cudaStreamCaptureModeThreadLocal));
        int64_t l0 = mm->launches;
        cudaError_t e = enqueue_train_step(mm, batch, seed, (float)lr, nullptr, true);
        cudaError_t e2 = cudaStreamEndCapture(mm->st, &g);
        mm->launches = l0;
        MCK(e);
        MCK(e2);
        e = cudaGraphInstantiate(&mm->gexec, g, 0);
        cudaGraphDestroy(g);
        MCK(e);
        mm->gB = batch;
        mm->gseed = seed;
        mm->glr = (float)lr;
    }
    for (int s = 0; s < steps; ++s) {
        MCK(cudaGraphLaunch(mm->gexec, mm->st));
        mm->launches += mm->fused ? 2 + 2 : 1 + 5 + 14 + 2;
        if (loss_hist) MCK(cudaMemcpyAsync(loss_hist + s, mm->loss.p, sizeof(float), cudaMemcpyDeviceToHost, mm->st));
    }
    rc = check_err(mm);
    if (rc) return rc;
    if (loss_hist)
        for (int s = 0; s < steps; ++s) loss_hist[s] /= (float)batch * N_OUT;
    return RBF_OK;
}

int rbf_mlp_predict(rbf_mlp *mm, int64_t n, const double *xyz, const float *radius, const float *sdf, float *out) {
    if (!mm || n < 1 || !xyz || !radius || !sdf || !out) return RBF_EINVAL;
    MDevGuard dg(mm->device);
    const int B = 16384;
    int rc = ensure_workspace(mm, std::max(mm->B, B));
    if (rc) return rc;
    const int Bw = mm->B;
    DevArr<double> px;
    DevArr<float> pr, ps;
    MCK(px.alloc(3 * n)); MCK(pr.alloc(n)); MCK(ps.alloc(n));
    MCK(cudaMemcpyAsync(px.p, xyz, 3 * n * sizeof(double), cudaMemcpyHostToDevice, mm->st));
    MCK(cudaMemcpyAsync(pr.p, radius, n * sizeof(float), cudaMemcpyHostToDevice, mm->st));
    MCK(cudaMemcpyAsync(ps.p, sdf, n * sizeof(float), cudaMemcpyHostToDevice, mm->st));
    std::vector<int64_t> ids(Bw);
    for (int64_t s0 = 0; s0 < n; s0 += Bw) {
        const int cnt = (int)std::min<int64_t>(Bw, n - s0);
        for (int b = 0; b < Bw; ++b) ids[b] = b < cnt ? s0 + b : s0;
        MCK(cudaMemcpyAsync(mm->idx.p, ids.data(), Bw * sizeof(int64_t), cudaMemcpyHostToDevice, mm->st));
        k_features<<<(Bw + 127) / 128, 128, 0, mm->st>>>(Bw, n, px.p, pr.p, ps.p, nullptr, mm->idx.p, 0, mm->counters.p + 1,
                                                        mm->X.p, nullptr, Bw, nullptr);
        ++mm->launches;
        MCK(enqueue_forward(mm, Bw, cnt, false));
        MCK(cudaMemcpyAsync(out + 4 * s0, mm->pred.p, (size_t)cnt * 4 * sizeof(float), cudaMemcpyDeviceToHost, mm->st));
        MCK(cudaStreamSynchronize(mm->st));  // ids is reused
    }
    return check_err(mm);
}

int rbf_mlp_warm_start(rbf_mlp *mm, rbf_ctx *ctx, const double *scale) {
    if (!mm || !ctx || !scale) return RBF_EINVAL;
    if (!ctx->inited || ctx->solver != RBF_SOLVER_ACM) return mfail(mm, RBF_EINVAL, "rbf_mlp_warm_start: needs an initialised ACM context");
    if (!ctx->has_sphere) return mfail(mm, RBF_EINVAL, "rbf_mlp_warm_start: the context has no sphere");
    if (ctx->device != mm->device) return mfail(mm, RBF_EINVAL, "rbf_mlp_warm_start: different devices");
    MDevGuard dg(mm->device);
    const int64_t n = ctx->n;
    // order the context's stream after the network's
    MCK(cudaStreamSynchronize(ctx->st));
    int rc = ensure_workspace(mm, std::max(mm->B, 16384));
    if (rc) return rc;
    const int Bw = mm->B;
    DevArr<float> rad, sdf, predall;
    MCK(rad.alloc(n)); MCK(sdf.alloc(n)); MCK(predall.alloc(4 * n));
    k_node_geo<<<(unsigned)((n + 255) / 256), 256, 0, mm->st>>>(n, ctx->xyz.p, ctx->c[0], ctx->c[1], ctx->c[2], ctx->r, rad.p, sdf.p);
    ++mm->launches;
    std::vector<int64_t> ids(Bw);
    for (int64_t s0 = 0; s0 < n; s0 += Bw) {
        const int cnt = (int)std::min<int64_t>(Bw, n - s0);
        for (int b = 0; b < Bw; ++b) ids[b] = b < cnt ? s0 + b : s0;
        MCK(cudaMemcpyAsync(mm->idx.p, ids.data(), Bw * sizeof(int64_t), cudaMemcpyHostToDevice, mm->st));
        k_features<<<(Bw + 127) / 128, 128, 0, mm->st>>>(Bw, n, ctx->xyz.p, rad.p, sdf.p, nullptr, mm->idx.p, 0,
                                                        mm->counters.p + 1, mm->X.p, nullptr, Bw, nullptr);
        ++mm->launches;
        MCK(enqueue_forward(mm, Bw, cnt, false));
        MCK(cudaMemcpyAsync(predall.p + 4 * s0, mm->pred.p, (size_t)cnt * 4 * sizeof(float), cudaMemcpyDeviceToDevice, mm->st));
        MCK(cudaStreamSynchronize(mm->st));
    }
    const unsigned gb = (unsigned)((n + 255) / 256);
    const float4 sc = make_float4((float)scale[0], (float)scale[1], (float)scale[2], (float)scale[3]);
    if (ctx->prec != RBF_FP64)
        k_inject<float><<<gb, 256, 0, mm->st>>>(n, predall.p, ctx->type.p, sc, ctx->a32[0].p, ctx->a32[1].p, ctx->a32[2].p, ctx->a32[3].p);
    else
        k_inject<double><<<gb, 256, 0, mm->st>>>(n, predall.p, ctx->type.p, sc, ctx->a64[0].p, ctx->a64[1].p, ctx->a64[2].p, ctx->a64[3].p);
    ++mm->launches;
    if (ctx->prec == RBF_FP32C)
        for (int c = 0; c < 4; ++c) MCK(ctx->l32[c].zero(mm->st));
    MCK(cudaGetLastError());
    MCK(cudaStreamSynchronize(mm->st));
    // C of Eq. MNS_C from the new velocity, in the slot the next pressure sweep reads
    const int slot = (ctx->parity + 1) & 1;
    if (ctx->prec != RBF_FP64) {
        AcmArgs<float> a;
        std::memset(&a, 0, sizeof(a));
        a.n = n; a.u = ctx->a32[0].p; a.v = ctx->a32[1].p; a.w_ = ctx->a32[2].p; a.vmax = ctx->vmax.p;
        MCK(acm_launch_vmax<float>(a, slot, ctx->st));
    } else {
        AcmArgs<double> a;
        std::memset(&a, 0, sizeof(a));
        a.n = n; a.u = ctx->a64[0].p; a.v = ctx->a64[1].p; a.w_ = ctx->a64[2].p; a.vmax = ctx->vmax.p;
        MCK(acm_launch_vmax<double>(a, slot, ctx->st));
    }
    MCK(cudaStreamSynchronize(ctx->st));
    return check_err(mm);
}

int64_t rbf_mlp_launch_count(const rbf_mlp *mm) { return mm ? mm->launches : -1; }

int rbf_mlp_set_fused(rbf_mlp *mm, int fused) {
    if (!mm) return RBF_EINVAL;
    MDevGuard dg(mm->device);
    if (mm->st) MCK(cudaStreamSynchronize(mm->st));
    if (mm->gexec) {
        cudaGraphExecDestroy(mm->gexec);
        mm->gexec = nullptr;
    }
    mm->fused = fused != 0;
    return RBF_OK;
}

}  // extern "C"
