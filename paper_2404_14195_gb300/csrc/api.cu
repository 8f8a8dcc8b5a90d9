// api.cu — the C ABI of include/rbfgb.h: device-resident state of one case and
// the host-side orchestration of the kernels (node ordering, stencils, weights,
// time stepping with CUDA graphs, reductions).  No arithmetic of the method
// runs on the host; host code validates arguments, sizes buffers and launches.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "rbfgb.h"
#include "acm.cuh"
#include "acm_persist.cuh"
#include "ctx.cuh"
#include "internal.cuh"
#include "lbm.cuh"
#include "reduce.cuh"

using namespace rbf;

namespace {

int fail(rbf_ctx *c, int code, const std::string &msg) {
    if (c) c->err = msg;
    return code;
}
int cuda_fail(rbf_ctx *c, cudaError_t e, const char *where) {
    std::string m = std::string(where) + ": " + cudaGetErrorString(e);
    return fail(c, e == cudaErrorMemoryAllocation ? RBF_ENOMEM : RBF_ECUDA, m);
}

#define CK(call)                                                    \
    do {                                                            \
        cudaError_t e_ = (call);                                    \
        if (e_ != cudaSuccess) return cuda_fail(ctx, e_, #call);    \
    } while (0)

struct DeviceGuard {
    int prev = -1;
    explicit DeviceGuard(int d) {
        cudaGetDevice(&prev);
        if (prev != d) cudaSetDevice(d);
    }
    ~DeviceGuard() {
        int now = -1;
        cudaGetDevice(&now);
        if (prev >= 0 && now != prev) cudaSetDevice(prev);
    }
};

// FP32 storage (plain or compensated)
bool is_f32(const rbf_ctx *c) { return c->prec != RBF_FP64; }
// low words of ACM field c (0..3: u, v, w, p) of a compensated FP32 state, else null
const float *low_words(const rbf_ctx *c, int f) { return c->prec == RBF_FP32C ? c->l32[f].p : nullptr; }

// stored values of one LBM population buffer (either layout, padding included)
int64_t lbm_state_len(const rbf_ctx *c) { return (int64_t)lbm_rec_len(c->q) * c->npad; }
// FP64 schedule of the refined FP32 mode's refresh step: one node per thread on
// the layout of the current FP32 schedule
int refine_schedule(const rbf_ctx *c) {
    return c->lbm_layout == LBM_LAYOUT_NODES ? LBM_RECORD_PER_THREAD : LBM_NODE_PER_THREAD;
}
// The current LBM state as shifted populations in FP64 (refined FP32: base plus
// correction, written into the FP64 scratch f64[1]), or null when it is plain FP32
// (then read f32[cur]).
cudaError_t lbm_state64(rbf_ctx *c, const double **out) {
    *out = nullptr;
    if (c->prec == RBF_FP64) { *out = c->f64[c->cur].p; return cudaSuccess; }
    if (c->prec != RBF_FP32R) return cudaSuccess;
    ++c->launches;
    *out = c->f64[1].p;
    return lbm_launch_refine_combine(lbm_state_len(c), c->f64[0].p, c->f32[c->cur].p, c->f64[1].p, c->st);
}
// moments of the current LBM state into c->mac (lbm_launch_macro; the caller
// counts that launch, lbm_state64 counts its own)
cudaError_t lbm_macro_current(rbf_ctx *c) {
    const double *f64 = nullptr;
    cudaError_t e = lbm_state64(c, &f64);
    if (e != cudaSuccess) return e;
    if (f64) return lbm_launch_macro<double>(c->n, c->npad, c->lbm_layout, c->q, f64, c->gl, c->mac.p, c->st);
    return lbm_launch_macro<float>(c->n, c->npad, c->lbm_layout, c->q, c->f32[c->cur].p, c->gl, c->mac.p, c->st);
}

int persistent_solve(std::vector<rbf_ctx *> &cs, const rbf_solve_opts *o, std::vector<int64_t> &steps,
                     std::vector<double> &resid, std::vector<int32_t> &done, std::string &err);
cudaError_t static_flux_lookup(double **out);

void drop_graph(rbf_ctx *ctx) {
    if (ctx->gexec) cudaGraphExecDestroy(ctx->gexec);
    ctx->gexec = nullptr;
    ctx->gsteps = 0;
}

// Select an LBM schedule; an initialised state whose layout differs is rewritten
// into the other population buffer, which becomes the current one.
int switch_schedule(rbf_ctx *ctx, int variant) {
    const int to = lbm_layout_of(variant);
    if (ctx->inited && ctx->solver == RBF_SOLVER_LBM && to != ctx->lbm_layout) {
        drop_graph(ctx);
        const int c = ctx->cur;
        if (ctx->prec == RBF_FP32R) {
            // base + correction into the scratch, relaid out as the new base; zero
            // correction, and a refresh at the next step
            const double *f = nullptr;
            CK(lbm_state64(ctx, &f));
            CK(lbm_launch_relayout<double>(ctx->npad, ctx->q, ctx->lbm_layout, ctx->f64[1].p, to, ctx->f64[0].p, ctx->st));
            CK(ctx->f32[0].zero(ctx->st));
            CK(ctx->f32[1].zero(ctx->st));
            ctx->refine_phase = 0;
            ++ctx->launches;
        } else if (ctx->prec == RBF_FP64) {
            CK(lbm_launch_relayout<double>(ctx->npad, ctx->q, ctx->lbm_layout, ctx->f64[c].p, to, ctx->f64[c ^ 1].p, ctx->st));
            ++ctx->launches;
            ctx->cur = c ^ 1;
        } else {
            CK(lbm_launch_relayout<float>(ctx->npad, ctx->q, ctx->lbm_layout, ctx->f32[c].p, to, ctx->f32[c ^ 1].p, ctx->st));
            ++ctx->launches;
            ctx->cur = c ^ 1;
        }
    }
    ctx->lbm_layout = to;
    ctx->variant = variant;
    return RBF_OK;
}

int binom(int a, int b) {
    long r = 1;
    for (int i = 1; i <= b; ++i) r = r * (a - b + i) / i;
    return (int)r;
}

double porosity_of(double r) {
    double v = 4.0 / 3.0 * M_PI * r * r * r;
    if (r > 0.5) {
        double h = r - 0.5;
        v -= 6.0 * M_PI * h * h * (3.0 * r - h) / 3.0;
    }
    return 1.0 - v;
}
double wall_area_of(double r) {
    double a = 4.0 * M_PI * r * r;
    if (r > 0.5) a -= 6.0 * 2.0 * M_PI * r * (r - 0.5);
    return a;
}

__global__ void k_iota(int32_t *a, int64_t n) {
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i < n) a[i] = (int32_t)i;
}
__global__ void k_gather_rows(int64_t nr, int n_l, const int32_t *rows, const int32_t *idx, int32_t *out) {
    int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (t >= nr * n_l) return;
    int64_t r = t / n_l;
    int j = (int)(t - r * n_l);
    out[t] = idx[(int64_t)rows[r] * n_l + j];
}
__global__ void k_gather_wrows(int64_t nr, int n_l, int n_ops, const int32_t *rows, const double *w, double *out) {
    int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (t >= nr * 3 * n_l) return;
    int64_t r = t / (3 * n_l);
    int rem = (int)(t - r * 3 * n_l);
    out[t] = w[(int64_t)rows[r] * n_ops * n_l + rem];
}
// probe points on the five planes x = 0, .2, .4, .6, .8; flag = fluid (outside every
// periodic image of the sphere)
__global__ void k_probe_points(int m_p, double cx, double cy, double cz, double r, int has_sphere, double *pts,
                               int32_t *flag) {
    int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    int64_t tot = 5LL * m_p * m_p;
    if (t >= tot) return;
    int pl = (int)(t / ((int64_t)m_p * m_p));
    int rem = (int)(t - (int64_t)pl * m_p * m_p);
    int a = rem / m_p, b = rem - a * m_p;
    double x = 0.2 * pl, y = (a + 0.5) / m_p, z = (b + 0.5) / m_p;
    pts[3 * t] = x; pts[3 * t + 1] = y; pts[3 * t + 2] = z;
    int fl = 1;
    if (has_sphere) {
        double dx = mimg(x - cx), dy = mimg(y - cy), dz = mimg(z - cz);
        fl = sqrt(dx * dx + dy * dy + dz * dz) - r >= 0.0;
    }
    flag[t] = fl;
}
__global__ void k_probe_compact(int64_t tot, const double *pts, const int32_t *flag, const int32_t *scan, double *out) {
    int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (t >= tot || !flag[t]) return;
    int64_t o = scan[t];
    out[3 * o] = pts[3 * t]; out[3 * o + 1] = pts[3 * t + 1]; out[3 * o + 2] = pts[3 * t + 2];
}

unsigned nblk(int64_t n, int b = 256) { return (unsigned)((n + b - 1) / b); }

template <typename T>
AcmArgs<T> acm_args(rbf_ctx *ctx, DevArr<T> *a, const DevArr<T> &ws, const DevArr<T> &wn) {
    AcmArgs<T> g;
    g.n = ctx->n; g.nb = ctx->nb; g.n_l = ctx->n_l;
    g.idx = ctx->idx_sell.p; g.w = ws.p; g.type = ctx->type.p; g.wall = ctx->wall.p;
    g.idxb = ctx->idxb_sell.p; g.wn = wn.p;
    g.u = a[0].p; g.v = a[1].p; g.w_ = a[2].p; g.p = a[3].p;
    g.us = a[4].p; g.vs = a[5].p; g.ws = a[6].p;
    g.ul = g.vl = g.wl = g.pl = g.usl = g.vsl = g.wsl = nullptr;
    if constexpr (sizeof(T) == 4) {
        if (ctx->prec == RBF_FP32C) {
            DevArr<float> *l = ctx->l32;
            g.ul = l[0].p; g.vl = l[1].p; g.wl = l[2].p; g.pl = l[3].p; g.usl = l[4].p; g.vsl = l[5].p; g.wsl = l[6].p;
        }
    }
    g.vmax = ctx->vmax.p;
    g.dt = (T)ctx->dt; g.nu = (T)ctx->prm.nu;
    g.gx = (T)ctx->prm.g[0]; g.gy = (T)ctx->prm.g[1]; g.gz = (T)ctx->prm.g[2];
    g.rho = (T)ctx->rho; g.beta = ctx->beta; g.vref = ctx->vref;
    return g;
}

template <typename T>
LbmArgs<T> lbm_args(rbf_ctx *ctx, DevArr<T> *f, const DevArr<T> &ws, int cur) {
    LbmArgs<T> g;
    g.n = ctx->n; g.npad = ctx->npad; g.n_l = ctx->n_l; g.layout = ctx->lbm_layout;
    g.idx = ctx->idx_sell.p; g.w = ws.p; g.mask = ctx->mask.p;
    g.fin = f[cur].p; g.fout = f[cur ^ 1].p;
    g.tp_inv = (T)(1.0 / ctx->tp); g.tm_inv = (T)(1.0 / ctx->tm);
    g.gx = (T)ctx->gl[0]; g.gy = (T)ctx->gl[1]; g.gz = (T)ctx->gl[2];
    return g;
}

// enqueue `steps` steps starting from (parity, cur, refined-FP32 phase); updates
// them (phase: ctx->refine_phase when null)
cudaError_t enqueue_steps(rbf_ctx *ctx, int steps, int &parity, int &cur, int64_t *launches,
                          LaunchRecorder *rec = nullptr, int *phase = nullptr) {
    cudaError_t e = cudaSuccess;
    int &ph = phase ? *phase : ctx->refine_phase;
    for (int s = 0; s < steps && e == cudaSuccess; ++s) {
        if (ctx->solver == RBF_SOLVER_LBM && ctx->prec == RBF_FP32R) {
            // f = base + delta.  Refresh: fold delta into the base, one FP64 step of
            // the base into the scratch, r = fl(F(base) - base), delta = r (so this
            // step ends exactly at F(base)).  Other steps: delta <- S(delta) + r with
            // S the FP32 step without the body force (its forcing is inside r).
            const int64_t tot = lbm_state_len(ctx);
            if (ph == 0) {
                e = lbm_launch_refine_fold(tot, ctx->f64[0].p, ctx->f32[cur].p, ctx->st);
                if (e == cudaSuccess)
                    e = lbm_launch_step<double>(lbm_args<double>(ctx, ctx->f64, ctx->ws64, 0), ctx->q, ctx->st,
                                                refine_schedule(ctx));
                if (e == cudaSuccess)
                    e = lbm_launch_refine_residual(tot, ctx->f64[1].p, ctx->f64[0].p, ctx->rr.p, ctx->f32[cur ^ 1].p,
                                                   ctx->st);
                *launches += 3;
            } else {
                LbmArgs<float> a = lbm_args<float>(ctx, ctx->f32, ctx->ws32, cur);
                a.gx = a.gy = a.gz = 0.0f;
                a.radd = ctx->rr.p;
                if (rec) rec->begin(ctx->st, 0);
                e = lbm_launch_step<float>(a, ctx->q, ctx->st, ctx->variant);
                if (rec) rec->end(ctx->st);
                ++*launches;
            }
            cur ^= 1;
            ph = (ph + 1) % ctx->refine_m;
            continue;
        }
        if (ctx->solver == RBF_SOLVER_ACM) {
            if (is_f32(ctx)) e = acm_launch_step<float>(acm_args<float>(ctx, ctx->a32, ctx->ws32, ctx->wn32), ctx->n_p, parity, ctx->st, launches, rec, ctx->acm_code);
            else e = acm_launch_step<double>(acm_args<double>(ctx, ctx->a64, ctx->ws64, ctx->wn64), ctx->n_p, parity, ctx->st, launches, rec, ctx->acm_code);
            parity = (parity + ctx->n_p) & 1;
        } else {
            if (rec) rec->begin(ctx->st, 0);
            if (is_f32(ctx)) e = lbm_launch_step<float>(lbm_args<float>(ctx, ctx->f32, ctx->ws32, cur), ctx->q, ctx->st, ctx->variant);
            else e = lbm_launch_step<double>(lbm_args<double>(ctx, ctx->f64, ctx->ws64, cur), ctx->q, ctx->st, ctx->variant);
            if (rec) rec->end(ctx->st);
            ++*launches;
            cur ^= 1;
        }
    }
    return e;
}

int run_steps(rbf_ctx *ctx, int64_t nsteps) {
    // even: parity / buffer return to start; refined FP32: one refresh window, so
    // the refresh phase returns to start as well
    const bool refined = ctx->solver == RBF_SOLVER_LBM && ctx->prec == RBF_FP32R;
    const int chunk = ctx->solver == RBF_SOLVER_ACM ? 16 : (refined ? ctx->refine_m : 32);
    int64_t full = nsteps / chunk, rem = nsteps % chunk;
    int64_t kl = 0;
    if (full > 0) {
        const int ph0 = refined ? ctx->refine_phase : 0;
        if (!ctx->gexec || ctx->gparity != ctx->parity || ctx->gcur != ctx->cur || ctx->gprec != ctx->prec ||
            ctx->gsteps != chunk || ctx->gvariant != ctx->variant || ctx->gblock != ctx->acm_code ||
            ctx->gphase != ph0) {
            drop_graph(ctx);
            cudaGraph_t g;
            CK(cudaStreamBeginCapture(ctx->st, cudaStreamCaptureModeThreadLocal));
            int par = ctx->parity, cu = ctx->cur, ph = ph0;
            int64_t dummy = 0;
            cudaError_t e = enqueue_steps(ctx, chunk, par, cu, &dummy, nullptr, &ph);
            cudaError_t e2 = cudaStreamEndCapture(ctx->st, &g);
            if (e != cudaSuccess) return cuda_fail(ctx, e, "capture");
            if (e2 != cudaSuccess) return cuda_fail(ctx, e2, "cudaStreamEndCapture");
            e = cudaGraphInstantiate(&ctx->gexec, g, 0);
            cudaGraphDestroy(g);
            if (e != cudaSuccess) return cuda_fail(ctx, e, "cudaGraphInstantiate");
            ctx->gsteps = chunk;
            ctx->gparity = ctx->parity;
            ctx->gcur = ctx->cur;
            ctx->gprec = ctx->prec;
            ctx->gvariant = ctx->variant;
            ctx->gblock = ctx->acm_code;
            ctx->gphase = ph0;
            ctx->last_kernel_launches = dummy;
        }
        int64_t per_graph = ctx->last_kernel_launches;
        for (int64_t r = 0; r < full; ++r) {
            CK(cudaGraphLaunch(ctx->gexec, ctx->st));
            kl += per_graph;
        }
    }
    if (rem > 0) {
        cudaError_t e = enqueue_steps(ctx, (int)rem, ctx->parity, ctx->cur, &kl);
        if (e != cudaSuccess) return cuda_fail(ctx, e, "step launch");
    }
    ctx->launches += kl;
    return RBF_OK;
}

}  // namespace

// ===========================================================================
extern "C" {

int rbf_create(rbf_ctx **out, int device, void *cuda_stream) {
    if (!out) return RBF_EINVAL;
    *out = nullptr;
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || ndev <= 0 || device < 0 || device >= ndev) return RBF_ECUDA;
    rbf_ctx *ctx = new rbf_ctx();
    ctx->device = device;
    DeviceGuard dg(device);
    if (cuda_stream) {
        ctx->st = (cudaStream_t)cuda_stream;
    } else {
        if (cudaStreamCreateWithFlags(&ctx->st, cudaStreamNonBlocking) != cudaSuccess) { delete ctx; return RBF_ECUDA; }
        ctx->own_stream = true;
    }
    if (cudaEventCreate(&ctx->ev0) != cudaSuccess || cudaEventCreate(&ctx->ev1) != cudaSuccess ||
        ctx->vmax.alloc(2) != cudaSuccess || ctx->scal.alloc(16) != cudaSuccess || ctx->status.alloc(4) != cudaSuccess ||
        static_flux_lookup(&ctx->static_flux) != cudaSuccess) {
        rbf_destroy(ctx);
        return RBF_ECUDA;
    }
    *out = ctx;
    return RBF_OK;
}

int rbf_destroy(rbf_ctx *ctx) {
    if (!ctx) return RBF_EINVAL;
    {
        DeviceGuard dg(ctx->device);
        if (ctx->st) cudaStreamSynchronize(ctx->st);
        drop_graph(ctx);
        if (ctx->ev0) cudaEventDestroy(ctx->ev0);
        if (ctx->ev1) cudaEventDestroy(ctx->ev1);
        if (ctx->own_stream && ctx->st) cudaStreamDestroy(ctx->st);
        ctx->st = nullptr;
    }
    {
        DeviceGuard dg(ctx->device);
        delete ctx;  // DevArr destructors free device memory on this device
    }
    return RBF_OK;
}

const char *rbf_last_error(const rbf_ctx *ctx) { return ctx ? ctx->err.c_str() : "null context"; }

int64_t rbf_launch_count(const rbf_ctx *ctx) { return ctx ? ctx->launches : -1; }

int rbf_lbm_set_unknown_rule(rbf_ctx *ctx, int rule) {
    if (!ctx) return RBF_EINVAL;
    if (rule != 0 && rule != 1) return fail(ctx, RBF_EINVAL, "rbf_lbm_set_unknown_rule: rule must be 0 or 1");
    if (rule == 1 && !ctx->has_sphere) return fail(ctx, RBF_EINVAL, "rbf_lbm_set_unknown_rule: the solid check needs rbf_set_sphere");
    DeviceGuard dg(ctx->device);
    ctx->lbm_rule = rule;
    if (ctx->weights_ok && ctx->solver == RBF_SOLVER_LBM && ctx->mask.p) {
        if (rule == 1) CK(lbm_launch_masks_solid(ctx->n, ctx->q, ctx->type.p, ctx->xyz.p, ctx->c, ctx->r, ctx->dx, ctx->mask.p, ctx->st));
        else CK(lbm_launch_masks(ctx->n, ctx->q, ctx->type.p, ctx->nrm.p, ctx->mask.p, ctx->st));
        ++ctx->launches;
        CK(cudaStreamSynchronize(ctx->st));
    }
    return RBF_OK;
}

int rbf_lbm_get_unknown_mask(rbf_ctx *ctx, uint32_t *mask) {
    if (!ctx || !mask) return RBF_EINVAL;
    if (!(ctx->weights_ok && ctx->solver == RBF_SOLVER_LBM && ctx->mask.p))
        return fail(ctx, RBF_EINVAL, "rbf_lbm_get_unknown_mask: no LBM weights");
    DeviceGuard dg(ctx->device);
    if (ctx->stage.n * sizeof(double) < (size_t)ctx->n * sizeof(uint32_t)) CK(ctx->stage.alloc((size_t)std::max<int64_t>(4, ctx->q) * ctx->n));
    uint32_t *tmp = reinterpret_cast<uint32_t *>(ctx->stage.p);
    CK(launch_scatter_u32(ctx->n, ctx->perm.p, ctx->mask.p, tmp, ctx->st));
    ++ctx->launches;
    CK(cudaMemcpyAsync(mask, tmp, ctx->n * sizeof(uint32_t), cudaMemcpyDeviceToHost, ctx->st));
    CK(cudaStreamSynchronize(ctx->st));
    return RBF_OK;
}

int rbf_time_step(rbf_ctx *ctx, double *dt) {
    if (!ctx || !dt) return RBF_EINVAL;
    if (!ctx->inited) return fail(ctx, RBF_EINVAL, "rbf_time_step: not initialised");
    *dt = ctx->dt;
    return RBF_OK;
}

int rbf_set_nodes(rbf_ctx *ctx, int64_t n, const double *xyz, const uint8_t *type, const double *normal) {
    if (!ctx) return RBF_EINVAL;
    if (n < 2 || n > (int64_t)INT32_MAX / 64 || !xyz || !type) return fail(ctx, RBF_EINVAL, "rbf_set_nodes: bad n or null array");
    int64_t nb = 0;
    for (int64_t i = 0; i < n; ++i) {
        for (int a = 0; a < 3; ++a) {
            double x = xyz[3 * i + a];
            if (!(x >= 0.0 && x <= 1.0)) return fail(ctx, RBF_EINVAL, "rbf_set_nodes: coordinates must lie in [0, 1]");
        }
        if (type[i] > 1) return fail(ctx, RBF_EINVAL, "rbf_set_nodes: type must be 0 (fluid) or 1 (wall)");
        if (type[i]) {
            if (!normal) return fail(ctx, RBF_EINVAL, "rbf_set_nodes: wall nodes need normals");
            double l = std::sqrt(normal[3 * i] * normal[3 * i] + normal[3 * i + 1] * normal[3 * i + 1] +
                                 normal[3 * i + 2] * normal[3 * i + 2]);
            if (!(std::fabs(l - 1.0) < 1e-6)) return fail(ctx, RBF_EINVAL, "rbf_set_nodes: wall normals must be unit");
            ++nb;
        }
    }
    DeviceGuard dg(ctx->device);
    CK(cudaStreamSynchronize(ctx->st));
    drop_graph(ctx);
    ctx->weights_ok = false;
    ctx->inited = false;
    ctx->n_l = 0;
    ctx->m_p = 0;
    ctx->n = n;
    ctx->npad = (n + 31) & ~31LL;
    ctx->nb = nb;
    ctx->nf = n - nb;
    int64_t npow = 1;
    while (npow < n) npow <<= 1;
    DevArr<double> xyz0, nrm0;
    DevArr<uint8_t> type0;
    DevArr<uint64_t> keys;
    DevArr<int32_t> vals;
    CK(xyz0.alloc(3 * n)); CK(nrm0.alloc(3 * n)); CK(type0.alloc(n));
    CK(keys.alloc(npow)); CK(vals.alloc(npow));
    CK(cudaMemcpyAsync(xyz0.p, xyz, 3 * n * sizeof(double), cudaMemcpyHostToDevice, ctx->st));
    CK(cudaMemcpyAsync(type0.p, type, n, cudaMemcpyHostToDevice, ctx->st));
    if (normal) CK(cudaMemcpyAsync(nrm0.p, normal, 3 * n * sizeof(double), cudaMemcpyHostToDevice, ctx->st));
    else CK(nrm0.zero(ctx->st));
    CK(launch_morton_keys(n, xyz0.p, keys.p, vals.p, npow, ctx->st));
    ++ctx->launches;
    CK(launch_bitonic_sort(keys.p, vals.p, npow, ctx->st, &ctx->launches));
    CK(ctx->xyz.alloc(3 * n)); CK(ctx->nrm.alloc(3 * n)); CK(ctx->type.alloc(n));
    CK(ctx->perm.alloc(n)); CK(ctx->iperm.alloc(n)); CK(ctx->iota.alloc(n));
    CK(cudaMemcpyAsync(ctx->perm.p, vals.p, n * sizeof(int32_t), cudaMemcpyDeviceToDevice, ctx->st));
    CK(launch_gather_nodes(n, ctx->perm.p, xyz0.p, type0.p, nrm0.p, ctx->xyz.p, ctx->type.p, ctx->nrm.p,
                           ctx->iperm.p, ctx->st));
    k_iota<<<nblk(n), 256, 0, ctx->st>>>(ctx->iota.p, n);
    ctx->launches += 2;
    // wall list (sorted order)
    CK(ctx->wall.alloc(nb));
    if (nb > 0) {
        DevArr<int32_t> flags, scan, tmp;
        CK(flags.alloc(n)); CK(scan.alloc(n)); CK(tmp.alloc(scan_tmp_len(n)));
        CK(launch_type_flags(n, ctx->type.p, 1, flags.p, ctx->st));
        CK(launch_scan_i32(flags.p, scan.p, n, tmp.p, tmp.n, ctx->st, &ctx->launches));
        CK(launch_flag_compact(n, ctx->type.p, 1, scan.p, ctx->wall.p, ctx->st));
        ctx->launches += 2;
        CK(cudaStreamSynchronize(ctx->st));
    }
    CK(cudaStreamSynchronize(ctx->st));
    CK(cudaGetLastError());
    return RBF_OK;
}

int rbf_set_sphere(rbf_ctx *ctx, const double c[3], double r) {
    if (!ctx || !c) return RBF_EINVAL;
    if (!(r > 0.0 && r < 0.7071)) return fail(ctx, RBF_EINVAL, "rbf_set_sphere: r must lie in (0, sqrt(2)/2)");
    for (int a = 0; a < 3; ++a) ctx->c[a] = c[a];
    ctx->r = r;
    ctx->has_sphere = true;
    ctx->m_p = 0;
    return RBF_OK;
}

int rbf_build_stencils(rbf_ctx *ctx, int n_l) {
    if (!ctx) return RBF_EINVAL;
    if (ctx->n == 0) return fail(ctx, RBF_EINVAL, "rbf_build_stencils: no nodes");
    if (n_l < 2 || n_l > RBF_MAX_NL || n_l > ctx->n) return fail(ctx, RBF_EINVAL, "rbf_build_stencils: need 2 <= n_l <= min(64, n)");
    if (ctx->nb > 0 && ctx->nf < n_l - 1) return fail(ctx, RBF_EINVAL, "rbf_build_stencils: too few fluid nodes for the wall stencils");
    DeviceGuard dg(ctx->device);
    drop_graph(ctx);
    ctx->weights_ok = false;
    ctx->inited = false;
    ctx->m_p = 0;
    const int64_t n = ctx->n;
    int G = (int)std::lround(std::cbrt((double)n / 4.0));
    G = std::max(1, std::min(G, 400));
    ctx->G = G;
    const int64_t ncell = (int64_t)G * G * G;
    DevArr<int32_t> cell_of, counts, fill, tmp;
    CK(cell_of.alloc(n)); CK(counts.alloc(ncell + 1)); CK(fill.alloc(ncell));
    CK(ctx->cstart.alloc(ncell + 1)); CK(ctx->citems.alloc(n)); CK(tmp.alloc(scan_tmp_len(ncell + 1)));
    CK(counts.zero(ctx->st)); CK(fill.zero(ctx->st));
    CK(launch_cell_count(n, ctx->xyz.p, G, cell_of.p, counts.p, ctx->st));
    CK(launch_scan_i32(counts.p, ctx->cstart.p, ncell + 1, tmp.p, tmp.n, ctx->st, &ctx->launches));
    CK(launch_cell_fill(n, cell_of.p, ctx->cstart.p, fill.p, ctx->citems.p, ctx->st));
    ctx->launches += 2;
    CK(ctx->idx.alloc(n * n_l));
    CK(ctx->status.zero(ctx->st));
    CK(launch_knn(n, nullptr, ctx->iota.p, ctx->xyz.p, ctx->perm.p, ctx->type.p, 0, G, ctx->cstart.p,
                  ctx->citems.p, n_l, ctx->idx.p, n_l, 0, ctx->status.p, ctx->st));
    ++ctx->launches;
    CK(ctx->idxb.alloc(ctx->nb * n_l));
    CK(ctx->idxw.alloc(ctx->nb * n_l));
    if (ctx->nb > 0) {
        CK(cudaMemcpy2DAsync(ctx->idxb.p, n_l * sizeof(int32_t), ctx->wall.p, sizeof(int32_t), sizeof(int32_t),
                             ctx->nb, cudaMemcpyDeviceToDevice, ctx->st));
        CK(launch_knn(ctx->nb, nullptr, ctx->wall.p, ctx->xyz.p, ctx->perm.p, ctx->type.p, 1, G, ctx->cstart.p,
                      ctx->citems.p, n_l - 1, ctx->idxb.p, n_l, 1, ctx->status.p, ctx->st));
        k_gather_rows<<<nblk(ctx->nb * n_l), 256, 0, ctx->st>>>(ctx->nb, n_l, ctx->wall.p, ctx->idx.p, ctx->idxw.p);
        ctx->launches += 2;
    }
    int32_t stat = 0;
    CK(cudaMemcpyAsync(&stat, ctx->status.p, sizeof(int32_t), cudaMemcpyDeviceToHost, ctx->st));
    CK(cudaStreamSynchronize(ctx->st));
    if (stat) return fail(ctx, RBF_EINVAL, "rbf_build_stencils: not enough candidate nodes");
    CK(ctx->idx_sell.alloc(ctx->npad * n_l));
    CK(launch_pack_idx(n, n_l, ctx->idx.p, ctx->idx_sell.p, ctx->st));
    CK(ctx->idxb_sell.alloc(((ctx->nb + 31) & ~31LL) * n_l));
    CK(launch_pack_idx(ctx->nb, n_l, ctx->idxb.p, ctx->idxb_sell.p, ctx->st));
    ctx->launches += 2;
    ctx->n_l = n_l;
    CK(cudaStreamSynchronize(ctx->st));
    return RBF_OK;
}

int rbf_get_stencils(rbf_ctx *ctx, int32_t *idx) {
    if (!ctx || !idx) return RBF_EINVAL;
    if (!ctx->n_l) return fail(ctx, RBF_EINVAL, "rbf_get_stencils: no stencils");
    DeviceGuard dg(ctx->device);
    DevArr<int32_t> out;
    CK(out.alloc(ctx->n * ctx->n_l));
    CK(launch_export_stencils(ctx->n, ctx->n_l, ctx->perm.p, ctx->iperm.p, ctx->idx.p, out.p, ctx->st));
    ++ctx->launches;
    CK(cudaMemcpyAsync(idx, out.p, out.n * sizeof(int32_t), cudaMemcpyDeviceToHost, ctx->st));
    CK(cudaStreamSynchronize(ctx->st));
    return RBF_OK;
}

}  // extern "C"

// Weights of one context.  presolved: the node and wall weight systems were already
// solved into ctx->w64 / ctx->delta / ctx->wgb64 by a multi-cell launch (ACM only),
// with `ext_sing` singular systems; only the derived arrays and packs remain.
int compute_weights_impl(rbf_ctx *ctx, int phs_k, int mono_m, int solver, int q, double dx, rbf_weight_report *rep,
                         bool presolved, int64_t ext_sing) {
    if (!ctx) return RBF_EINVAL;
    if (!ctx->n_l) return fail(ctx, RBF_EINVAL, "rbf_compute_weights: build stencils first");
    if (phs_k < 3 || phs_k % 2 == 0 || phs_k > 9) return fail(ctx, RBF_EINVAL, "rbf_compute_weights: phs_k must be odd, 3..9");
    if (mono_m < 0 || mono_m > 4) return fail(ctx, RBF_EINVAL, "rbf_compute_weights: mono_m must lie in 0..4");
    const int np = binom(mono_m + 3, 3);
    if (ctx->n_l < np) return fail(ctx, RBF_EINVAL, "rbf_compute_weights: n_l < N_p");
    if (solver != RBF_SOLVER_ACM && solver != RBF_SOLVER_LBM) return fail(ctx, RBF_EINVAL, "rbf_compute_weights: bad solver");
    if (solver == RBF_SOLVER_LBM && (q != 15 && q != 19)) return fail(ctx, RBF_EINVAL, "rbf_compute_weights: q must be 15 or 19");
    if (solver == RBF_SOLVER_LBM && !(dx > 0.0 && dx < 0.25)) return fail(ctx, RBF_EINVAL, "rbf_compute_weights: bad dx");
    DeviceGuard dg(ctx->device);
    drop_graph(ctx);
    ctx->weights_ok = false;
    ctx->inited = false;
    const int64_t n = ctx->n, nb = ctx->nb;
    const int n_l = ctx->n_l;
    std::vector<OpSpec> ops;
    if (solver == RBF_SOLVER_ACM) {
        for (int kind : {OP_DX, OP_DY, OP_DZ, OP_LAP}) ops.push_back(OpSpec{kind, {0.0, 0.0, 0.0}});
    } else {
        const int *e = host_velocity_set(q);
        for (int k = 1; k < q; ++k)
            ops.push_back(OpSpec{OP_INTERP, {-dx * e[3 * k], -dx * e[3 * k + 1], -dx * e[3 * k + 2]}});
    }
    std::vector<OpSpec> gops;
    for (int kind : {OP_DX, OP_DY, OP_DZ}) gops.push_back(OpSpec{kind, {0.0, 0.0, 0.0}});
    const int n_ops = (int)ops.size();
    DevArr<OpSpec> d_ops, d_gops;
    CK(d_ops.alloc(ops.size())); CK(d_gops.alloc(3));
    CK(cudaMemcpyAsync(d_ops.p, ops.data(), ops.size() * sizeof(OpSpec), cudaMemcpyHostToDevice, ctx->st));
    CK(cudaMemcpyAsync(d_gops.p, gops.data(), 3 * sizeof(OpSpec), cudaMemcpyHostToDevice, ctx->st));
    if (presolved && solver != RBF_SOLVER_ACM) return fail(ctx, RBF_EINVAL, "presolved weights: ACM only");
    CK(ctx->status.zero(ctx->st));
    if (!presolved) {
        CK(ctx->w64.alloc(n * n_ops * n_l));
        CK(ctx->delta.alloc(n));
        CK(launch_weights(n, ctx->xyz.p, nullptr, ctx->iota.p, 1, n_l, ctx->idx.p, phs_k, mono_m, n_ops, d_ops.p, 1,
                          ctx->w64.p, ctx->delta.p, ctx->status.p, ctx->st));
        ++ctx->launches;
        CK(ctx->wgb64.alloc(nb * 3 * n_l));
    }
    CK(ctx->wgw64.alloc(nb * 3 * n_l));
    if (nb > 0) {
        if (solver == RBF_SOLVER_ACM) {
            k_gather_wrows<<<nblk(nb * 3 * n_l), 256, 0, ctx->st>>>(nb, n_l, 4, ctx->wall.p, ctx->w64.p, ctx->wgw64.p);
            ++ctx->launches;
            if (!presolved)
                CK(launch_weights(nb, ctx->xyz.p, nullptr, ctx->wall.p, 1, n_l, ctx->idxb.p, phs_k, mono_m, 3, d_gops.p,
                                  1, ctx->wgb64.p, nullptr, ctx->status.p + 1, ctx->st));
        } else {
            CK(launch_weights(nb, ctx->xyz.p, nullptr, ctx->wall.p, 1, n_l, ctx->idxw.p, phs_k, mono_m, 3, d_gops.p, 1,
                              ctx->wgw64.p, nullptr, ctx->status.p + 1, ctx->st));
        }
        ++ctx->launches;
    }
    if (ctx->partial.n < (size_t)(4 * (nblk(n) + 8))) CK(ctx->partial.alloc(4 * (nblk(n) + 8)));
    CK(launch_min_f64(ctx->delta.p, n, ctx->partial.p, ctx->scal.p, ctx->st));
    ctx->launches += 2;
    int32_t sing[2] = {0, 0};
    double hmin = 0.0;
    CK(cudaMemcpyAsync(sing, ctx->status.p, 2 * sizeof(int32_t), cudaMemcpyDeviceToHost, ctx->st));
    CK(cudaMemcpyAsync(&hmin, ctx->scal.p, sizeof(double), cudaMemcpyDeviceToHost, ctx->st));
    CK(cudaStreamSynchronize(ctx->st));
    // SELL packs in both precisions
    const int n_out = n_ops;
    CK(ctx->ws32.alloc(ctx->npad * n_out * n_l));
    CK(ctx->ws64.alloc(ctx->npad * n_out * n_l));
    {
        // the FP32 pack is made from rows rounded with their sums kept
        DevArr<double> wr;
        CK(wr.alloc(n * n_ops * n_l));
        CK(launch_round_rows_f32(n * n_ops, n_l, ctx->w64.p, wr.p, ctx->st));
        if (solver == RBF_SOLVER_ACM) {
            CK(launch_pack_f32(n, n_ops, 0, n_out, n_l, wr.p, ctx->ws32.p, ctx->st));
            CK(launch_pack_f64(n, n_ops, 0, n_out, n_l, ctx->w64.p, ctx->ws64.p, ctx->st));
        } else {
            CK(lbm_launch_pack_f32(n, q, n_l, wr.p, ctx->ws32.p, ctx->st));
            CK(lbm_launch_pack_f64(n, q, n_l, ctx->w64.p, ctx->ws64.p, ctx->st));
        }
        ctx->launches += 3;
        CK(cudaStreamSynchronize(ctx->st));  // wr is freed on return
    }
    const int64_t nbpad = (nb + 31) & ~31LL;
    if (solver == RBF_SOLVER_ACM) {
        CK(ctx->wn32.alloc(nbpad * n_l));
        CK(ctx->wn64.alloc(nbpad * n_l));
        {
            DevArr<double> nr, nrr;
            CK(nr.alloc(nb * n_l));
            CK(nrr.alloc(nb * n_l));
            CK(launch_normal_rows(nb, n_l, ctx->wall.p, ctx->nrm.p, ctx->wgb64.p, nr.p, ctx->st));
            CK(launch_round_rows_f32(nb, n_l, nr.p, nrr.p, ctx->st));
            CK(launch_pack_f32(nb, 1, 0, 1, n_l, nrr.p, ctx->wn32.p, ctx->st));
            CK(cudaStreamSynchronize(ctx->st));  // nr, nrr are freed on return
        }
        CK(launch_pack_normal_f64(nb, n_l, ctx->wall.p, ctx->nrm.p, ctx->wgb64.p, ctx->wn64.p, ctx->st));
        ctx->launches += 4;
        ctx->mask.release();
    } else {
        ctx->wn32.release();
        ctx->wn64.release();
        if (ctx->lbm_rule == 1 && !ctx->has_sphere) return fail(ctx, RBF_EINVAL, "rbf_compute_weights: the solid-check rule needs rbf_set_sphere");
        CK(ctx->mask.alloc(n));
        if (ctx->lbm_rule == 1) CK(lbm_launch_masks_solid(n, q, ctx->type.p, ctx->xyz.p, ctx->c, ctx->r, dx, ctx->mask.p, ctx->st));
        else CK(lbm_launch_masks(n, q, ctx->type.p, ctx->nrm.p, ctx->mask.p, ctx->st));
        ++ctx->launches;
    }
    CK(cudaStreamSynchronize(ctx->st));
    ctx->solver = solver;
    ctx->q = solver == RBF_SOLVER_LBM ? q : 0;
    ctx->dx = dx;
    ctx->phs_k = phs_k;
    ctx->mono_m = mono_m;
    ctx->n_ops = n_ops;
    ctx->h_min = hmin;
    ctx->m_p = 0;
    if (rep) {
        rep->n_systems = n + nb;
        rep->n_singular = sing[0] + sing[1] + ext_sing;
        rep->h_min = hmin;
    }
    if (sing[0] + sing[1] + ext_sing > 0) return fail(ctx, RBF_ESINGULAR, "rbf_compute_weights: singular stencil systems");
    ctx->weights_ok = true;
    return RBF_OK;
}

extern "C" {

int rbf_compute_weights(rbf_ctx *ctx, int phs_k, int mono_m, int solver, int q, double dx, rbf_weight_report *rep) {
    return compute_weights_impl(ctx, phs_k, mono_m, solver, q, dx, rep, false, 0);
}

int rbf_get_weights(rbf_ctx *ctx, int op, double *out) {
    if (!ctx || !out) return RBF_EINVAL;
    if (!ctx->weights_ok) return fail(ctx, RBF_EINVAL, "rbf_get_weights: no weights");
    int o;
    if (ctx->solver == RBF_SOLVER_ACM) {
        if (op < RBF_OP_DX || op > RBF_OP_LAP) return fail(ctx, RBF_EINVAL, "rbf_get_weights: bad op for ACM");
        o = op;
    } else {
        o = op - RBF_OP_LBM0 - 1;
        if (o < 0 || o >= ctx->q - 1) return fail(ctx, RBF_EINVAL, "rbf_get_weights: bad op for LBM");
    }
    DeviceGuard dg(ctx->device);
    DevArr<double> d;
    CK(d.alloc(ctx->n * ctx->n_l));
    CK(launch_export_weights(ctx->n, ctx->n_l, ctx->n_ops, o, ctx->iperm.p, nullptr, ctx->w64.p, d.p, ctx->st));
    ++ctx->launches;
    CK(cudaMemcpyAsync(out, d.p, d.n * sizeof(double), cudaMemcpyDeviceToHost, ctx->st));
    CK(cudaStreamSynchronize(ctx->st));
    return RBF_OK;
}

int rbf_init(rbf_ctx *ctx, const rbf_params *p) {
    if (!ctx || !p) return RBF_EINVAL;
    if (!ctx->weights_ok) return fail(ctx, RBF_EINVAL, "rbf_init: compute weights first");
    if (p->precision != RBF_FP32 && p->precision != RBF_FP64 && p->precision != RBF_FP32C &&
        p->precision != RBF_FP32R)
        return fail(ctx, RBF_EINVAL, "rbf_init: bad precision");
    if (p->precision == RBF_FP32C && ctx->solver != RBF_SOLVER_ACM)
        return fail(ctx, RBF_EINVAL, "rbf_init: RBF_FP32C applies to the ACM solver only");
    if (p->precision == RBF_FP32R && ctx->solver != RBF_SOLVER_LBM)
        return fail(ctx, RBF_EINVAL, "rbf_init: RBF_FP32R applies to the LBM solver only");
    if (!(p->nu > 0.0)) return fail(ctx, RBF_EINVAL, "rbf_init: nu must be > 0");
    DeviceGuard dg(ctx->device);
    CK(cudaStreamSynchronize(ctx->st));
    drop_graph(ctx);
    ctx->prm = *p;
    ctx->prec = p->precision;
    ctx->rho = p->rho > 0.0 ? p->rho : 1.0;
    ctx->prm.rho = ctx->rho;
    const double gmag = std::sqrt(p->g[0] * p->g[0] + p->g[1] * p->g[1] + p->g[2] * p->g[2]);
    const int64_t n = ctx->n, npad = ctx->npad;
    for (auto &a : ctx->a32) a.release();
    for (auto &a : ctx->l32) a.release();
    for (auto &a : ctx->a64) a.release();
    for (auto &a : ctx->f32) a.release();
    for (auto &a : ctx->f64) a.release();
    ctx->rr.release();
    ctx->refine_phase = 0;
    if (ctx->solver == RBF_SOLVER_ACM) {
        const double cfl = p->cfl > 0.0 ? p->cfl : 0.1;
        ctx->dt = p->dt > 0.0 ? p->dt : cfl * ctx->h_min * ctx->h_min / (2.0 * p->nu);
        ctx->beta = p->beta > 0.0 ? p->beta : 10.0;
        ctx->vref = p->v_ref > 0.0 ? p->v_ref : 0.01 * gmag / p->nu;
        ctx->n_p = p->n_p > 0 ? p->n_p : 3;
        ctx->parity = 0;
        for (int a = 0; a < 10; ++a) {
            if (is_f32(ctx)) { CK(ctx->a32[a].alloc(npad)); CK(ctx->a32[a].zero(ctx->st)); }
            else { CK(ctx->a64[a].alloc(npad)); CK(ctx->a64[a].zero(ctx->st)); }
            if (ctx->prec == RBF_FP32C) { CK(ctx->l32[a].alloc(npad)); CK(ctx->l32[a].zero(ctx->st)); }
        }
        CK(ctx->vmax.zero(ctx->st));  // v = 0: max |v| = 0, C = beta v_ref
    } else {
        ctx->tp = p->tau_plus > 0.5 ? p->tau_plus : 0.8;
        const double magic = p->magic > 0.0 ? p->magic : 3.0 / 16.0;
        ctx->tm = 0.5 + magic / (ctx->tp - 0.5);
        const double nu_lb = (ctx->tp - 0.5) / 3.0;
        ctx->lbm_dt = nu_lb * ctx->dx * ctx->dx / p->nu;
        ctx->dt = ctx->lbm_dt;
        for (int a = 0; a < 3; ++a) ctx->gl[a] = p->g[a] * ctx->lbm_dt * ctx->lbm_dt / ctx->dx;
        ctx->cur = 0;
        ctx->lbm_layout = lbm_layout_of(ctx->variant);
        const int64_t sz = (int64_t)lbm_rec_len(ctx->q) * npad;  // room for either layout
        if (ctx->prec == RBF_FP32R) {
            // base = the initial state in FP64, correction and residual zero
            CK(ctx->f64[0].alloc(sz)); CK(ctx->f64[1].alloc(sz)); CK(ctx->f64[0].zero(ctx->st));
            LbmArgs<double> a = lbm_args<double>(ctx, ctx->f64, ctx->ws64, 1);  // writes f64[0]
            CK(lbm_launch_init<double>(a, ctx->q, ctx->st));
            CK(ctx->f32[0].alloc(sz)); CK(ctx->f32[1].alloc(sz)); CK(ctx->rr.alloc(sz));
            CK(ctx->f32[0].zero(ctx->st)); CK(ctx->f32[1].zero(ctx->st)); CK(ctx->rr.zero(ctx->st));
        } else if (is_f32(ctx)) {
            CK(ctx->f32[0].alloc(sz)); CK(ctx->f32[1].alloc(sz)); CK(ctx->f32[1].zero(ctx->st));
            LbmArgs<float> a = lbm_args<float>(ctx, ctx->f32, ctx->ws32, 1);  // writes f32[0]
            CK(lbm_launch_init<float>(a, ctx->q, ctx->st));
        } else {
            CK(ctx->f64[0].alloc(sz)); CK(ctx->f64[1].alloc(sz)); CK(ctx->f64[1].zero(ctx->st));
            LbmArgs<double> a = lbm_args<double>(ctx, ctx->f64, ctx->ws64, 1);
            CK(lbm_launch_init<double>(a, ctx->q, ctx->st));
        }
        ++ctx->launches;
    }
    CK(ctx->mac.alloc(4 * n));
    CK(ctx->stage.alloc((size_t)std::max(4, ctx->q) * n));
    {
        const size_t need = (size_t)(8 * (std::max<int64_t>(n, 5LL * 512 * 512) / 256 + 8));
        if (ctx->partial.n < need) CK(ctx->partial.alloc(need));
    }
    CK(cudaStreamSynchronize(ctx->st));
    ctx->inited = true;
    return RBF_OK;
}

int rbf_step(rbf_ctx *ctx, int nsteps) {
    if (!ctx) return RBF_EINVAL;
    if (!ctx->inited) return fail(ctx, RBF_EINVAL, "rbf_step: call rbf_init first");
    if (nsteps < 0) return fail(ctx, RBF_EINVAL, "rbf_step: nsteps < 0");
    DeviceGuard dg(ctx->device);
    CK(cudaEventRecord(ctx->ev0, ctx->st));
    int rc = run_steps(ctx, nsteps);
    if (rc) return rc;
    CK(cudaEventRecord(ctx->ev1, ctx->st));
    ctx->last_steps = nsteps;
    CK(cudaGetLastError());
    return RBF_OK;
}

int rbf_last_step_timing(rbf_ctx *ctx, double *total_ms, double *kernel_ms, int64_t *kernel_launches) {
    if (!ctx) return RBF_EINVAL;
    DeviceGuard dg(ctx->device);
    CK(cudaEventSynchronize(ctx->ev1));
    float ms = 0.f;
    CK(cudaEventElapsedTime(&ms, ctx->ev0, ctx->ev1));
    if (total_ms) *total_ms = ms;
    if (kernel_ms) *kernel_ms = ctx->last_steps ? ms / ctx->last_steps : 0.0;
    if (kernel_launches) *kernel_launches = ctx->last_steps;
    return RBF_OK;
}

int rbf_set_kernel_variant(rbf_ctx *ctx, int variant) {
    if (!ctx) return RBF_EINVAL;
    if (ctx->weights_ok && ctx->solver == RBF_SOLVER_ACM) {
        if (!acm_code_ok(variant)) return fail(ctx, RBF_EINVAL, "rbf_set_kernel_variant: ACM schedule code not in {64, 128, 256} + 1000 x {0, 2, 4}");
        drop_graph(ctx);
        ctx->acm_code = variant;
        return RBF_OK;
    }
    if (variant < 0 || variant >= LBM_N_SCHEDULES)
        return fail(ctx, RBF_EINVAL, "rbf_set_kernel_variant: schedule code out of range");
    DeviceGuard dg(ctx->device);
    const int rc = switch_schedule(ctx, variant);
    return rc;
}

namespace {
// snapshot / restore of the stepping state around autotuning trials
struct StateCopy {
    std::vector<DevArr<char> *> bufs;
    std::vector<std::pair<void *, size_t>> src;
    ~StateCopy() { for (auto *b : bufs) delete b; }
};
int save_state(rbf_ctx *ctx, StateCopy &sc) {
    auto add = [&](void *p, size_t bytes) -> cudaError_t {
        if (!p || !bytes) return cudaSuccess;
        auto *b = new DevArr<char>();
        sc.bufs.push_back(b);
        cudaError_t e = b->alloc(bytes);
        if (e != cudaSuccess) return e;
        sc.src.push_back({p, bytes});
        return cudaMemcpyAsync(b->p, p, bytes, cudaMemcpyDeviceToDevice, ctx->st);
    };
    for (int i = 0; i < 10; ++i) {
        CK(add(ctx->a32[i].p, ctx->a32[i].n * sizeof(float)));
        CK(add(ctx->l32[i].p, ctx->l32[i].n * sizeof(float)));
        CK(add(ctx->a64[i].p, ctx->a64[i].n * sizeof(double)));
    }
    for (int i = 0; i < 2; ++i) {
        CK(add(ctx->f32[i].p, ctx->f32[i].n * sizeof(float)));
        CK(add(ctx->f64[i].p, ctx->f64[i].n * sizeof(double)));
    }
    CK(add(ctx->rr.p, ctx->rr.n * sizeof(float)));
    CK(add(ctx->vmax.p, ctx->vmax.n * sizeof(unsigned long long)));
    return RBF_OK;
}
int restore_state(rbf_ctx *ctx, StateCopy &sc) {
    for (size_t i = 0; i < sc.src.size(); ++i)
        CK(cudaMemcpyAsync(sc.src[i].first, sc.bufs[i]->p, sc.src[i].second, cudaMemcpyDeviceToDevice, ctx->st));
    CK(cudaStreamSynchronize(ctx->st));
    return RBF_OK;
}
}  // namespace

int rbf_autotune(rbf_ctx *ctx, int trial_steps, rbf_tune_report *rep) {
    if (!ctx) return RBF_EINVAL;
    if (!ctx->inited) return fail(ctx, RBF_EINVAL, "rbf_autotune: call rbf_init first");
    if (trial_steps < 2 || trial_steps > 2000) return fail(ctx, RBF_EINVAL, "rbf_autotune: 2 <= trial_steps <= 2000");
    DeviceGuard dg(ctx->device);
    drop_graph(ctx);
    const int par0 = ctx->parity, cur0 = ctx->cur, lay0 = ctx->lbm_layout, ph0 = ctx->refine_phase;
    StateCopy sc;
    int rc = save_state(ctx, sc);
    if (rc) return rc;
    // back to the saved state: buffers, current buffer, layout
    auto back = [&]() -> int {
        const int r = restore_state(ctx, sc);
        ctx->parity = par0;
        ctx->cur = cur0;
        ctx->lbm_layout = lay0;
        ctx->refine_phase = ph0;
        return r;
    };
    std::vector<int> cands;
    if (ctx->solver == RBF_SOLVER_LBM)
        cands = {LBM_PAIR_PER_WARP, LBM_NODE_PER_THREAD, LBM_NODE_PER_THREAD_128, LBM_PAIR_PER_WARP_U3,
                 LBM_PAIR_PER_WARP_U6, LBM_PAIR_PER_WARP_U2, LBM_RECORD_PER_THREAD, LBM_RECORD_PER_THREAD_OCC,
                 LBM_RECORD_PER_THREAD_128, LBM_RECORD_PER_THREAD_64, LBM_RECORD_PER_THREAD_PDL};
    else
        cands = {256, 128, 64, 2128, 2256, 4128, 4256};
    rbf_tune_report r;
    std::memset(&r, 0, sizeof(r));
    double best = 1e300;
    int best_code = cands[0];
    for (size_t c = 0; c < cands.size() && c < RBF_TUNE_MAX; ++c) {
        if (ctx->solver == RBF_SOLVER_LBM) {
            rc = switch_schedule(ctx, cands[c]);
            if (rc) return rc;
        } else {
            ctx->acm_code = cands[c];
        }
        int64_t kl = 0;
        int par = ctx->parity, cu = ctx->cur, ph = ctx->refine_phase;
        cudaError_t e = enqueue_steps(ctx, 2, par, cu, &kl, nullptr, &ph);  // warm-up
        CK(e);
        CK(cudaEventRecord(ctx->ev0, ctx->st));
        e = enqueue_steps(ctx, trial_steps, par, cu, &kl, nullptr, &ph);
        CK(e);
        CK(cudaEventRecord(ctx->ev1, ctx->st));
        CK(cudaEventSynchronize(ctx->ev1));
        ctx->launches += kl;
        float ms = 0.f;
        CK(cudaEventElapsedTime(&ms, ctx->ev0, ctx->ev1));
        const double per = ms / trial_steps;
        r.code[c] = cands[c];
        r.ms_per_step[c] = per;
        r.n_candidates = (int)c + 1;
        if (per < best) { best = per; best_code = cands[c]; }
        rc = back();
        if (rc) return rc;
    }
    if (ctx->solver == RBF_SOLVER_LBM) {
        rc = switch_schedule(ctx, best_code);
        if (rc) return rc;
    } else {
        ctx->acm_code = best_code;
    }
    r.chosen = best_code;
    r.solver = ctx->solver;
    if (rep) *rep = r;
    return RBF_OK;
}

}  // extern "C"

namespace {
// schedule code of the persistent driver: block (32 .. 256) + 1000 group for a grid
// with `group` lanes per node (group 1: the code is the block size), -8 / -16 for a
// cluster; false for anything else
bool persist_code_ok(int code) {
    if (code == -8 || code == -16) return true;
    const int block = code % 1000, group = code / 1000;
    return (block == 32 || block == 64 || block == 128 || block == 256) &&
           (group == 0 || group == 2 || group == 4 || group == 8);
}
void set_persist_code(rbf_ctx *x, int code) {
    if (code < 0) {
        x->persist_cluster = -code;
        return;
    }
    x->persist_cluster = 0;
    x->persist_block = code % 1000;
    x->persist_group = code / 1000 ? code / 1000 : 1;
}

// Time the persistent driver over `cs` for every block size and keep the fastest
// in every cell; the cells' fields and parities are restored after each trial.
int tune_persistent(std::vector<rbf_ctx *> &cs, int trial_steps, rbf_tune_report *rep, std::string &err) {
    rbf_ctx *ctx = cs[0];
    std::vector<StateCopy> sc(cs.size());
    std::vector<int> par0(cs.size());
    for (size_t c = 0; c < cs.size(); ++c) {
        drop_graph(cs[c]);
        par0[c] = cs[c]->parity;
        int rc = save_state(cs[c], sc[c]);
        if (rc) { err = cs[c]->err; return rc; }
    }
    // grid schedules (code = threads per block + 1000 (lanes per node - 1 ... ) as
    // described at rbf_set_persistent_block) and, where the device can place them,
    // single clusters of 16 and 8 CTAs (codes -16, -8)
    std::vector<int> cands = {256, 128, 64, 32, 2128, 4128, 8128, 4256};
    for (int c : {16, 8}) {
        bool ok = false;
        if (is_f32(ctx)) CK(acm_persistent_cluster_ok<float>(c, ctx->prec == RBF_FP32C, &ok));
        else CK(acm_persistent_cluster_ok<double>(c, false, &ok));
        if (ok) cands.push_back(-c);
    }
    rbf_tune_report r;
    std::memset(&r, 0, sizeof(r));
    double best = 1e300;
    int best_code = cands[0];
    rbf_solve_opts o;
    std::memset(&o, 0, sizeof(o));
    o.tol = 1e-300;
    std::vector<int64_t> st;
    std::vector<double> rs;
    std::vector<int32_t> dn;
    for (int k = 0; k < (int)cands.size() && k < RBF_TUNE_MAX; ++k) {
        for (rbf_ctx *x : cs) set_persist_code(x, cands[k]);
        double ms = 0.0;
        for (int pass = 0; pass < 2; ++pass) {  // warm-up, then the timed trial
            o.max_steps = pass ? trial_steps : 2;
            o.check_every = (int)o.max_steps;
            const int rc = persistent_solve(cs, &o, st, rs, dn, err);
            if (rc) return rc;
            ms = ctx->persist_ms;
        }
        for (size_t c = 0; c < cs.size(); ++c) {
            cs[c]->parity = par0[c];
            const int rc = restore_state(cs[c], sc[c]);
            if (rc) { err = cs[c]->err; return rc; }
        }
        r.code[k] = cands[k];
        r.ms_per_step[k] = ms / trial_steps;
        r.n_candidates = k + 1;
        if (r.ms_per_step[k] < best) { best = r.ms_per_step[k]; best_code = cands[k]; }
    }
    for (rbf_ctx *x : cs) set_persist_code(x, best_code);
    r.chosen = best_code;
    r.solver = RBF_SOLVER_ACM;
    if (rep) *rep = r;
    return RBF_OK;
}
}  // namespace

extern "C" {

int rbf_set_persistent_block(rbf_ctx *ctx, int code) {
    if (!ctx) return RBF_EINVAL;
    if (!persist_code_ok(code))
        return fail(ctx, RBF_EINVAL, "rbf_set_persistent_block: code = block (32, 64, 128, 256) + 1000 x lanes per "
                                     "node (2, 4, 8; 0 for 1), or -8 / -16");
    set_persist_code(ctx, code);
    return RBF_OK;
}

int rbf_set_wait_limit(rbf_ctx *ctx, double seconds) {
    if (!ctx) return RBF_EINVAL;
    if (!(seconds >= 1e-9 && seconds <= 60.0)) return fail(ctx, RBF_EINVAL, "rbf_set_wait_limit: 1e-9 <= seconds <= 60");
    ctx->wait_ns = (uint64_t)std::llround(seconds * 1e9);
    if (ctx->wait_ns < 1) ctx->wait_ns = 1;
    return RBF_OK;
}

int rbf_autotune_persistent(rbf_ctx *ctx, int trial_steps, rbf_tune_report *rep) {
    if (!ctx) return RBF_EINVAL;
    if (!ctx->inited || ctx->solver != RBF_SOLVER_ACM)
        return fail(ctx, RBF_EINVAL, "rbf_autotune_persistent: needs an initialised ACM context");
    if (trial_steps < 2 || trial_steps > 20000) return fail(ctx, RBF_EINVAL, "rbf_autotune_persistent: 2 <= trial_steps <= 20000");
    DeviceGuard dg(ctx->device);
    std::vector<rbf_ctx *> cs{ctx};
    std::string msg;
    const int rc = tune_persistent(cs, trial_steps, rep, msg);
    return rc ? fail(ctx, rc, msg.empty() ? std::string("rbf_autotune_persistent failed") : msg) : RBF_OK;
}

int rbf_profile_steps(rbf_ctx *ctx, int nsteps, double *kernel_ms, int *n_classes) {
    if (!ctx || !kernel_ms) return RBF_EINVAL;
    if (!ctx->inited) return fail(ctx, RBF_EINVAL, "rbf_profile_steps: not initialised");
    if (nsteps < 1 || nsteps > 4096) return fail(ctx, RBF_EINVAL, "rbf_profile_steps: 1 <= nsteps <= 4096");
    DeviceGuard dg(ctx->device);
    const int per_step = ctx->solver == RBF_SOLVER_ACM ? 1 + 3 * ctx->n_p : 1;
    const int cap = nsteps * per_step;
    std::vector<cudaEvent_t> ev(2 * cap, nullptr);
    std::vector<int> cls(cap, 0);
    for (auto &e : ev) CK(cudaEventCreate(&e));
    LaunchRecorder rec;
    rec.ev = ev.data();
    rec.cls = cls.data();
    rec.cap = cap;
    int64_t kl = 0;
    cudaError_t e = enqueue_steps(ctx, nsteps, ctx->parity, ctx->cur, &kl, &rec);
    ctx->launches += kl;
    cudaError_t es = cudaStreamSynchronize(ctx->st);
    const int ncls = ctx->solver == RBF_SOLVER_ACM ? 4 : 1;
    double sum[4] = {0, 0, 0, 0};
    int cnt[4] = {0, 0, 0, 0};
    for (int i = 0; i < rec.count && e == cudaSuccess && es == cudaSuccess; ++i) {
        float ms = 0.f;
        if (cudaEventElapsedTime(&ms, ev[2 * i], ev[2 * i + 1]) == cudaSuccess) {
            sum[cls[i]] += ms;
            ++cnt[cls[i]];
        }
    }
    for (auto &x : ev) cudaEventDestroy(x);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "rbf_profile_steps launch");
    if (es != cudaSuccess) return cuda_fail(ctx, es, "rbf_profile_steps sync");
    for (int c = 0; c < ncls; ++c) kernel_ms[c] = cnt[c] ? sum[c] / cnt[c] : 0.0;
    if (n_classes) *n_classes = ncls;
    return RBF_OK;
}

int rbf_get_fields(rbf_ctx *ctx, double *uvwp) {
    if (!ctx || !uvwp) return RBF_EINVAL;
    if (!ctx->inited) return fail(ctx, RBF_EINVAL, "rbf_get_fields: not initialised");
    DeviceGuard dg(ctx->device);
    DevArr<double> &out = ctx->stage;
    if (ctx->solver == RBF_SOLVER_ACM) {
        if (ctx->prec == RBF_FP32C) CK(launch_acm_export_pair(ctx->n, ctx->perm.p, ctx->a32[0].p, ctx->a32[1].p, ctx->a32[2].p, ctx->a32[3].p, ctx->l32[0].p, ctx->l32[1].p, ctx->l32[2].p, ctx->l32[3].p, out.p, ctx->st));
        else if (is_f32(ctx)) CK(launch_acm_export<float>(ctx->n, ctx->perm.p, ctx->a32[0].p, ctx->a32[1].p, ctx->a32[2].p, ctx->a32[3].p, out.p, ctx->st));
        else CK(launch_acm_export<double>(ctx->n, ctx->perm.p, ctx->a64[0].p, ctx->a64[1].p, ctx->a64[2].p, ctx->a64[3].p, out.p, ctx->st));
        ++ctx->launches;
    } else {
        CK(lbm_macro_current(ctx));
        CK(launch_sum_f64(ctx->mac.p, ctx->n, 4, 4, ctx->partial.p, ctx->scal.p, ctx->st));
        const double vel = ctx->dx / ctx->lbm_dt, ps = ctx->rho * vel * vel;
        CK(launch_lbm_fields(ctx->n, ctx->perm.p, ctx->mac.p, vel, ps, ctx->scal.p + 3, out.p, ctx->st));
        ctx->launches += 4;
    }
    CK(cudaMemcpyAsync(uvwp, out.p, 4 * ctx->n * sizeof(double), cudaMemcpyDeviceToHost, ctx->st));
    CK(cudaStreamSynchronize(ctx->st));
    return RBF_OK;
}

int rbf_set_fields(rbf_ctx *ctx, const double *uvwp) {
    if (!ctx || !uvwp) return RBF_EINVAL;
    if (!ctx->inited) return fail(ctx, RBF_EINVAL, "rbf_set_fields: not initialised");
    if (ctx->solver != RBF_SOLVER_ACM) return fail(ctx, RBF_EINVAL, "rbf_set_fields: ACM only (use rbf_lbm_set_populations)");
    DeviceGuard dg(ctx->device);
    DevArr<double> &in = ctx->stage;
    CK(cudaMemcpyAsync(in.p, uvwp, 4 * ctx->n * sizeof(double), cudaMemcpyHostToDevice, ctx->st));
    const int slot = (ctx->parity + 1) & 1;  // read by the next pressure sweep
    if (is_f32(ctx)) {
        if (ctx->prec == RBF_FP32C) CK(launch_acm_import_pair(ctx->n, ctx->perm.p, ctx->a32[0].p, ctx->a32[1].p, ctx->a32[2].p, ctx->a32[3].p, ctx->l32[0].p, ctx->l32[1].p, ctx->l32[2].p, ctx->l32[3].p, in.p, ctx->st));
        else CK(launch_acm_import<float>(ctx->n, ctx->perm.p, ctx->a32[0].p, ctx->a32[1].p, ctx->a32[2].p, ctx->a32[3].p, in.p, ctx->st));
        CK(acm_launch_vmax<float>(acm_args<float>(ctx, ctx->a32, ctx->ws32, ctx->wn32), slot, ctx->st));
    } else {
        CK(launch_acm_import<double>(ctx->n, ctx->perm.p, ctx->a64[0].p, ctx->a64[1].p, ctx->a64[2].p, ctx->a64[3].p, in.p, ctx->st));
        CK(acm_launch_vmax<double>(acm_args<double>(ctx, ctx->a64, ctx->ws64, ctx->wn64), slot, ctx->st));
    }
    ctx->launches += 2;
    CK(cudaStreamSynchronize(ctx->st));
    return RBF_OK;
}

int rbf_lbm_get_populations(rbf_ctx *ctx, double *f) {
    if (!ctx || !f) return RBF_EINVAL;
    if (!ctx->inited || ctx->solver != RBF_SOLVER_LBM) return fail(ctx, RBF_EINVAL, "rbf_lbm_get_populations: no LBM state");
    DeviceGuard dg(ctx->device);
    DevArr<double> &out = ctx->stage;
    const double *f64 = nullptr;
    CK(lbm_state64(ctx, &f64));
    if (f64) CK(lbm_launch_export<double>(ctx->n, ctx->npad, ctx->lbm_layout, ctx->q, f64, ctx->perm.p, out.p, ctx->st));
    else CK(lbm_launch_export<float>(ctx->n, ctx->npad, ctx->lbm_layout, ctx->q, ctx->f32[ctx->cur].p, ctx->perm.p, out.p, ctx->st));
    ++ctx->launches;
    CK(cudaMemcpyAsync(f, out.p, (size_t)ctx->q * ctx->n * sizeof(double), cudaMemcpyDeviceToHost, ctx->st));
    CK(cudaStreamSynchronize(ctx->st));
    return RBF_OK;
}

int rbf_lbm_set_populations(rbf_ctx *ctx, const double *f) {
    if (!ctx || !f) return RBF_EINVAL;
    if (!ctx->inited || ctx->solver != RBF_SOLVER_LBM) return fail(ctx, RBF_EINVAL, "rbf_lbm_set_populations: no LBM state");
    DeviceGuard dg(ctx->device);
    DevArr<double> &in = ctx->stage;
    CK(cudaMemcpyAsync(in.p, f, (size_t)ctx->q * ctx->n * sizeof(double), cudaMemcpyHostToDevice, ctx->st));
    if (ctx->prec == RBF_FP32R) {  // the new state becomes the base; refresh at the next step
        CK(lbm_launch_import<double>(ctx->n, ctx->npad, ctx->lbm_layout, ctx->q, ctx->f64[0].p, ctx->perm.p, in.p, ctx->st));
        CK(ctx->f32[ctx->cur].zero(ctx->st));
        ctx->refine_phase = 0;
    } else if (is_f32(ctx)) {
        CK(lbm_launch_import<float>(ctx->n, ctx->npad, ctx->lbm_layout, ctx->q, ctx->f32[ctx->cur].p, ctx->perm.p, in.p, ctx->st));
    } else {
        CK(lbm_launch_import<double>(ctx->n, ctx->npad, ctx->lbm_layout, ctx->q, ctx->f64[ctx->cur].p, ctx->perm.p, in.p, ctx->st));
    }
    ++ctx->launches;
    CK(cudaStreamSynchronize(ctx->st));
    return RBF_OK;
}

namespace {
// Probe set of Eq. k_definition for m_p: built into local arrays and committed
// to the context (points, stencils, weights, fluid count, m_p) only once every
// step has succeeded, so a failed rebuild leaves the previous probe set whole.
int ensure_probes(rbf_ctx *ctx, int m_p) {
    if (ctx->m_p == m_p && ctx->pidx.p) return RBF_OK;
    const int64_t tot = 5LL * m_p * m_p;
    const int n_l = ctx->n_l;
    DevArr<double> pts, pxyz, pw;
    DevArr<int32_t> flag, scan, tmp, pidx;
    CK(pts.alloc(3 * tot)); CK(flag.alloc(tot + 1)); CK(scan.alloc(tot + 1)); CK(tmp.alloc(scan_tmp_len(tot + 1)));
    CK(flag.zero(ctx->st));
    k_probe_points<<<nblk(tot), 256, 0, ctx->st>>>(m_p, ctx->c[0], ctx->c[1], ctx->c[2], ctx->r, ctx->has_sphere, pts.p, flag.p);
    CK(launch_scan_i32(flag.p, scan.p, tot + 1, tmp.p, tmp.n, ctx->st, &ctx->launches));
    int32_t nfl = 0;
    CK(cudaMemcpyAsync(&nfl, scan.p + tot, sizeof(int32_t), cudaMemcpyDeviceToHost, ctx->st));
    CK(cudaStreamSynchronize(ctx->st));
    CK(pxyz.alloc(3 * std::max<int64_t>(nfl, 1)));
    k_probe_compact<<<nblk(tot), 256, 0, ctx->st>>>(tot, pts.p, flag.p, scan.p, pxyz.p);
    ctx->launches += 2;
    CK(pidx.alloc(std::max<int64_t>(nfl, 1) * n_l));
    CK(pw.alloc(std::max<int64_t>(nfl, 1) * n_l));
    CK(ctx->status.zero(ctx->st));
    if (nfl > 0) {
        CK(launch_knn(nfl, pxyz.p, nullptr, ctx->xyz.p, ctx->perm.p, ctx->type.p, 0, ctx->G, ctx->cstart.p,
                      ctx->citems.p, n_l, pidx.p, n_l, 0, ctx->status.p, ctx->st));
        OpSpec op{OP_INTERP, {0.0, 0.0, 0.0}};
        DevArr<OpSpec> d_op;
        CK(d_op.alloc(1));
        CK(cudaMemcpyAsync(d_op.p, &op, sizeof(OpSpec), cudaMemcpyHostToDevice, ctx->st));
        CK(launch_weights(nfl, ctx->xyz.p, pxyz.p, nullptr, 0, n_l, pidx.p, ctx->phs_k, ctx->mono_m, 1,
                          d_op.p, 1, pw.p, nullptr, ctx->status.p + 1, ctx->st));
        ctx->launches += 2;
    }
    int32_t st2[2] = {0, 0};
    CK(cudaMemcpyAsync(st2, ctx->status.p, 2 * sizeof(int32_t), cudaMemcpyDeviceToHost, ctx->st));
    CK(cudaStreamSynchronize(ctx->st));
    if (st2[0] || st2[1]) return fail(ctx, RBF_ESINGULAR, "probe stencils failed");
    ctx->pxyz.swap(pxyz);
    ctx->pidx.swap(pidx);
    ctx->pw.swap(pw);
    ctx->np_fluid = nfl;
    ctx->m_p = m_p;
    return RBF_OK;
}

// q = mean probe v_x (physical units), FP64
int probe_q(rbf_ctx *ctx, int m_p, double *qout) {
    int rc = ensure_probes(ctx, m_p);
    if (rc) return rc;
    if (ctx->solver == RBF_SOLVER_ACM) {
        if (is_f32(ctx)) CK(launch_probe_sum<float>(ctx->np_fluid, ctx->n_l, ctx->pidx.p, ctx->pw.p, ctx->a32[0].p, low_words(ctx, 0), 1, ctx->partial.p, ctx->scal.p + 4, ctx->st));
        else CK(launch_probe_sum<double>(ctx->np_fluid, ctx->n_l, ctx->pidx.p, ctx->pw.p, ctx->a64[0].p, nullptr, 1, ctx->partial.p, ctx->scal.p + 4, ctx->st));
        ctx->launches += 2;
    } else {
        CK(lbm_macro_current(ctx));
        CK(launch_probe_sum<double>(ctx->np_fluid, ctx->n_l, ctx->pidx.p, ctx->pw.p, ctx->mac.p, nullptr, 4, ctx->partial.p, ctx->scal.p + 4, ctx->st));
        ctx->launches += 3;
    }
    double s = 0.0;
    CK(cudaMemcpyAsync(&s, ctx->scal.p + 4, sizeof(double), cudaMemcpyDeviceToHost, ctx->st));
    CK(cudaStreamSynchronize(ctx->st));
    if (ctx->solver == RBF_SOLVER_LBM) s *= ctx->dx / ctx->lbm_dt;
    *qout = s / (5.0 * m_p * m_p);
    return RBF_OK;
}
}  // namespace

int rbf_permeability(rbf_ctx *ctx, int m_p, double *k_over_d2, double *q) {
    if (!ctx) return RBF_EINVAL;
    if (!ctx->inited) return fail(ctx, RBF_EINVAL, "rbf_permeability: not initialised");
    if (m_p < 1 || m_p > 512) return fail(ctx, RBF_EINVAL, "rbf_permeability: m_p must lie in 1..512");
    DeviceGuard dg(ctx->device);
    double qq = 0.0;
    int rc = probe_q(ctx, m_p, &qq);
    if (rc) return rc;
    const double *g = ctx->prm.g;
    const double gmag = std::sqrt(g[0] * g[0] + g[1] * g[1] + g[2] * g[2]);
    if (q) *q = qq;
    if (k_over_d2) *k_over_d2 = gmag > 0.0 ? qq * ctx->prm.nu / gmag : 0.0;
    return RBF_OK;
}

int rbf_drag(rbf_ctx *ctx, int m_p, double F[3], double *K) {
    if (!ctx || !F) return RBF_EINVAL;
    if (!ctx->inited) return fail(ctx, RBF_EINVAL, "rbf_drag: not initialised");
    if (!ctx->has_sphere) return fail(ctx, RBF_EINVAL, "rbf_drag: set the sphere first");
    DeviceGuard dg(ctx->device);
    const double mu = ctx->rho * ctx->prm.nu;
    if (ctx->solver == RBF_SOLVER_ACM) {
        if (is_f32(ctx)) {
            FieldView<float> f{ctx->a32[0].p, ctx->a32[1].p, ctx->a32[2].p, ctx->a32[3].p, 1, 1.0, 0.0, 1.0,
                               low_words(ctx, 0), low_words(ctx, 1), low_words(ctx, 2), low_words(ctx, 3)};
            CK(launch_drag<float>(ctx->nb, ctx->n_l, ctx->wall.p, ctx->idx.p, ctx->wgw64.p, ctx->nrm.p, f, mu, ctx->partial.p, ctx->scal.p + 8, ctx->st));
        } else {
            FieldView<double> f{ctx->a64[0].p, ctx->a64[1].p, ctx->a64[2].p, ctx->a64[3].p, 1, 1.0, 0.0, 1.0};
            CK(launch_drag<double>(ctx->nb, ctx->n_l, ctx->wall.p, ctx->idx.p, ctx->wgw64.p, ctx->nrm.p, f, mu, ctx->partial.p, ctx->scal.p + 8, ctx->st));
        }
        ctx->launches += 2;
    } else {
        CK(lbm_macro_current(ctx));
        CK(launch_sum_f64(ctx->mac.p, ctx->n, 4, 4, ctx->partial.p, ctx->scal.p, ctx->st));
        double sums[4];
        CK(cudaMemcpyAsync(sums, ctx->scal.p, 4 * sizeof(double), cudaMemcpyDeviceToHost, ctx->st));
        CK(cudaStreamSynchronize(ctx->st));
        const double vel = ctx->dx / ctx->lbm_dt;
        const double dmean = sums[3] / (double)ctx->n;  // <rho> - 1
        FieldView<double> f{ctx->mac.p, ctx->mac.p + 1, ctx->mac.p + 2, ctx->mac.p + 3, 4, vel,
                            dmean, ctx->rho * vel * vel / (3.0 * (1.0 + dmean))};
        CK(launch_drag<double>(ctx->nb, ctx->n_l, ctx->wall.p, ctx->idx.p, ctx->wgw64.p, ctx->nrm.p, f, mu, ctx->partial.p, ctx->scal.p + 8, ctx->st));
        ctx->launches += 5;
    }
    double Fs[7];
    CK(cudaMemcpyAsync(Fs, ctx->scal.p + 8, 7 * sizeof(double), cudaMemcpyDeviceToHost, ctx->st));
    CK(cudaStreamSynchronize(ctx->st));
    // wall quadrature with the wall-mean pressure removed: sum (sigma + pbar I) . n
    const double A = wall_area_of(ctx->r);
    const double pbar = ctx->nb ? Fs[3] / (double)ctx->nb : 0.0;
    for (int a = 0; a < 3; ++a) F[a] = ctx->nb ? A / (double)ctx->nb * (Fs[a] + pbar * Fs[4 + a]) : 0.0;
    if (K) {
        double qq = 0.0;
        int rc = probe_q(ctx, m_p > 0 ? m_p : 32, &qq);
        if (rc) return rc;
        *K = F[0] / (6.0 * M_PI * ctx->r * porosity_of(ctx->r) * qq * mu);
    }
    return RBF_OK;
}

}  // extern "C"

namespace {
// A context's velocity (physical units, FP64) scattered into out[3n] in the
// caller's node order.
int velocity_to(rbf_ctx *ctx, double *out) {
    if (ctx->solver == RBF_SOLVER_ACM) {
        if (ctx->prec == RBF_FP32C)
            CK(launch_velocity<float>(ctx->n, ctx->perm.p, ctx->a32[0].p, ctx->a32[1].p, ctx->a32[2].p, ctx->l32[0].p, ctx->l32[1].p, ctx->l32[2].p, 1, 1.0, out, ctx->st));
        else if (is_f32(ctx))
            CK(launch_velocity<float>(ctx->n, ctx->perm.p, ctx->a32[0].p, ctx->a32[1].p, ctx->a32[2].p, nullptr, nullptr, nullptr, 1, 1.0, out, ctx->st));
        else
            CK(launch_velocity<double>(ctx->n, ctx->perm.p, ctx->a64[0].p, ctx->a64[1].p, ctx->a64[2].p, nullptr, nullptr, nullptr, 1, 1.0, out, ctx->st));
        ++ctx->launches;
    } else {
        CK(lbm_macro_current(ctx));
        const double *m = ctx->mac.p;
        CK(launch_velocity<double>(ctx->n, ctx->perm.p, m, m + 1, m + 2, nullptr, nullptr, nullptr, 4, ctx->dx / ctx->lbm_dt, out, ctx->st));
        ctx->launches += 2;
    }
    return RBF_OK;
}
}  // namespace

extern "C" {

int rbf_pointwise_difference(rbf_ctx *a, rbf_ctx *b, double *delta, double *dv) {
    if (!a || !b || a == b) return RBF_EINVAL;
    if (!a->inited || !b->inited) return fail(a, RBF_EINVAL, "rbf_pointwise_difference: not initialised");
    if (a->device != b->device) return fail(a, RBF_EINVAL, "rbf_pointwise_difference: contexts on different devices");
    if (a->n != b->n) return fail(a, RBF_EINVAL, "rbf_pointwise_difference: node counts differ");
    if (!delta && !dv) return RBF_OK;
    DeviceGuard dg(a->device);
    const int64_t n = a->n;
    rbf_ctx *ctx = a;  // for CK's error reporting
    // stage holds at least 4n doubles: [0, 3n) velocity, [3n, 4n) one output
    int rc = velocity_to(a, a->stage.p);
    if (rc) return rc;
    CK(cudaStreamSynchronize(a->st));
    rc = velocity_to(b, b->stage.p);
    if (rc) return rc;
    ctx = b;
    CK(launch_pointwise(n, a->stage.p, b->stage.p, a->stage.p + 3 * n, b->stage.p + 3 * n, b->st));
    ++b->launches;
    if (delta) CK(cudaMemcpyAsync(delta, a->stage.p + 3 * n, n * sizeof(double), cudaMemcpyDeviceToHost, b->st));
    if (dv) CK(cudaMemcpyAsync(dv, b->stage.p + 3 * n, n * sizeof(double), cudaMemcpyDeviceToHost, b->st));
    CK(cudaStreamSynchronize(b->st));
    return RBF_OK;
}

}  // extern "C"

namespace {

// Steady ACM solve of one or more initialised contexts (same device, stream,
// precision and n_p) in one persistent cooperative launch.  Per cell: steps taken,
// last residual, status (1 converged, 0 step cap, 3 non-finite).
template <typename T>
int persistent_solve_T(std::vector<rbf_ctx *> &cs, cudaStream_t st, const rbf_solve_opts *o, std::vector<int64_t> &steps,
                       std::vector<double> &resid, std::vector<int32_t> &done, std::string &err) {
    rbf_ctx *ctx = cs[0];  // for CK's error reporting
    const int nc = (int)cs.size();
    std::vector<CellDesc<T>> desc(nc);
    std::vector<int2> sl, wsl;
    for (int c = 0; c < nc; ++c) {
        rbf_ctx *x = cs[c];
        DevArr<T> *a = nullptr;
        const DevArr<T> *ws = nullptr, *wn = nullptr;
        if constexpr (sizeof(T) == 4) { a = x->a32; ws = &x->ws32; wn = &x->wn32; }
        else { a = x->a64; ws = &x->ws64; wn = &x->wn64; }
        CellDesc<T> &d = desc[c];
        std::memset(&d, 0, sizeof(d));
        d.n = x->n; d.nb = x->nb; d.n_l = x->n_l; d.parity0 = x->parity;
        d.idx = x->idx_sell.p; d.w = ws->p; d.type = x->type.p; d.wall = x->wall.p; d.idxb = x->idxb_sell.p; d.wn = wn->p;
        d.u = a[0].p; d.v = a[1].p; d.w_ = a[2].p; d.p = a[3].p; d.us = a[4].p; d.vs = a[5].p; d.ws = a[6].p;
        d.uo = a[7].p; d.vo = a[8].p; d.wo = a[9].p; d.vmax = x->vmax.p;
        if constexpr (sizeof(T) == 4) {
            if (x->prec == RBF_FP32C) {
                DevArr<float> *l = x->l32;
                d.ul = l[0].p; d.vl = l[1].p; d.wl = l[2].p; d.pl = l[3].p; d.usl = l[4].p; d.vsl = l[5].p;
                d.wsl = l[6].p; d.uol = l[7].p; d.vol = l[8].p; d.wol = l[9].p;
            }
        }
        d.dt = (T)x->dt; d.nu = (T)x->prm.nu; d.gx = (T)x->prm.g[0]; d.gy = (T)x->prm.g[1]; d.gz = (T)x->prm.g[2];
        d.rho = (T)x->rho; d.beta = x->beta; d.vref = x->vref;
        for (int64_t s = 0; s < x->npad / 32; ++s) sl.push_back(make_int2(c, (int)s));
        for (int64_t s = 0; s < (x->nb + 31) / 32; ++s) wsl.push_back(make_int2(c, (int)s));
    }
    const bool cp = cs[0]->prec == RBF_FP32C;
    const int csize = cs[0]->persist_cluster;
    const int block = csize ? 256 : cs[0]->persist_block, wpb = block / 32;
    const int group = csize ? 1 : cs[0]->persist_group;
    int nblocks = csize;
    if (!csize) {
        int maxb = 0;
        CK(acm_persistent_max_blocks<T>(&maxb, block, group, cp));
        const int64_t units = (int64_t)sl.size() * group;  // work units of 32 / group nodes
        nblocks = std::max(1, std::min<int>(maxb, (int)((units + wpb - 1) / wpb)));
    }
    DevArr<CellDesc<T>> d_desc;
    DevArr<int2> d_sl, d_wsl;
    DevArr<unsigned> d_bar;
    DevArr<int32_t> d_err, d_done;
    DevArr<int64_t> d_steps;
    DevArr<double> d_res, d_part;
    CK(d_desc.alloc(nc)); CK(d_sl.alloc(sl.size())); CK(d_wsl.alloc(std::max<size_t>(wsl.size(), 1)));
    CK(d_bar.alloc(2)); CK(d_err.alloc(1)); CK(d_done.alloc(nc)); CK(d_steps.alloc(nc)); CK(d_res.alloc(nc));
    CK(d_part.alloc((size_t)nblocks * 2 * PERSIST_MAX_CELLS));
    CK(cudaMemcpyAsync(d_desc.p, desc.data(), nc * sizeof(CellDesc<T>), cudaMemcpyHostToDevice, st));
    CK(cudaMemcpyAsync(d_sl.p, sl.data(), sl.size() * sizeof(int2), cudaMemcpyHostToDevice, st));
    if (!wsl.empty()) CK(cudaMemcpyAsync(d_wsl.p, wsl.data(), wsl.size() * sizeof(int2), cudaMemcpyHostToDevice, st));
    CK(d_bar.zero(st)); CK(d_err.zero(st)); CK(d_done.zero(st)); CK(d_steps.zero(st)); CK(d_res.zero(st));
    PersistCtl ctl;
    std::memset(&ctl, 0, sizeof(ctl));
    ctl.bar_count = d_bar.p; ctl.bar_gen = d_bar.p + 1; ctl.err = d_err.p; ctl.done = d_done.p; ctl.steps = d_steps.p;
    ctl.resid = d_res.p; ctl.partial = d_part.p; ctl.ncells = nc; ctl.nslices = (int64_t)sl.size();
    ctl.nwslices = (int64_t)wsl.size(); ctl.slices = d_sl.p; ctl.wslices = d_wsl.p; ctl.max_steps = o->max_steps;
    ctl.check_every = o->check_every > 0 ? o->check_every : 100; ctl.tol = o->tol; ctl.n_p = cs[0]->n_p;
    ctl.wait_ns = cs[0]->wait_ns;
    CK(cudaEventRecord(ctx->ev0, st));
    if (csize) CK(acm_launch_persistent_cluster<T>(d_desc.p, ctl, csize, cp, st));
    else CK(acm_launch_persistent<T>(d_desc.p, ctl, nblocks, block, group, cp, st));
    CK(cudaEventRecord(ctx->ev1, st));
    for (rbf_ctx *x : cs) x->launches += 1;
    CK(cudaStreamSynchronize(st));
    {
        float ms = 0.f;
        CK(cudaEventElapsedTime(&ms, ctx->ev0, ctx->ev1));
        ctx->persist_ms = ms;
    }
    int32_t e = 0;
    steps.assign(nc, 0); resid.assign(nc, 0.0); done.assign(nc, 0);
    CK(cudaMemcpy(&e, d_err.p, sizeof(int32_t), cudaMemcpyDeviceToHost));
    CK(cudaMemcpy(steps.data(), d_steps.p, nc * sizeof(int64_t), cudaMemcpyDeviceToHost));
    CK(cudaMemcpy(resid.data(), d_res.p, nc * sizeof(double), cudaMemcpyDeviceToHost));
    CK(cudaMemcpy(done.data(), d_done.p, nc * sizeof(int32_t), cudaMemcpyDeviceToHost));
    for (int c = 0; c < nc; ++c) {
        cs[c]->parity = (int)((cs[c]->parity + (int64_t)cs[c]->n_p * steps[c]) & 1);
        drop_graph(cs[c]);
    }
    if (e) {
        err = "persistent ACM driver: a grid barrier timed out";
        return RBF_ETIMEOUT;
    }
    return RBF_OK;
}

int persistent_solve(std::vector<rbf_ctx *> &cs, const rbf_solve_opts *o, std::vector<int64_t> &steps,
                     std::vector<double> &resid, std::vector<int32_t> &done, std::string &err) {
    for (rbf_ctx *x : cs)
        if (!x->inited || x->solver != RBF_SOLVER_ACM || x->prec != cs[0]->prec || x->n_p != cs[0]->n_p ||
            x->device != cs[0]->device)
            return RBF_EINVAL;
    if ((int)cs.size() > PERSIST_MAX_CELLS) return RBF_EINVAL;
    if (is_f32(cs[0])) return persistent_solve_T<float>(cs, cs[0]->st, o, steps, resid, done, err);
    return persistent_solve_T<double>(cs, cs[0]->st, o, steps, resid, done, err);
}

}  // namespace

extern "C" {

int rbf_solve(rbf_ctx *ctx, const rbf_solve_opts *opts, rbf_solve_result *res) {
    if (!ctx || !opts || !res) return RBF_EINVAL;
    if (!ctx->inited) return fail(ctx, RBF_EINVAL, "rbf_solve: not initialised");
    if (opts->max_steps < 1 || !(opts->tol > 0.0)) return fail(ctx, RBF_EINVAL, "rbf_solve: bad options");
    DeviceGuard dg(ctx->device);
    const int every = opts->check_every > 0 ? opts->check_every : 100;
    const int m_p = opts->m_p > 0 ? opts->m_p : 32;
    std::memset(res, 0, sizeof(*res));
    double kprev = NAN;
    int64_t done = 0;
    if (ctx->solver == RBF_SOLVER_ACM) {
        std::vector<rbf_ctx *> cs{ctx};
        std::vector<int64_t> st;
        std::vector<double> rs;
        std::vector<int32_t> dn;
        std::string msg;
        rbf_solve_opts o = *opts;
        o.check_every = every;
        const int rc = persistent_solve(cs, &o, st, rs, dn, msg);
        if (rc) return fail(ctx, rc, msg.empty() ? std::string("rbf_solve: persistent driver failed: ") + ctx->err : msg);
        res->steps = st[0];
        res->residual = rs[0];
        res->converged = dn[0] == 1;
        if (dn[0] == 3) return fail(ctx, RBF_EDIVERGED, "rbf_solve: non-finite velocity");
        double k = 0.0;
        int rc2 = rbf_permeability(ctx, m_p, &k, nullptr);
        if (rc2) return rc2;
        res->k_over_d2 = k;
        return res->converged ? RBF_OK : fail(ctx, RBF_ENOTCONVERGED, "rbf_solve: step cap reached");
    }
    // MLBM: stop when k/d^2 changes by less than tol between checks
    while (done < opts->max_steps) {
        const int64_t chunk = std::min<int64_t>(every, opts->max_steps - done);
        int rc = run_steps(ctx, chunk);
        if (rc) return rc;
        done += chunk;
        double k = 0.0;
        rc = rbf_permeability(ctx, m_p, &k, nullptr);
        if (rc) return rc;
        if (!std::isfinite(k)) {
            res->steps = done;
            return fail(ctx, RBF_EDIVERGED, "rbf_solve: non-finite permeability");
        }
        if (std::isfinite(kprev) && k != 0.0) {
            const double crit = std::fabs(k - kprev) / std::fabs(k);
            res->residual = crit;
            if (crit < opts->tol) { kprev = k; res->converged = 1; break; }
        }
        kprev = k;
    }
    res->steps = done;
    double k = 0.0;
    int rc = rbf_permeability(ctx, m_p, &k, nullptr);
    if (rc) return rc;
    res->k_over_d2 = k;
    return res->converged ? RBF_OK : fail(ctx, RBF_ENOTCONVERGED, "rbf_solve: step cap reached");
}

}  // extern "C"

// ===========================================================================
// Permeability without device allocation.
//
// rbf_permeability keeps its per-block partial sums in a buffer the context
// allocated.  rbf_permeability_static runs a copy of the same probe reduction
// whose partials and result live in the file-scope array below instead, so the
// call itself allocates no device memory.  Host code cannot use the array's name
// as a device address (it names a host-side stand-in), so rbf_create looks the
// address up with cudaGetSymbolAddress, with the context's device current, and
// keeps it in the context (static_flux_lookup); a context cannot outlive its
// device's reset, so the address stays valid for the context's whole life.
#define RBF_STATIC_FLUX_BLOCKS 4096  // up to 4096 * 256 = 1,048,576 fluid probes
// [0, RBF_STATIC_FLUX_BLOCKS): block partials; [RBF_STATIC_FLUX_BLOCKS]: their sum
static __device__ __align__(256) double g_static_flux[RBF_STATIC_FLUX_BLOCKS + 1];

namespace {

// block b writes its partial to scratch[b]; every launch overwrites the partials of
// the blocks it runs, so nothing has to start at zero.  vxl: the low words of a
// compensated FP32 vx (summed as hi + lo in FP64), or null.
template <typename T>
__global__ void __launch_bounds__(256) k_probe_sum_static(int64_t np, int n_l, const int32_t *idx, const double *w,
                                                          const T *vx, const T *vxl, int64_t stride, double *scratch) {
    __shared__ double red[8];
    int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    double s = 0.0;
    if (p < np)
        for (int j = 0; j < n_l; ++j) {
            const int64_t q = idx[p * n_l + j] * stride;
            s += w[p * n_l + j] * (vxl ? (double)vx[q] + (double)vxl[q] : (double)vx[q]);
        }
    for (int off = 16; off > 0; off >>= 1) s += __shfl_xor_sync(0xffffffffu, s, off);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int k = 0; k < (int)(blockDim.x >> 5); ++k) t += red[k];
        scratch[blockIdx.x] = t;
    }
}

// fixed-order sum of nb partials into scratch[RBF_STATIC_FLUX_BLOCKS]
__global__ void k_static_final(double *scratch, int64_t nb) {
    double s = 0.0;
    for (int64_t b = threadIdx.x; b < nb; b += 32) s += scratch[b];
    for (int off = 16; off > 0; off >>= 1) s += __shfl_xor_sync(0xffffffffu, s, off);
    if (threadIdx.x == 0) scratch[RBF_STATIC_FLUX_BLOCKS] = s;
}

// the device address of g_static_flux on the current device
cudaError_t static_flux_lookup(double **out) {
    void *p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_static_flux);
    *out = (double *)p;
    return e;
}

}  // namespace

extern "C" int rbf_permeability_static(rbf_ctx *ctx, int m_p, double *k_over_d2, double *q) {
    if (!ctx) return RBF_EINVAL;
    if (!ctx->inited) return fail(ctx, RBF_EINVAL, "rbf_permeability_static: not initialised");
    if (ctx->m_p != m_p || !ctx->pidx.p)
        return fail(ctx, RBF_EINVAL, "rbf_permeability_static: build the probe set first with rbf_permeability(m_p)");
    const int64_t nb = (ctx->np_fluid + 255) / 256;
    if (nb > RBF_STATIC_FLUX_BLOCKS)
        return fail(ctx, RBF_EINVAL, "rbf_permeability_static: more than 1,048,576 fluid probes (static scratch limit)");
    DeviceGuard dg(ctx->device);
    double *scratch = ctx->static_flux;
    if (!scratch) return fail(ctx, RBF_ECUDA, "rbf_permeability_static: no scratch address (rbf_create failed to look it up)");
    double s = 0.0;
    if (nb > 0) {
        if (ctx->solver == RBF_SOLVER_ACM) {
            if (is_f32(ctx))
                k_probe_sum_static<float><<<(unsigned)nb, 256, 0, ctx->st>>>(ctx->np_fluid, ctx->n_l, ctx->pidx.p, ctx->pw.p, ctx->a32[0].p, low_words(ctx, 0), 1, scratch);
            else
                k_probe_sum_static<double><<<(unsigned)nb, 256, 0, ctx->st>>>(ctx->np_fluid, ctx->n_l, ctx->pidx.p, ctx->pw.p, ctx->a64[0].p, nullptr, 1, scratch);
        } else {
            CK(lbm_macro_current(ctx));
            ++ctx->launches;
            k_probe_sum_static<double><<<(unsigned)nb, 256, 0, ctx->st>>>(ctx->np_fluid, ctx->n_l, ctx->pidx.p, ctx->pw.p, ctx->mac.p, nullptr, 4, scratch);
        }
        k_static_final<<<1, 32, 0, ctx->st>>>(scratch, nb);
        ctx->launches += 2;
        CK(cudaGetLastError());
        CK(cudaMemcpyAsync(&s, scratch + RBF_STATIC_FLUX_BLOCKS, sizeof(double), cudaMemcpyDeviceToHost, ctx->st));
        CK(cudaStreamSynchronize(ctx->st));
    }
    if (ctx->solver == RBF_SOLVER_LBM) s *= ctx->dx / ctx->lbm_dt;
    const double qq = s / (5.0 * m_p * m_p);
    const double *g = ctx->prm.g;
    const double gmag = std::sqrt(g[0] * g[0] + g[1] * g[1] + g[2] * g[2]);
    if (q) *q = qq;
    if (k_over_d2) *k_over_d2 = gmag > 0.0 ? qq * ctx->prm.nu / gmag : 0.0;
    return RBF_OK;
}

// ===========================================================================
// Batched cells: many periodic cells (own nodes, sphere and stencil size) whose
// weight systems are solved in one launch and whose ACM steps run in one
// persistent launch until each cell's criterion holds.
struct rbf_batch {
    int device = 0;
    cudaStream_t st = nullptr;
    bool own_stream = false;
    std::string err;
    std::vector<rbf_ctx *> cells;
    std::vector<int> n_l;
    bool built = false;
};

namespace {
int bfail(rbf_batch *b, int code, const std::string &m) {
    if (b) b->err = m;
    return code;
}
}  // namespace

extern "C" {

int rbf_batch_create(rbf_batch **out, int device, void *cuda_stream) {
    if (!out) return RBF_EINVAL;
    *out = nullptr;
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || device < 0 || device >= ndev) return RBF_ECUDA;
    rbf_batch *b = new rbf_batch();
    b->device = device;
    DeviceGuard dg(device);
    if (cuda_stream) b->st = (cudaStream_t)cuda_stream;
    else {
        if (cudaStreamCreateWithFlags(&b->st, cudaStreamNonBlocking) != cudaSuccess) { delete b; return RBF_ECUDA; }
        b->own_stream = true;
    }
    *out = b;
    return RBF_OK;
}

int rbf_batch_destroy(rbf_batch *b) {
    if (!b) return RBF_EINVAL;
    for (rbf_ctx *c : b->cells) rbf_destroy(c);
    {
        DeviceGuard dg(b->device);
        if (b->own_stream && b->st) cudaStreamDestroy(b->st);
    }
    delete b;
    return RBF_OK;
}

const char *rbf_batch_last_error(const rbf_batch *b) { return b ? b->err.c_str() : "null batch"; }

int rbf_batch_add_cell(rbf_batch *b, int64_t n, const double *xyz, const uint8_t *type, const double *normal,
                       const double c[3], double r, int n_l) {
    if (!b) return RBF_EINVAL;
    if ((int)b->cells.size() >= PERSIST_MAX_CELLS) return bfail(b, RBF_EINVAL, "rbf_batch_add_cell: at most 128 cells");
    rbf_ctx *x = nullptr;
    int rc = rbf_create(&x, b->device, b->st);
    if (rc) return bfail(b, rc, "rbf_batch_add_cell: context creation failed");
    rc = rbf_set_nodes(x, n, xyz, type, normal);
    if (!rc) rc = rbf_set_sphere(x, c, r);
    if (rc) {
        b->err = x->err;
        rbf_destroy(x);
        return rc;
    }
    if (n_l < 2 || n_l > RBF_MAX_NL) { rbf_destroy(x); return bfail(b, RBF_EINVAL, "rbf_batch_add_cell: bad n_l"); }
    b->cells.push_back(x);
    b->n_l.push_back(n_l);
    b->built = false;
    return (int)b->cells.size() - 1;
}

int rbf_batch_build(rbf_batch *b, int phs_k, int mono_m, rbf_weight_report *rep) {
    if (!b) return RBF_EINVAL;
    if (b->cells.empty()) return bfail(b, RBF_EINVAL, "rbf_batch_build: no cells");
    if (phs_k < 3 || phs_k % 2 == 0 || phs_k > 9 || mono_m < 0 || mono_m > 4) return bfail(b, RBF_EINVAL, "rbf_batch_build: bad k or m");
    DeviceGuard dg(b->device);
    const int nc = (int)b->cells.size();
    int max_nl = 0;
    for (int c = 0; c < nc; ++c) {
        int rc = rbf_build_stencils(b->cells[c], b->n_l[c]);
        if (rc) return bfail(b, rc, std::string("cell ") + std::to_string(c) + ": " + b->cells[c]->err);
        if (b->n_l[c] < binom(mono_m + 3, 3)) return bfail(b, RBF_EINVAL, "rbf_batch_build: n_l < N_p");
        max_nl = std::max(max_nl, b->n_l[c]);
    }
    // the node systems of every cell in one launch, then the wall Neumann systems of every cell in one launch
    std::vector<WeightJob> nodes(nc), walls;
    std::vector<int64_t> pn(nc + 1, 0), pw(1, 0);
    for (int c = 0; c < nc; ++c) {
        rbf_ctx *ctx = b->cells[c];
        CK(ctx->w64.alloc(ctx->n * 4 * ctx->n_l));
        CK(ctx->delta.alloc(ctx->n));
        CK(ctx->wgb64.alloc(ctx->nb * 3 * ctx->n_l));
        nodes[c] = WeightJob{ctx->n, ctx->xyz.p, ctx->iota.p, ctx->n_l, ctx->idx.p, ctx->w64.p, ctx->delta.p};
        pn[c + 1] = pn[c] + ctx->n;
        if (ctx->nb > 0) {
            walls.push_back(WeightJob{ctx->nb, ctx->xyz.p, ctx->wall.p, ctx->n_l, ctx->idxb.p, ctx->wgb64.p, nullptr});
            pw.push_back(pw.back() + ctx->nb);
        }
    }
    rbf_ctx *ctx = b->cells[0];  // for CK
    std::vector<OpSpec> ops, gops;
    for (int kind : {OP_DX, OP_DY, OP_DZ, OP_LAP}) ops.push_back(OpSpec{kind, {0.0, 0.0, 0.0}});
    for (int kind : {OP_DX, OP_DY, OP_DZ}) gops.push_back(OpSpec{kind, {0.0, 0.0, 0.0}});
    DevArr<WeightJob> dj, dwj;
    DevArr<int64_t> dpn, dpw;
    DevArr<OpSpec> dops, dgops;
    DevArr<int32_t> dsing;
    CK(dj.alloc(nc)); CK(dpn.alloc(nc + 1)); CK(dops.alloc(4)); CK(dgops.alloc(3)); CK(dsing.alloc(2));
    CK(cudaMemcpyAsync(dj.p, nodes.data(), nc * sizeof(WeightJob), cudaMemcpyHostToDevice, b->st));
    CK(cudaMemcpyAsync(dpn.p, pn.data(), (nc + 1) * sizeof(int64_t), cudaMemcpyHostToDevice, b->st));
    CK(cudaMemcpyAsync(dops.p, ops.data(), 4 * sizeof(OpSpec), cudaMemcpyHostToDevice, b->st));
    CK(cudaMemcpyAsync(dgops.p, gops.data(), 3 * sizeof(OpSpec), cudaMemcpyHostToDevice, b->st));
    CK(dsing.zero(b->st));
    CK(launch_weights_multi(nc, dj.p, dpn.p, pn[nc], max_nl, phs_k, mono_m, 4, dops.p, 1, dsing.p, b->st));
    if (!walls.empty()) {
        CK(dwj.alloc(walls.size())); CK(dpw.alloc(pw.size()));
        CK(cudaMemcpyAsync(dwj.p, walls.data(), walls.size() * sizeof(WeightJob), cudaMemcpyHostToDevice, b->st));
        CK(cudaMemcpyAsync(dpw.p, pw.data(), pw.size() * sizeof(int64_t), cudaMemcpyHostToDevice, b->st));
        CK(launch_weights_multi((int)walls.size(), dwj.p, dpw.p, pw.back(), max_nl, phs_k, mono_m, 3, dgops.p, 1,
                                dsing.p + 1, b->st));
    }
    int32_t sing[2] = {0, 0};
    CK(cudaMemcpyAsync(sing, dsing.p, 2 * sizeof(int32_t), cudaMemcpyDeviceToHost, b->st));
    CK(cudaStreamSynchronize(b->st));
    int64_t nsys = 0, nsing = sing[0] + sing[1];
    double hmin = 1e300;
    for (int c = 0; c < nc; ++c) {
        rbf_weight_report r;
        const int rc = compute_weights_impl(b->cells[c], phs_k, mono_m, RBF_SOLVER_ACM, 0, 0.0, &r, true, c == 0 ? nsing : 0);
        nsys += r.n_systems;
        hmin = std::min(hmin, r.h_min);
        if (rc) {
            if (rep) { rep->n_systems = nsys; rep->n_singular = nsing; rep->h_min = hmin; }
            return bfail(b, rc, std::string("cell ") + std::to_string(c) + ": " + b->cells[c]->err);
        }
    }
    if (rep) { rep->n_systems = nsys; rep->n_singular = nsing; rep->h_min = hmin; }
    b->built = true;
    return RBF_OK;
}

int rbf_batch_init(rbf_batch *b, const rbf_params *p) {
    if (!b || !p) return RBF_EINVAL;
    if (!b->built) return bfail(b, RBF_EINVAL, "rbf_batch_init: build first");
    for (size_t c = 0; c < b->cells.size(); ++c) {
        const int rc = rbf_init(b->cells[c], p);
        if (rc) return bfail(b, rc, b->cells[c]->err);
    }
    return RBF_OK;
}

int rbf_batch_autotune(rbf_batch *b, int trial_steps, rbf_tune_report *rep) {
    if (!b) return RBF_EINVAL;
    if (b->cells.empty() || !b->cells[0]->inited) return bfail(b, RBF_EINVAL, "rbf_batch_autotune: init first");
    if (trial_steps < 2 || trial_steps > 20000) return bfail(b, RBF_EINVAL, "rbf_batch_autotune: 2 <= trial_steps <= 20000");
    DeviceGuard dg(b->device);
    std::string msg;
    const int rc = tune_persistent(b->cells, trial_steps, rep, msg);
    return rc ? bfail(b, rc, msg.empty() ? std::string("rbf_batch_autotune failed") : msg) : RBF_OK;
}

int rbf_batch_solve(rbf_batch *b, const rbf_solve_opts *opts, rbf_batch_cell_result *res) {
    if (!b || !opts || !res) return RBF_EINVAL;
    if (b->cells.empty() || !b->cells[0]->inited) return bfail(b, RBF_EINVAL, "rbf_batch_solve: init first");
    if (opts->max_steps < 1 || !(opts->tol > 0.0)) return bfail(b, RBF_EINVAL, "rbf_batch_solve: bad options");
    DeviceGuard dg(b->device);
    std::vector<int64_t> st;
    std::vector<double> rs;
    std::vector<int32_t> dn;
    std::string msg;
    const int rc = persistent_solve(b->cells, opts, st, rs, dn, msg);
    if (rc) return bfail(b, rc, msg.empty() ? "rbf_batch_solve: persistent driver failed" : msg);
    const int m_p = opts->m_p > 0 ? opts->m_p : 32;
    bool all = true;
    for (size_t c = 0; c < b->cells.size(); ++c) {
        res[c].steps = st[c];
        res[c].residual = rs[c];
        res[c].status = dn[c] == 1 ? 0 : (dn[c] == 3 ? 2 : 1);
        all &= dn[c] == 1;
        double k = 0.0;
        const int r2 = rbf_permeability(b->cells[c], m_p, &k, nullptr);
        if (r2) return bfail(b, r2, b->cells[c]->err);
        res[c].k_over_d2 = k;
    }
    return all ? RBF_OK : bfail(b, RBF_ENOTCONVERGED, "rbf_batch_solve: not every cell converged");
}

int rbf_batch_num_cells(const rbf_batch *b) { return b ? (int)b->cells.size() : -1; }

rbf_ctx *rbf_batch_cell(rbf_batch *b, int cell) {
    if (!b || cell < 0 || cell >= (int)b->cells.size()) return nullptr;
    return b->cells[cell];
}

}  // extern "C"
