// reduce.cuh — launchers of the FP64 reductions and field marshalling kernels.
#pragma once
#include "internal.cuh"

namespace rbf {

// Read-only view of a velocity / pressure field: component pointers with a
// common element stride, scaled to physical units v = raw * vel,
// p = (raw - p0) * ps.  ul .. pl: the low words of a compensated FP32 state
// (raw = hi + lo, summed in FP64), null otherwise.
template <typename T>
struct FieldView {
    const T *u, *v, *w, *p;
    int64_t stride;
    double vel, p0, ps;
    const T *ul = nullptr, *vl = nullptr, *wl = nullptr, *pl = nullptr;
};

template <typename T>
cudaError_t launch_residual(int64_t n, const uint8_t *type, const T *u, const T *v, const T *w, const T *uo,
                            const T *vo, const T *wo, double *partial, double *out2, cudaStream_t st);
// vxl: low words of a compensated FP32 vx (value = hi + lo in FP64), or null
template <typename T>
cudaError_t launch_probe_sum(int64_t np, int n_l, const int32_t *idx, const double *w, const T *vx, const T *vxl,
                             int64_t stride, double *partial, double *out, cudaStream_t st);
// out7 = (sum_b sigma . n [3], sum_b p_b, sum_b n_b [3]) over the wall nodes;
// partial needs 7 doubles per 256 wall nodes
template <typename T>
cudaError_t launch_drag(int64_t nb, int n_l, const int32_t *wall, const int32_t *idx, const double *wg,
                        const double *nrm, const FieldView<T> &f, double mu, double *partial, double *out7,
                        cudaStream_t st);
template <typename T>
cudaError_t launch_acm_export(int64_t n, const int32_t *perm, const T *u, const T *v, const T *w, const T *p,
                              double *out, cudaStream_t st);
template <typename T>
cudaError_t launch_acm_import(int64_t n, const int32_t *perm, T *u, T *v, T *w, T *p, const double *in,
                              cudaStream_t st);
// compensated FP32 fields: exports hi + lo in FP64; imports x as hi = fl(x),
// lo = fl(x - hi)
cudaError_t launch_acm_export_pair(int64_t n, const int32_t *perm, const float *u, const float *v, const float *w,
                                   const float *p, const float *ul, const float *vl, const float *wl,
                                   const float *pl, double *out, cudaStream_t st);
cudaError_t launch_acm_import_pair(int64_t n, const int32_t *perm, float *u, float *v, float *w, float *p,
                                   float *ul, float *vl, float *wl, float *pl, const double *in, cudaStream_t st);
template <typename T>
cudaError_t launch_nonfinite(const T *a, int64_t n, int32_t *flag, cudaStream_t st);
// velocity scale (u[i stride] + ul[i], ...) scattered to caller order [n][3] FP64
// (ul, vl, wl null for a plain state)
template <typename T>
cudaError_t launch_velocity(int64_t n, const int32_t *perm, const T *u, const T *v, const T *w, const T *ul,
                            const T *vl, const T *wl, int64_t stride, double scale, double *out, cudaStream_t st);
// pointwise difference of two [n][3] velocity fields in one node order
cudaError_t launch_pointwise(int64_t n, const double *va, const double *vb, double *delta, double *dv,
                             cudaStream_t st);
cudaError_t launch_lbm_fields(int64_t n, const int32_t *perm, const double *mac, double vel, double ps,
                              const double *drho_sum, double *out, cudaStream_t st);
cudaError_t launch_export_stencils(int64_t n, int n_l, const int32_t *perm, const int32_t *iperm,
                                   const int32_t *idx, int32_t *out, cudaStream_t st);
cudaError_t launch_export_weights(int64_t n, int n_l, int n_ops, int op, const int32_t *iperm, const int32_t *rowmap,
                                  const double *w, double *out, cudaStream_t st);

}  // namespace rbf
