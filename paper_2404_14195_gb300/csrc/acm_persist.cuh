// acm_persist.cuh — per-cell descriptors and control block of the persistent
// multi-cell ACM driver (acm_persist.cu).
#pragma once
#include "internal.cuh"

namespace rbf {

#define PERSIST_MAX_CELLS 128

template <typename T>
struct CellDesc {
    int64_t n, nb;
    int n_l;
    int64_t parity0;         // slot parity of this cell's next pressure iteration
    const int32_t *idx;      // SELL [slice][j][lane]
    const T *w;              // SELL [slice][4][j][lane]
    const uint8_t *type;
    const int32_t *wall;
    const int32_t *idxb;     // wall Neumann stencils, SELL over the wall list
    const T *wn;
    T *u, *v, *w_, *p;
    T *us, *vs, *ws;
    T *uo, *vo, *wo;         // snapshot for the residual
    // compensated state (RBF_FP32C, else null): low words of u, v, w, p, u', v',
    // w' and of the snapshot
    T *ul, *vl, *wl, *pl, *usl, *vsl, *wsl, *uol, *vol, *wol;
    unsigned long long *vmax;  // 2 slots
    T dt, nu, gx, gy, gz, rho;
    double beta, vref;
};

struct PersistCtl {
    unsigned *bar_count, *bar_gen;
    int32_t *err;            // 2 = a grid barrier timed out
    int32_t *done;           // per cell: 0 running, 1 converged, 3 non-finite residual
    int64_t *steps;          // per cell: steps taken in this launch
    double *resid;           // per cell: last residual
    double *partial;         // [block][PERSIST_MAX_CELLS][2]
    int ncells;
    int64_t nslices, nwslices;
    const int2 *slices;      // (cell, slice within the cell) of every node slice
    const int2 *wslices;     // the same for the wall lists
    int64_t max_steps;
    int check_every;
    double tol;
    int n_p;
    uint64_t wait_ns;        // wall-clock limit of one grid-barrier wait (nanoseconds)
};

// cp selects the compensated kernel (every cell then carries low words); block:
// threads per block, 32, 64, 128 or 256; group: lanes per node, 1, 2, 4 or 8 (a
// warp takes 32 / group nodes of a slice at a time)
template <typename T>
cudaError_t acm_launch_persistent(const CellDesc<T> *cells_dev, const PersistCtl &ctl, int nblocks, int block,
                                  int group, bool cp, cudaStream_t st);
template <typename T>
cudaError_t acm_persistent_max_blocks(int *blocks, int block, int group, bool cp);
// the same kernel as one thread-block cluster of csize (8 or 16) CTAs of 256
// threads, synchronised by the cluster barrier
template <typename T>
cudaError_t acm_launch_persistent_cluster(const CellDesc<T> *cells_dev, const PersistCtl &ctl, int csize, bool cp,
                                          cudaStream_t st);
// whether a cluster of csize CTAs of the kernel can be scheduled on this device
template <typename T>
cudaError_t acm_persistent_cluster_ok(int csize, bool cp, bool *ok);

}  // namespace rbf
