// Constraint rows (a2), their a-priori pre-check (a3) and parallel relaxed clipping (a4).
//
// a2: a split z_g >= 0 of a cached neuron gives the row -Abar_g x - cbar_g <= 0, a split
//     z_g <= 0 gives Aund_g x + cund_g <= 0 (paper Section 3.4, validity of activation-split
//     constraints); extra rows are read from the caller's CSR.  Rows are never copied: the
//     kernels read the cached plane (L2-resident) through a (plane, sign) descriptor.
// a3: infeasible iff min_box(g.x + h) > 0, redundant iff max_box(g.x + h) <= 0 (Section 3.2;
//     Appendix D.3).  Sums of exact FP32xFP32 products in FP64; the infeasible decision is
//     taken on the sum minus its FP64 error bound, so a feasible row is never declared empty.
// a4: Theorem 2 for every active row on the input box (Algorithm 2):
//     g_i > 0: hi_i <- min(hi_i, lo_i - v_min/g_i);  g_i < 0: lo_i <- max(lo_i, hi_i - v_min/g_i),
//     evaluated in FP64 with v_min replaced by its certified lower bound and the result rounded
//     outward to FP32.
#include "cv_internal.cuh"

#include <math.h>

namespace {

struct RowRef {
    const float* g;  // row vector (plane or extra row)
    float sign;      // multiply g and h by sign
    float h;         // already signed
    int kind;        // 0 row, 3 none (no row: split on a stable neuron / beyond count)
};

__device__ __forceinline__ RowRef row_ref(const cv_cache& cc, const cv_batch_in& in, int b, int k,
                                          int* status, bool* contradiction) {
    RowRef r;
    r.kind = 3; r.g = nullptr; r.sign = 1.f; r.h = 0.f;
    const int ns = in.split_off ? in.split_off[b + 1] - in.split_off[b] : 0;
    if (k < ns) {
        const int code = in.split_ids[in.split_off[b] + k];
        const int side = code > 0 ? 1 : -1;
        const int g = (code > 0 ? code : -code) - 1;
        if (code == 0 || g >= cc.H) { atomicOr(status, CV_DEV_SPLIT_RANGE); return r; }
        const int slot = cc.slot_of[g];
        if (slot < 0) {
            const int st = cc.root_state[g];
            if (st != side) *contradiction = true;
            return r;
        }
        r.kind = 0;
        if (side > 0) { r.g = cc.uA + (size_t)slot * cc.n0; r.sign = -1.f; r.h = -cc.uc[slot]; }
        else          { r.g = cc.lA + (size_t)slot * cc.n0; r.sign = 1.f;  r.h = cc.lc[slot]; }
        return r;
    }
    const int e = k - ns;
    const int ne = in.row_off ? in.row_off[b + 1] - in.row_off[b] : 0;
    if (e < ne) {
        const int row = in.row_off[b] + e;
        r.kind = 0;
        r.g = in.G + (size_t)row * cc.n0;
        r.sign = 1.f;
        r.h = in.h[row];
    }
    return r;
}

// one warp per (subdomain, row slot)
__global__ void k_rows(cv_cache cc, cv_batch_in in, int Rmax, int max_splits, int max_rows,
                       int8_t* rowflag, double* vmin_lo, uint8_t* infeasible, int* status) {
    const int b = blockIdx.x;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int nw = blockDim.x >> 5;
    const int n0 = cc.n0;
    if (warp == 0 && lane == 0) {
        const int ns = in.split_off ? in.split_off[b + 1] - in.split_off[b] : 0;
        const int ne = in.row_off ? in.row_off[b + 1] - in.row_off[b] : 0;
        if (ns < 0 || ns > max_splits || ne < 0 || ne > max_rows) atomicOr(status, CV_DEV_CSR_COUNT);
    }
    for (int k = warp; k < Rmax; k += nw) {
        bool contra = false;
        RowRef r;
        const int ns = in.split_off ? in.split_off[b + 1] - in.split_off[b] : 0;
        const int ne = in.row_off ? in.row_off[b + 1] - in.row_off[b] : 0;
        if (ns < 0 || ns > max_splits || ne < 0 || ne > max_rows) { r.kind = 3; }
        else r = row_ref(cc, in, b, k, status, &contra);
        if (contra && lane == 0) infeasible[b] = 1;
        int8_t flag = 3;
        double vl = 0.0;
        if (r.kind == 0) {
            double smin = 0.0, smax = 0.0, mag = 0.0;
            const float* lo = in.lo + (size_t)b * n0;
            const float* hi = in.hi + (size_t)b * n0;
            for (int j = lane; j < n0; j += 32) {
                const double g = (double)(r.sign * r.g[j]);
                const double a = g * (double)lo[j], c = g * (double)hi[j];
                smin += fmin(a, c);
                smax += fmax(a, c);
                mag += fmax(fabs(a), fabs(c));
            }
#pragma unroll
            for (int off = 16; off > 0; off >>= 1) {
                smin += __shfl_xor_sync(0xffffffffu, smin, off);
                smax += __shfl_xor_sync(0xffffffffu, smax, off);
                mag += __shfl_xor_sync(0xffffffffu, mag, off);
            }
            const double h = (double)r.h;
            const double err = ldexp(mag + fabs(h), -40);
            const double vmin = smin + h, vmax = smax + h;
            if (vmin - err > 0.0) flag = 1;
            else if (vmax <= 0.0) flag = 2;
            else flag = 0;
            vl = vmin - err;
            if (flag == 1 && lane == 0) infeasible[b] = 1;
        }
        if (lane == 0) {
            rowflag[(size_t)b * Rmax + k] = flag;
            vmin_lo[(size_t)b * Rmax + k] = vl;
        }
    }
}

// one block per subdomain, threads over coordinates
__global__ void k_relaxed(cv_cache cc, cv_batch_in in, int Rmax, int relaxed, const int8_t* rowflag,
                          const double* vmin_lo, float* lo_clip, float* hi_clip, uint8_t* infeasible,
                          int* status) {
    const int b = blockIdx.x;
    const int n0 = cc.n0;
    const float* lo = in.lo + (size_t)b * n0;
    const float* hi = in.hi + (size_t)b * n0;
    const bool inf0 = infeasible[b] != 0;
    __shared__ int any_empty;
    if (threadIdx.x == 0) any_empty = 0;
    __syncthreads();
    const int ns = in.split_off ? in.split_off[b + 1] - in.split_off[b] : 0;
    for (int i = threadIdx.x; i < n0; i += blockDim.x) {
        const double l0 = (double)lo[i], h0 = (double)hi[i];
        if (!isfinite(l0) || !isfinite(h0)) atomicOr(status, CV_DEV_NONFINITE);
        double nl = l0, nh = h0;
        if (relaxed && !inf0) {
            for (int k = 0; k < Rmax; ++k) {
                if (rowflag[(size_t)b * Rmax + k] != 0) continue;
                // rows are re-derived from the CSR (descriptor only, no copy)
                const float* gp; float sg;
                if (k < ns) {
                    const int code = in.split_ids[in.split_off[b] + k];
                    const int g = (code > 0 ? code : -code) - 1;
                    const int slot = cc.slot_of[g];
                    if (code > 0) { gp = cc.uA + (size_t)slot * n0; sg = -1.f; }
                    else { gp = cc.lA + (size_t)slot * n0; sg = 1.f; }
                } else {
                    const int row = in.row_off[b] + (k - ns);
                    gp = in.G + (size_t)row * n0; sg = 1.f;
                }
                const double g = (double)(sg * gp[i]);
                if (g == 0.0) continue;
                const double v = vmin_lo[(size_t)b * Rmax + k];  // certified lower bound, <= 0
                const double t = -v / g;
                if (g > 0.0) {
                    double c = l0 + t;
                    c += ldexp(fabs(l0) + fabs(t), -50);
                    if (c < nh) nh = c;
                } else {
                    double c = h0 + t;
                    c -= ldexp(fabs(h0) + fabs(t), -50);
                    if (c > nl) nl = c;
                }
            }
        }
        const float fl = __double2float_rd(nl), fh = __double2float_ru(nh);
        lo_clip[(size_t)b * n0 + i] = fl;
        hi_clip[(size_t)b * n0 + i] = fh;
        if (fl > fh) any_empty = 1;
    }
    __syncthreads();
    if (threadIdx.x == 0 && any_empty) infeasible[b] = 1;
}

}  // namespace

cv_status cv_launch_rows(const cv_net* net, const cv_cache* cache, const cv_batch_in* in,
                         const cv_ws_layout* lay, char* ws, uint8_t* infeasible, cudaStream_t st) {
    (void)net;
    if (lay->Rmax == 0) return CV_OK;
    k_rows<<<in->B, 128, 0, st>>>(*cache, *in, lay->Rmax, in->max_splits, in->max_rows,
                                  (int8_t*)(ws + lay->rowflag), (double*)(ws + lay->vmin), infeasible,
                                  cache->net->status);
    CV_LAUNCH_CHECK("k_rows");
    return CV_OK;
}

cv_status cv_launch_relaxed(const cv_net* net, const cv_cache* cache, const cv_batch_in* in,
                            const cv_options* opt, const cv_ws_layout* lay, char* ws,
                            float* lo_clip, float* hi_clip, uint8_t* infeasible, cudaStream_t st) {
    (void)net;
    k_relaxed<<<in->B, 256, 0, st>>>(*cache, *in, lay->Rmax, opt->relaxed && lay->Rmax > 0,
                                     (const int8_t*)(ws + lay->rowflag), (const double*)(ws + lay->vmin),
                                     lo_clip, hi_clip, infeasible, cache->net->status);
    CV_LAUNCH_CHECK("k_relaxed");
    return CV_OK;
}
