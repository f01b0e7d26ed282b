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
//     Sequential variant (Algorithm 3, Appendix "Sequential Clipping"): the active rows one at a
//     time, each on the box the earlier rows left (kept in FP64 in shared memory), with the
//     pre-check repeated on that box (stop when a row is infeasible or the box empties, skip a
//     redundant row); optionally in the constraint-importance order of the Appendix's heuristics
//     (ascending |g.xhat + h| / ||g||_2 on the input box, equal distances in row order).
#include "cv_internal.cuh"

#include <math.h>

#include <string>

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

// Warp then block sum of NV doubles per thread; every thread returns the same totals (warps added
// in a fixed order).  `red` holds NV x (blockDim.x / 32) doubles; the caller separates uses with a
// barrier.
template <int NV>
__device__ __forceinline__ void block_sums(double (&v)[NV], double* red) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
#pragma unroll
    for (int q = 0; q < NV; ++q)
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) v[q] += __shfl_xor_sync(0xffffffffu, v[q], off);
    if (lane == 0)
#pragma unroll
        for (int q = 0; q < NV; ++q) red[q * nw + warp] = v[q];
    __syncthreads();
#pragma unroll
    for (int q = 0; q < NV; ++q) {
        double t = 0.0;
        for (int w = 0; w < nw; ++w) t += red[q * nw + w];
        v[q] = t;
    }
}

// Algorithm 3: one block per subdomain, threads over coordinates; shared memory holds the
// current box [2 x n0] in FP64, then the row order [Rmax] and distances [Rmax].
__global__ void k_relaxed_seq(cv_cache cc, cv_batch_in in, int Rmax, int ordered, const int8_t* rowflag,
                              float* lo_clip, float* hi_clip, uint8_t* infeasible, int* status) {
    extern __shared__ __align__(16) unsigned char rs_smem[];
    __shared__ double red[3 * 32];
    __shared__ int s_empty, s_nact;
    const int b = blockIdx.x;
    const int n0 = cc.n0;
    double* cl = (double*)rs_smem;
    double* ch = cl + n0;
    double* dist = ch + n0;
    int* ord = (int*)(dist + Rmax);
    const float* lo = in.lo + (size_t)b * n0;
    const float* hi = in.hi + (size_t)b * n0;
    const bool inf0 = infeasible[b] != 0;
    if (threadIdx.x == 0) {
        s_empty = 0;
        int a = 0;
        for (int k = 0; k < Rmax; ++k)
            if (rowflag[(size_t)b * Rmax + k] == 0) ord[a++] = k;
        s_nact = a;
    }
    for (int i = threadIdx.x; i < n0; i += blockDim.x) {
        cl[i] = (double)lo[i];
        ch[i] = (double)hi[i];
        if (!isfinite(cl[i]) || !isfinite(ch[i])) atomicOr(status, CV_DEV_NONFINITE);
    }
    __syncthreads();
    const int nact = inf0 ? 0 : s_nact;
    bool dummy = false;
    if (ordered && nact > 1) {
        // distances of the active rows' hyperplanes from the input box centre
        for (int a = 0; a < nact; ++a) {
            const RowRef r = row_ref(cc, in, b, ord[a], status, &dummy);
            double v[2] = {0.0, 0.0};
            for (int j = threadIdx.x; j < n0; j += blockDim.x) {
                const double g = (double)(r.sign * r.g[j]);
                v[0] += g * (0.5 * (cl[j] + ch[j]));
                v[1] += g * g;
            }
            block_sums<2>(v, red);
            if (threadIdx.x == 0) dist[a] = v[1] > 0.0 ? fabs(v[0] + (double)r.h) / sqrt(v[1]) : INFINITY;
            __syncthreads();
        }
        if (threadIdx.x == 0) {  // stable insertion sort of (distance, row)
            for (int a = 1; a < nact; ++a) {
                const double d = dist[a];
                const int k = ord[a];
                int c = a - 1;
                while (c >= 0 && dist[c] > d) { dist[c + 1] = dist[c]; ord[c + 1] = ord[c]; --c; }
                dist[c + 1] = d;
                ord[c + 1] = k;
            }
        }
        __syncthreads();
    }
    bool stop = false;
    for (int a = 0; a < nact && !stop; ++a) {
        const RowRef r = row_ref(cc, in, b, ord[a], status, &dummy);
        // pre-check of the row on the current box (the certified minimum, as in k_rows)
        double v[3] = {0.0, 0.0, 0.0};
        for (int j = threadIdx.x; j < n0; j += blockDim.x) {
            const double g = (double)(r.sign * r.g[j]);
            const double p = g * cl[j], q = g * ch[j];
            v[0] += fmin(p, q);
            v[1] += fmax(p, q);
            v[2] += fmax(fabs(p), fabs(q));
        }
        block_sums<3>(v, red);
        const double h = (double)r.h;
        const double vmin = v[0] + h, vmax = v[1] + h;
        const double vlo = vmin - ldexp(v[2] + fabs(h), -40);
        if (vlo > 0.0) {  // infeasible on the current box: the subdomain is empty
            stop = true;
            if (threadIdx.x == 0) infeasible[b] = 1;
        } else if (vmax > 0.0) {  // not redundant: Theorem 2 on the current box
            for (int i = threadIdx.x; i < n0; i += blockDim.x) {
                const double g = (double)(r.sign * r.g[i]);
                if (g == 0.0) continue;
                const double t = -vlo / g;
                if (g > 0.0) {
                    double c = cl[i] + t;
                    c += ldexp(fabs(cl[i]) + fabs(t), -50);
                    if (c < ch[i]) ch[i] = c;
                } else {
                    double c = ch[i] + t;
                    c -= ldexp(fabs(ch[i]) + fabs(t), -50);
                    if (c > cl[i]) cl[i] = c;
                }
                if (cl[i] > ch[i]) s_empty = 1;
            }
        }
        __syncthreads();
        if (s_empty) stop = true;
    }
    for (int i = threadIdx.x; i < n0; i += blockDim.x) {
        const float fl = __double2float_rd(cl[i]), fh = __double2float_ru(ch[i]);
        lo_clip[(size_t)b * n0 + i] = fl;
        hi_clip[(size_t)b * n0 + i] = fh;
        if (fl > fh) s_empty = 1;
    }
    __syncthreads();
    if (threadIdx.x == 0 && s_empty) infeasible[b] = 1;
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
    if ((opt->relaxed == CV_RELAX_SEQUENTIAL || opt->relaxed == CV_RELAX_SEQUENTIAL_ORDERED) && lay->Rmax > 0 &&
        in->B > 0) {
        const size_t smem = (size_t)cache->n0 * 16 + (size_t)lay->Rmax * 12;
        if (smem > CV_SEQ_SMEM_MAX) {
            cv_set_error("sequential relaxed clipping keeps the box in shared memory: 16 n0 + 12 (max_splits + "
                         "max_rows) must stay within " + std::to_string((size_t)CV_SEQ_SMEM_MAX) + " bytes");
            return CV_EUNSUPPORTED;
        }
        CV_CUDA(cudaFuncSetAttribute(k_relaxed_seq, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
        k_relaxed_seq<<<in->B, 256, smem, st>>>(*cache, *in, lay->Rmax,
                                                opt->relaxed == CV_RELAX_SEQUENTIAL_ORDERED,
                                                (const int8_t*)(ws + lay->rowflag), lo_clip, hi_clip, infeasible,
                                                cache->net->status);
        CV_LAUNCH_CHECK("k_relaxed_seq");
        return CV_OK;
    }
    k_relaxed<<<in->B, 256, 0, st>>>(*cache, *in, lay->Rmax, opt->relaxed == CV_RELAX_PARALLEL && lay->Rmax > 0,
                                     (const int8_t*)(ws + lay->rowflag), (const double*)(ws + lay->vmin),
                                     lo_clip, hi_clip, infeasible, cache->net->status);
    CV_LAUNCH_CHECK("k_relaxed");
    return CV_OK;
}
