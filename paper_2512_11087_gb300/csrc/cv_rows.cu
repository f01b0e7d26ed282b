// Constraint rows (a2), their a-priori pre-check (a3) and parallel relaxed clipping (a4).
//
// a2: a split z_g >= 0 of a cached neuron gives the row -Abar_g x - cbar_g <= 0, a split
//     z_g <= 0 gives Aund_g x + cund_g <= 0 (paper Section 3.4, validity of activation-split
//     constraints); extra rows are read from the caller's CSR.  Rows are never copied: the
//     kernels read the cached plane (L2-resident) through a (plane, sign) descriptor.
// a3: infeasible iff min_box(g.x + h) > 0, redundant iff max_box(g.x + h) <= 0 (Section 3.2;
//     Appendix D.3).  The FP32 products are exact as float-float pairs (fma) and summed in
//     float-float; the infeasible decision is taken on the sum minus an a-priori bound of its
//     error, so a feasible row is never declared empty.
// a4: Theorem 2 for every active row on the input box (Algorithm 2):
//     g_i > 0: hi_i <- min(hi_i, lo_i - v_min/g_i);  g_i < 0: lo_i <- max(lo_i, hi_i - v_min/g_i),
//     in float-float with v_min replaced by its certified lower bound, widened by a bound of the
//     float-float error and rounded outward to FP32.
//     Sequential variant (Algorithm 3, Appendix "Sequential Clipping"): the active rows one at a
//     time, each on the box the earlier rows left (kept in float-float in shared memory), with the
//     pre-check repeated on that box (stop when a row is infeasible or the box empties, skip a
//     redundant row); optionally in the constraint-importance order of the Appendix's heuristics
//     (ascending |g.xhat + h| / ||g||_2 on the input box, equal distances in row order).
// All arithmetic is FP32 (float-float: about 44 bits, error-free transformations of Knuth and
// Dekker); the pads below cover its error with a wide margin, and the results are FP32.
#include "cv_internal.cuh"

#include <math.h>

#include <string>

namespace {

// ---------------------------------------------------------------- float-float
// An unevaluated sum hi + lo of two FP32 values with hi = fl(hi + lo).
struct ff { float hi, lo; };

__device__ __forceinline__ ff ff_two_sum(float a, float b) {  // exact: a + b = s + e
    const float s = a + b, bp = s - a;
    return {s, (a - (s - bp)) + (b - bp)};
}
__device__ __forceinline__ ff ff_add(ff a, ff b) {
    const ff s = ff_two_sum(a.hi, b.hi);
    return ff_two_sum(s.hi, s.lo + (a.lo + b.lo));
}
__device__ __forceinline__ ff ff_of(float a) { return {a, 0.f}; }
__device__ __forceinline__ ff ff_neg(ff a) { return {-a.hi, -a.lo}; }
__device__ __forceinline__ ff ff_prod(float a, float b) {  // exact: a b = p + e
    const float p = a * b;
    return {p, fmaf(a, b, -p)};
}
__device__ __forceinline__ ff ff_mulf(ff a, float b) {  // (a.hi + a.lo) b, error O(u^2 |a b|)
    const ff p = ff_prod(a.hi, b);
    return ff_two_sum(p.hi, fmaf(a.lo, b, p.lo));
}
__device__ __forceinline__ ff ff_div(ff a, float g) {  // a / g, g != 0; error O(u^2 |a / g|)
    const float q1 = a.hi / g;
    const float r = fmaf(-q1, g, a.hi) + a.lo;  // the remainder of a.hi is exact
    return ff_two_sum(q1, r / g);
}
__device__ __forceinline__ bool ff_lt(ff a, ff b) { return a.hi < b.hi || (a.hi == b.hi && a.lo < b.lo); }
__device__ __forceinline__ bool ff_gt0(ff a) { return a.hi > 0.f || (a.hi == 0.f && a.lo > 0.f); }
__device__ __forceinline__ bool ff_le0(ff a) { return !ff_gt0(a); }
__device__ __forceinline__ float ff_absf(ff a) { return fabsf(a.hi); }
// FP32 rounding of hi + lo downward / upward (hi is its nearest rounding)
__device__ __forceinline__ float ff_rd(ff a) { return a.lo < 0.f ? nextafterf(a.hi, -INFINITY) : a.hi; }
__device__ __forceinline__ float ff_ru(ff a) { return a.lo > 0.f ? nextafterf(a.hi, INFINITY) : a.hi; }
__device__ __forceinline__ ff ff_shfl_xor(ff a, int off) {
    return {__shfl_xor_sync(0xffffffffu, a.hi, off), __shfl_xor_sync(0xffffffffu, a.lo, off)};
}
// A bound of the error of a float-float sum of n exact products of total magnitude mag: one
// ff_add errs by at most 3 u^2 (|a| + |b|) <= 3 u^2 mag (its low-part additions), so a lane's
// n / 32 additions and the five butterfly levels stay below 3 (n / 32 + 6) u^2 mag; charged as
// (n + 16) 2^-46 mag, rounded up
__device__ __forceinline__ float ff_sum_err(float mag, int n) {
    return __fmul_ru(__fmul_ru(mag, (float)(n + 16)), 1.4210855e-14f);  // 2^-46
}
// margin for one clip step c = x + t, t = -v / g in float-float (at most 6 u^2 (|x| + |t|)):
// (|x| + |t|) 2^-40
__device__ __forceinline__ float ff_step_err(float x, float t) {
    return __fmul_ru(__fadd_ru(fabsf(x), fabsf(t)), 9.094947e-13f);  // 2^-40
}

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
                       int8_t* rowflag, ff* vmin_lo, uint8_t* infeasible, int* status) {
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
        ff vl = ff_of(0.f);
        if (r.kind == 0) {
            ff smin = ff_of(0.f), smax = ff_of(0.f);
            float mag = 0.f;  // sum of max(|g lo|, |g hi|), rounded up
            const float* lo = in.lo + (size_t)b * n0;
            const float* hi = in.hi + (size_t)b * n0;
            for (int j = lane; j < n0; j += 32) {
                const float g = r.sign * r.g[j];
                const ff a = ff_prod(g, lo[j]), c = ff_prod(g, hi[j]);
                const bool al = ff_lt(a, c);
                smin = ff_add(smin, al ? a : c);
                smax = ff_add(smax, al ? c : a);
                mag = __fadd_ru(mag, fmaxf(ff_absf(a), ff_absf(c)));
            }
#pragma unroll
            for (int off = 16; off > 0; off >>= 1) {
                smin = ff_add(smin, ff_shfl_xor(smin, off));
                smax = ff_add(smax, ff_shfl_xor(smax, off));
                mag = __fadd_ru(mag, __shfl_xor_sync(0xffffffffu, mag, off));
            }
            // |products| <= (1 + u) |their high parts|: the magnitude bound gains 2^-22 of itself
            const float magb = __fmul_ru(__fadd_ru(mag, fabsf(r.h)), 1.00000024f);
            const float err = ff_sum_err(magb, n0);
            const ff vmin = ff_add(smin, ff_of(r.h)), vmax = ff_add(smax, ff_of(r.h));
            vl = ff_add(vmin, ff_of(-err));
            if (ff_gt0(vl)) flag = 1;
            else if (ff_le0(vmax)) flag = 2;
            else flag = 0;
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
                          const ff* vmin_lo, float* lo_clip, float* hi_clip, uint8_t* infeasible,
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
        const float l0 = lo[i], h0 = hi[i];
        if (!isfinite(l0) || !isfinite(h0)) atomicOr(status, CV_DEV_NONFINITE);
        ff nl = ff_of(l0), nh = ff_of(h0);
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
                const float g = sg * gp[i];
                if (g == 0.f) continue;
                const ff v = vmin_lo[(size_t)b * Rmax + k];  // certified lower bound, <= 0
                const ff t = ff_div(ff_neg(v), g);
                if (g > 0.f) {
                    ff c = ff_add(ff_of(l0), t);
                    c = ff_add(c, ff_of(ff_step_err(l0, t.hi)));
                    if (ff_lt(c, nh)) nh = c;
                } else {
                    ff c = ff_add(ff_of(h0), t);
                    c = ff_add(c, ff_of(-ff_step_err(h0, t.hi)));
                    if (ff_lt(nl, c)) nl = c;
                }
            }
        }
        const float fl = ff_rd(nl), fh = ff_ru(nh);
        lo_clip[(size_t)b * n0 + i] = fl;
        hi_clip[(size_t)b * n0 + i] = fh;
        if (fl > fh) any_empty = 1;
    }
    __syncthreads();
    if (threadIdx.x == 0 && any_empty) infeasible[b] = 1;
}

// Warp then block float-float sums of NV values per thread; every thread returns the same totals
// (warps added in a fixed order).  `red` holds NV x (blockDim.x / 32) pairs; the caller separates
// uses with a barrier.
template <int NV>
__device__ __forceinline__ void block_sums(ff (&v)[NV], ff* red) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
#pragma unroll
    for (int q = 0; q < NV; ++q)
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) v[q] = ff_add(v[q], ff_shfl_xor(v[q], off));
    if (lane == 0)
#pragma unroll
        for (int q = 0; q < NV; ++q) red[q * nw + warp] = v[q];
    __syncthreads();
#pragma unroll
    for (int q = 0; q < NV; ++q) {
        ff t = ff_of(0.f);
        for (int w = 0; w < nw; ++w) t = ff_add(t, red[q * nw + w]);
        v[q] = t;
    }
}

// the same for an FP32 sum rounded up (magnitudes)
__device__ __forceinline__ float block_sum_ru(float v, float* red) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) v = __fadd_ru(v, __shfl_xor_sync(0xffffffffu, v, off));
    if (lane == 0) red[warp] = v;
    __syncthreads();
    float t = 0.f;
    for (int w = 0; w < nw; ++w) t = __fadd_ru(t, red[w]);
    return t;
}

// sqrt of a float-float (one Newton correction of the FP32 root)
__device__ __forceinline__ ff ff_sqrt(ff a) {
    if (a.hi <= 0.f) return ff_of(0.f);
    const float r = sqrtf(a.hi);
    const float e = (fmaf(-r, r, a.hi) + a.lo) / (2.f * r);
    return ff_two_sum(r, e);
}
// a / b for float-float b > 0
__device__ __forceinline__ ff ff_div_ff(ff a, ff b) {
    const float q1 = a.hi / b.hi;
    const ff p = ff_mulf(b, q1);
    const ff r = ff_add(a, ff_neg(p));
    return ff_two_sum(q1, r.hi / b.hi);
}

// Algorithm 3: one block per subdomain, threads over coordinates; shared memory holds the
// current box [2 x n0] in float-float, then the row distances [Rmax] (float-float) and the row
// order [Rmax].
__global__ void k_relaxed_seq(cv_cache cc, cv_batch_in in, int Rmax, int ordered, const int8_t* rowflag,
                              float* lo_clip, float* hi_clip, uint8_t* infeasible, int* status) {
    extern __shared__ __align__(16) unsigned char rs_smem[];
    __shared__ ff red[3 * 32];
    __shared__ float redm[32];
    __shared__ int s_empty, s_nact;
    const int b = blockIdx.x;
    const int n0 = cc.n0;
    ff* cl = (ff*)rs_smem;
    ff* ch = cl + n0;
    ff* dist = ch + n0;
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
        cl[i] = ff_of(lo[i]);
        ch[i] = ff_of(hi[i]);
        if (!isfinite(lo[i]) || !isfinite(hi[i])) atomicOr(status, CV_DEV_NONFINITE);
    }
    __syncthreads();
    const int nact = inf0 ? 0 : s_nact;
    bool dummy = false;
    if (ordered && nact > 1) {
        // distances of the active rows' hyperplanes from the input box centre (exact centre: the
        // halved FP32 sum is a float-float)
        for (int a = 0; a < nact; ++a) {
            const RowRef r = row_ref(cc, in, b, ord[a], status, &dummy);
            ff v[2] = {ff_of(0.f), ff_of(0.f)};
            for (int j = threadIdx.x; j < n0; j += blockDim.x) {
                const float g = r.sign * r.g[j];
                const ff c = ff_two_sum(0.5f * cl[j].hi, 0.5f * ch[j].hi);
                v[0] = ff_add(v[0], ff_mulf(c, g));
                v[1] = ff_add(v[1], ff_prod(g, g));
            }
            block_sums<2>(v, red);
            if (threadIdx.x == 0) {
                const ff num = ff_add(v[0], ff_of(r.h));
                const ff an = num.hi < 0.f ? ff_neg(num) : num;
                dist[a] = ff_gt0(v[1]) ? ff_div_ff(an, ff_sqrt(v[1])) : ff_of(INFINITY);
            }
            __syncthreads();
        }
        if (threadIdx.x == 0) {  // stable insertion sort of (distance, row)
            for (int a = 1; a < nact; ++a) {
                const ff d = dist[a];
                const int k = ord[a];
                int c = a - 1;
                while (c >= 0 && ff_lt(d, dist[c])) { dist[c + 1] = dist[c]; ord[c + 1] = ord[c]; --c; }
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
        ff v[2] = {ff_of(0.f), ff_of(0.f)};
        float mag = 0.f;
        for (int j = threadIdx.x; j < n0; j += blockDim.x) {
            const float g = r.sign * r.g[j];
            const ff p = ff_mulf(cl[j], g), q = ff_mulf(ch[j], g);
            const bool pl = ff_lt(p, q);
            v[0] = ff_add(v[0], pl ? p : q);
            v[1] = ff_add(v[1], pl ? q : p);
            mag = __fadd_ru(mag, fmaxf(ff_absf(p), ff_absf(q)));
        }
        block_sums<2>(v, red);
        mag = block_sum_ru(mag, redm);
        const float magb = __fmul_ru(__fadd_ru(mag, fabsf(r.h)), 1.00000024f);
        const ff vmin = ff_add(v[0], ff_of(r.h)), vmax = ff_add(v[1], ff_of(r.h));
        const ff vlo = ff_add(vmin, ff_of(-ff_sum_err(magb, n0)));
        if (ff_gt0(vlo)) {  // infeasible on the current box: the subdomain is empty
            stop = true;
            if (threadIdx.x == 0) infeasible[b] = 1;
        } else if (ff_gt0(vmax)) {  // not redundant: Theorem 2 on the current box
            for (int i = threadIdx.x; i < n0; i += blockDim.x) {
                const float g = r.sign * r.g[i];
                if (g == 0.f) continue;
                const ff t = ff_div(ff_neg(vlo), g);
                if (g > 0.f) {
                    ff c = ff_add(cl[i], t);
                    c = ff_add(c, ff_of(ff_step_err(cl[i].hi, t.hi)));
                    if (ff_lt(c, ch[i])) ch[i] = c;
                } else {
                    ff c = ff_add(ch[i], t);
                    c = ff_add(c, ff_of(-ff_step_err(ch[i].hi, t.hi)));
                    if (ff_lt(cl[i], c)) cl[i] = c;
                }
                if (ff_lt(ch[i], cl[i])) s_empty = 1;
            }
        }
        __syncthreads();
        if (s_empty) stop = true;
    }
    for (int i = threadIdx.x; i < n0; i += blockDim.x) {
        const float fl = ff_rd(cl[i]), fh = ff_ru(ch[i]);
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
                                  (int8_t*)(ws + lay->rowflag), (ff*)(ws + lay->vmin), infeasible,
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
                                     (const int8_t*)(ws + lay->rowflag), (const ff*)(ws + lay->vmin),
                                     lo_clip, hi_clip, infeasible, cache->net->status);
    CV_LAUNCH_CHECK("k_relaxed");
    return CV_OK;
}
