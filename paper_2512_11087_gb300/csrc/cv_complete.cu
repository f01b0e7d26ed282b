// Complete clipping (a6): the paper's Theorem 1 / Algorithm 1, coordinate ascent on the dual
//   max_{beta >= 0} (a + beta^T G).xhat - |a + beta^T G|.eps + c + beta^T h
// for both sides of every still-unstable target neuron of every subdomain, over the
// subdomain's active constraint rows and its clipped box, repeated for `sweeps` passes.
//
// One step for row k with the other multipliers fixed: breakpoints q_j = -a'_j / g_kj with
// weights w_j = |g_kj| eps_j; beta_k is the smallest breakpoint q* whose cumulative weight
// sum_{q_j <= q*} w_j reaches T_k = max_box(g_k.x + h_k) / 2 (the first non-positive
// supergradient), clamped at 0.  This is the sorted-breakpoint rule of Algorithm 1 written as
// a weighted quantile, so no sort is needed.
//
// GB300 mapping: one CTA per subdomain; the subdomain's rows (g, 1/g, weights) live in shared
// memory; one warp owns one (target, side) problem with a' held in registers (n0/32 values per
// lane).  Weights are exact 64-bit fixed-point integers (w scaled by 2^s_k, s_k chosen so the
// row's total stays below 2^62): every cumulative sum is exact and order independent, so the
// quantile decision matches an FP64 evaluation.  The quantile is found by bisection on the
// order-preserving 32-bit key of q.  A sweep that changes no multiplier ends the ascent (the
// next sweep would repeat it bit for bit).  The bound is the dual objective at the final beta,
// evaluated in FP32 and padded by its rounding bound (any beta >= 0 gives a valid bound).
#include "cv_internal.cuh"

#include <climits>
#include <math.h>

namespace {

constexpr int RMAX_CC = 8;  // rows held in shared memory per subdomain

__device__ __forceinline__ unsigned fkey(float q) {
    unsigned u = __float_as_uint(q);
    return (u & 0x80000000u) ? ~u : (u | 0x80000000u);
}
__device__ __forceinline__ float fkey_inv(unsigned k) {
    unsigned u = (k & 0x80000000u) ? (k & 0x7fffffffu) : ~k;
    return __uint_as_float(u);
}

__device__ __forceinline__ long long warp_sum64(long long v) {
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
    return v;
}

struct CCArgs {
    int B, U, n0, H, Rmax, sweeps;
    const int8_t* rowflag;
    const float* lA; const float* lc; const float* uA; const float* uc;
    const int* slot_of; const float* pscale;
    const float* root_lo; const float* root_hi;
    const int* split_off; const int* split_ids;
    const int* row_off; const float* G; const float* h;
    const int* tgt_off; const int* tgt_ids;
    const float* lo; const float* hi;
    float* l; float* u; int8_t* mask; uint8_t* infeasible; int* status;
    unsigned long long* steps;  // optional counter of executed row steps
};

template <int NE>
__global__ void __launch_bounds__(256) k_complete(CCArgs a) {
    extern __shared__ __align__(16) unsigned char smem[];
    const int b = blockIdx.x;
    if (a.infeasible[b]) return;
    const int n0 = a.n0;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    // shared layout: w64 [R][n0] | g [R][n0] | rg [R][n0] | lo [n0] | hi [n0] | per-row scalars
    long long* w64 = (long long*)smem;
    float* gs = (float*)(w64 + (size_t)RMAX_CC * n0);
    float* rg = gs + (size_t)RMAX_CC * n0;
    float* slo = rg + (size_t)RMAX_CC * n0;
    float* shi = slo + n0;
    __shared__ long long T64[RMAX_CC];
    __shared__ float hrow[RMAX_CC], sgrow[RMAX_CC];
    __shared__ double Wrow[RMAX_CC], Vmax[RMAX_CC], Sg[RMAX_CC];
    __shared__ int R, rowsel[RMAX_CC];

    if (threadIdx.x == 0) {
        int r = 0;
        for (int k = 0; k < a.Rmax && r < RMAX_CC; ++k)
            if (a.rowflag[(size_t)b * a.Rmax + k] == 0) rowsel[r++] = k;
        R = r;
    }
    for (int i = threadIdx.x; i < n0; i += blockDim.x) {
        slo[i] = a.lo[(size_t)b * n0 + i];
        shi[i] = a.hi[(size_t)b * n0 + i];
    }
    __syncthreads();
    if (R == 0) return;
    const int ns = a.split_off ? a.split_off[b + 1] - a.split_off[b] : 0;
    // rows into shared memory; per-row FP64 reductions by one warp each
    for (int r = warp; r < R; r += nw) {
        const int k = rowsel[r];
        const float* gp; float sg, hh;
        if (k < ns) {
            const int code = a.split_ids[a.split_off[b] + k];
            const int g = (code > 0 ? code : -code) - 1;
            const int slot = a.slot_of[g];
            if (code > 0) { gp = a.uA + (size_t)slot * n0; sg = -1.f; hh = -a.uc[slot]; }
            else { gp = a.lA + (size_t)slot * n0; sg = 1.f; hh = a.lc[slot]; }
        } else {
            const int row = a.row_off[b] + (k - ns);
            gp = a.G + (size_t)row * n0; sg = 1.f; hh = a.h[row];
        }
        double smax = 0.0, wsum = 0.0, sgm = 0.0;
        for (int j = lane; j < n0; j += 32) {
            const float g = sg * gp[j];
            gs[(size_t)r * n0 + j] = g;
            rg[(size_t)r * n0 + j] = (g != 0.f) ? 1.f / g : 0.f;
            const double gd = (double)g, lo = (double)slo[j], hi = (double)shi[j];
            smax += fmax(gd * lo, gd * hi);
            wsum += fabs(gd) * (0.5 * (hi - lo));
            sgm += fabs(gd) * fmax(fabs((double)a.root_lo[j]), fabs((double)a.root_hi[j]));
        }
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) {
            smax += __shfl_xor_sync(0xffffffffu, smax, off);
            wsum += __shfl_xor_sync(0xffffffffu, wsum, off);
            sgm += __shfl_xor_sync(0xffffffffu, sgm, off);
        }
        if (lane == 0) {
            Vmax[r] = smax + (double)hh;
            Wrow[r] = wsum;
            Sg[r] = sgm;
            hrow[r] = hh;
            sgrow[r] = sg;
        }
    }
    __syncthreads();
    // fixed-point weights: scale so that the row total stays below 2^62
    for (int r = warp; r < R; r += nw) {
        const int sh = (Wrow[r] > 0.0) ? 61 - ilogb(Wrow[r]) : 0;
        for (int j = lane; j < n0; j += 32) {
            const double w = fabs((double)gs[(size_t)r * n0 + j]) * (0.5 * ((double)shi[j] - (double)slo[j]));
            w64[(size_t)r * n0 + j] = __double2ll_rn(ldexp(w, sh));
        }
        if (lane == 0) {
            const double T = 0.5 * Vmax[r];
            T64[r] = (T <= 0.0) ? LLONG_MIN : __double2ll_ru(ldexp(T, sh));
        }
    }
    __syncthreads();

    // tasks: (target, side)
    const bool have_list = a.tgt_off != nullptr;
    const int t0 = have_list ? a.tgt_off[b] : 0;
    const int nt = have_list ? a.tgt_off[b + 1] - t0 : a.U;
    __shared__ unsigned long long nsteps;
    if (threadIdx.x == 0) nsteps = 0;
    __syncthreads();
    unsigned long long my_steps = 0;
    const unsigned KZERO = 0x80000000u;         // key(+0.0)
    const unsigned KINF = 0xff800000u;          // key(+inf)
    for (int task = warp; task < 2 * nt; task += nw) {
        const int ti = task >> 1, side = task & 1;
        const int c = have_list ? a.tgt_ids[t0 + ti] : ti;
        if (c < 0 || c >= a.U) { if (lane == 0) atomicOr(a.status, CV_DEV_TARGET); continue; }
        const size_t o = (size_t)b * a.U + c;
        if (a.mask[o] != 0) continue;
        const float* ap = side ? a.uA + (size_t)c * n0 : a.lA + (size_t)c * n0;
        const float sa = side ? -1.f : 1.f;
        const float c0 = side ? -a.uc[c] : a.lc[c];
        float af[NE];
#pragma unroll
        for (int e = 0; e < NE; ++e) {
            const int j = lane + 32 * e;
            af[e] = (j < n0) ? sa * ap[j] : 0.f;
        }
        float beta[RMAX_CC];
#pragma unroll
        for (int k = 0; k < RMAX_CC; ++k) beta[k] = 0.f;
        for (int sw = 0; sw < a.sweeps; ++sw) {
            bool changed = false;
            my_steps += R;
            for (int k = 0; k < R; ++k) {
                const float* gk = gs + (size_t)k * n0;
                const float* rk = rg + (size_t)k * n0;
                const long long* wk = w64 + (size_t)k * n0;
                const float bk = beta[k];
                unsigned key[NE];
                long long f0 = 0;
#pragma unroll
                for (int e = 0; e < NE; ++e) {
                    const int j = lane + 32 * e;
                    if (j < n0) {
                        const float apr = fmaf(-bk, gk[j], af[e]);  // a' = a + sum_{p != k} beta_p g_p
                        const float r = rk[j];
                        key[e] = (r != 0.f) ? fkey(-apr * r) : 0xffffffffu;
                        if (key[e] <= KZERO) f0 += wk[j];
                    } else { key[e] = 0xffffffffu; }
                }
                f0 = warp_sum64(f0);
                const long long T = T64[k];
                float bn = 0.f;
                if (f0 < T) {
                    // F(KINF) < T only for a row infeasible on this machine: beta stays 0
                    long long ftot = 0;
#pragma unroll
                    for (int e = 0; e < NE; ++e) {
                        const int j = lane + 32 * e;
                        if (j < n0 && key[e] <= KINF) ftot += wk[j];
                    }
                    ftot = warp_sum64(ftot);
                    if (ftot >= T) {
                        unsigned lo = KZERO + 1, hi = KINF;
                        while (lo < hi) {
                            const unsigned mid = lo + ((hi - lo) >> 1);
                            long long f = 0;
#pragma unroll
                            for (int e = 0; e < NE; ++e) {
                                const int j = lane + 32 * e;
                                if (j < n0 && key[e] <= mid) f += wk[j];
                            }
                            f = warp_sum64(f);
                            if (f >= T) hi = mid; else lo = mid + 1;
                        }
                        bn = fkey_inv(lo);
                        if (!(bn > 0.f)) bn = 0.f;
                    }
                }
                if (bn != bk) {
#pragma unroll
                    for (int e = 0; e < NE; ++e) {
                        const int j = lane + 32 * e;
                        if (j < n0) af[e] = fmaf(bn, gk[j], fmaf(-bk, gk[j], af[e]));
                    }
                    beta[k] = bn;
                    changed = true;
                }
            }
            if (!changed) break;
        }
        // dual objective at beta, FP32 with its rounding bound
        float part = 0.f;
#pragma unroll
        for (int e = 0; e < NE; ++e) {
            const int j = lane + 32 * e;
            if (j < n0) {
                float v = sa * ap[j];
                for (int k = 0; k < R; ++k) v = fmaf(beta[k], gs[(size_t)k * n0 + j], v);
                part += fminf(v * slo[j], v * shi[j]);
            }
        }
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) part += __shfl_xor_sync(0xffffffffu, part, off);
        float cst = c0;
        double scale = (double)a.pscale[side ? a.U + c : c] + fabs((double)c0);
        for (int k = 0; k < R; ++k) {
            cst = fmaf(beta[k], hrow[k], cst);
            scale += (double)beta[k] * (Sg[k] + fabs((double)hrow[k]));
        }
        const double gam = (double)(R + NE + 12) * CV_U32;
        const float pad = __double2float_ru(gam * scale * 1.0001);
        float val = __fsub_rd(__fadd_rd(part, cst), pad);
        const float valhi = __fadd_ru(__fadd_ru(part, cst), pad);
        const float cur = side == 0 ? a.l[o] : -a.u[o];
        if (val < 0.f && valhi >= 0.f && cur < 0.f) {
            // the stability decision is uncertain in FP32: evaluate D(beta) in FP64
            double d = 0.0;
            for (int j = lane; j < n0; j += 32) {
                double v = (double)(sa * ap[j]);
                for (int k = 0; k < R; ++k) v += (double)beta[k] * (double)gs[(size_t)k * n0 + j];
                d += fmin(v * (double)slo[j], v * (double)shi[j]);
            }
#pragma unroll
            for (int off = 16; off > 0; off >>= 1) d += __shfl_xor_sync(0xffffffffu, d, off);
            d += (double)c0;
            for (int k = 0; k < R; ++k) d += (double)beta[k] * (double)hrow[k];
            val = __double2float_rd(d - ldexp(scale, -40));
        }
        if (lane == 0) {
            if (side == 0) { if (val > a.l[o]) a.l[o] = val; }
            else { const float ub = -val; if (ub < a.u[o]) a.u[o] = ub; }
        }
    }
    if (a.steps && lane == 0 && my_steps) atomicAdd(&nsteps, my_steps);
    __syncthreads();
    if (a.steps && threadIdx.x == 0 && nsteps) atomicAdd(a.steps, nsteps);
    // stability of the targets after clipping; l > u means the subdomain is empty
    __shared__ int bad;
    if (threadIdx.x == 0) bad = 0;
    __syncthreads();
    for (int ti = threadIdx.x; ti < nt; ti += blockDim.x) {
        const int c = have_list ? a.tgt_ids[t0 + ti] : ti;
        if (c < 0 || c >= a.U) continue;
        const size_t o = (size_t)b * a.U + c;
        if (a.mask[o] == 0) a.mask[o] = (a.l[o] >= 0.f) ? 1 : ((a.u[o] <= 0.f) ? -1 : 0);
        if (a.l[o] > a.u[o]) bad = 1;
    }
    __syncthreads();
    if (threadIdx.x == 0 && bad) a.infeasible[b] = 1;
}

template <int NE>
cv_status launch_ne(const CCArgs& a, cudaStream_t st) {
    const size_t smem = (size_t)RMAX_CC * a.n0 * (8 + 4 + 4) + 2 * (size_t)a.n0 * 4;
    if (smem > 200 * 1024) {
        cv_set_error("complete clipping: input dimension too large for the shared-memory row cache");
        return CV_EUNSUPPORTED;
    }
    cudaFuncSetAttribute(k_complete<NE>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    k_complete<NE><<<a.B, 256, smem, st>>>(a);
    CV_LAUNCH_CHECK("k_complete");
    return CV_OK;
}

}  // namespace

cv_status cv_launch_complete(const cv_net* net, const cv_cache* cache, const cv_batch_in* in,
                             const cv_options* opt, const cv_ws_layout* lay, char* ws,
                             const float* lo_clip, const float* hi_clip, float* l, float* u,
                             int8_t* mask, uint8_t* infeasible, unsigned long long* step_counter,
                             int* launches, cudaStream_t st) {
    if (opt->sweeps <= 0 || lay->Rmax == 0 || cache->U == 0) return CV_OK;
    ++*launches;
    if (lay->Rmax > RMAX_CC) {
        cv_set_error("complete clipping: more than 8 constraint rows per subdomain is not supported by this build");
        return CV_EUNSUPPORTED;
    }
    CCArgs a;
    a.B = in->B; a.U = cache->U; a.n0 = cache->n0; a.H = cache->H; a.Rmax = lay->Rmax; a.sweeps = opt->sweeps;
    a.rowflag = (const int8_t*)(ws + lay->rowflag);
    a.lA = cache->lA; a.lc = cache->lc; a.uA = cache->uA; a.uc = cache->uc;
    a.slot_of = cache->slot_of; a.pscale = cache->pscale;
    a.root_lo = cache->root_lo; a.root_hi = cache->root_hi;
    a.split_off = in->split_off; a.split_ids = in->split_ids;
    a.row_off = in->row_off; a.G = in->G; a.h = in->h;
    a.tgt_off = in->tgt_off; a.tgt_ids = in->tgt_ids;
    a.lo = lo_clip; a.hi = hi_clip;
    a.l = l; a.u = u; a.mask = mask; a.infeasible = infeasible; a.status = net->status;
    a.steps = step_counter;
    const int ne = (cache->n0 + 31) / 32;
    if (ne <= 1) return launch_ne<1>(a, st);
    if (ne <= 2) return launch_ne<2>(a, st);
    if (ne <= 4) return launch_ne<4>(a, st);
    if (ne <= 8) return launch_ne<8>(a, st);
    if (ne <= 16) return launch_ne<16>(a, st);
    if (ne <= 25) return launch_ne<25>(a, st);
    if (ne <= 32) return launch_ne<32>(a, st);
    cv_set_error("complete clipping: input dimension above 1024 is not supported by this build");
    return CV_EUNSUPPORTED;
}
