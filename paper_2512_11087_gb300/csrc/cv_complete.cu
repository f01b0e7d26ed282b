// Complete clipping (a6): the paper's Theorem 1 / Algorithm 1, coordinate ascent on the dual
//   max_{beta >= 0} (a + beta^T G).xhat - |a + beta^T G|.eps + c + beta^T h
// for both sides of every still-unstable target neuron of every subdomain, over the
// subdomain's active constraint rows and its clipped box, repeated for `sweeps` passes.
//
// One step for row k with the other multipliers fixed: breakpoints q_j = -a'_j / g_kj with
// weights w_j = |g_kj| eps_j; beta_k is the smallest breakpoint q* whose cumulative weight
// sum_{q_j <= q*} w_j reaches T_k = max_box(g_k.x + h_k) / 2 (the first non-positive
// supergradient), clamped at 0.  This is the sorted-breakpoint rule of Algorithm 1 written as
// a weighted quantile, so no sort is needed.  The quantile is found by shrinking a key bracket
// (lo, hi] with F(lo) < T <= F(hi): each pass takes the min and max breakpoint key inside it
// (done when they coincide) and splits it at the pivot interpolated from the weight still
// needed (after eight passes, every other pass halves the range instead, which bounds the
// count); the previous sweep's breakpoint is tried first (coordinate ascent mostly re-selects it).
//
// Decision arithmetic (reproduced by the oracle): a'_j = a_j + sum_{p != k} beta_p g_pj as an FP32
// fma chain over increasing p, q_j = (-a'_j) * fl(1/g_kj), compared through an order-preserving
// 32-bit key.  Weights are exact 64-bit fixed-point integers (w scaled by 2^s_k, s_k chosen so
// the row's total stays below 2^62), so every cumulative sum is exact and order independent and
// the quantile decision matches an FP64 evaluation; warp sums use three 21-bit redux.sync limbs.
// A sweep that changes no multiplier ends the ascent (the next would repeat it bit for bit); with
// a single row a' = a, so one pass suffices.  The bound is the dual objective at the final beta,
// evaluated in FP32 and padded by its rounding bound (any beta >= 0 gives a valid bound), or in
// FP64 when the padded value straddles 0 so that the stability decision is exact.
//
// GB300 mapping (persistent scheduling of uneven work): k_cc_prep writes each subdomain's active
// rows (g, 1/g, fixed-point weights, threshold) to the workspace once; a single-block scan turns
// the per-subdomain task counts into work items of TPI (target, side) tasks, subdomains with more
// rows first; a persistent k_complete grid (one block per resident slot) takes items from an
// atomic ticket, stages the item's rows in shared memory and runs one warp per task; each warp
// keeps its breakpoint keys in its own shared buffer, so the element loops stay short and rolled
// (small code, few registers, 32 resident warps per SM).
#include "cv_internal.cuh"

#include <climits>
#include <math.h>

namespace {

constexpr int RMAX_CC = 8;  // rows per subdomain handled by complete clipping
constexpr int TPI = 64;     // (target, side) tasks per work item
constexpr int NWARP = 16;   // warps per block

__device__ __forceinline__ unsigned fkey(float q) {
    unsigned u = __float_as_uint(q);
    return (u & 0x80000000u) ? ~u : (u | 0x80000000u);
}
__device__ __forceinline__ float fkey_inv(unsigned k) {
    unsigned u = (k & 0x80000000u) ? (k & 0x7fffffffu) : ~k;
    return __uint_as_float(u);
}

// Exact warp sum of non-negative per-lane 64-bit values whose total is below 2^62: three
// 21-bit limbs, each summed with one redux.sync (32 x 2^21 < 2^26, no overflow).
__device__ __forceinline__ long long warp_sum64(unsigned long long v) {
    const unsigned a = (unsigned)(v & 0x1fffffull);
    const unsigned b = (unsigned)((v >> 21) & 0x1fffffull);
    const unsigned c = (unsigned)(v >> 42);
    const unsigned A = __reduce_add_sync(0xffffffffu, a);
    const unsigned B = __reduce_add_sync(0xffffffffu, b);
    const unsigned C = __reduce_add_sync(0xffffffffu, c);
    return (long long)A + ((long long)B << 21) + ((long long)C << 42);
}

struct CCArgs {
    int B, U, n0, H, Rmax, Rs, sweeps;
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
    // workspace
    float* wg; float* wrg; long long* ww;   // [B][Rs][n0]
    long long* wT; double* wSg; float* wh;  // [B][Rs]
    int* wR;                                 // [B] active rows used
    int* wcnt;                               // [B] work items
    int* order;                              // [B] positions -> subdomains, more rows first
    int* ioff;                               // [B+1] first item of every position; [B] = total
    int* nplaced;                            // positions holding subdomains with work
    unsigned* ticket;
};

__device__ __forceinline__ int ntargets(const CCArgs& a, int b) {
    return a.tgt_off ? a.tgt_off[b + 1] - a.tgt_off[b] : a.U;
}

// Per subdomain: the first Rs active rows, their data in the workspace, and the item count.
__global__ void __launch_bounds__(256) k_cc_prep(CCArgs a) {
    const int b = blockIdx.x;
    const int n0 = a.n0, Rs = a.Rs;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    __shared__ int R, rowsel[RMAX_CC];
    if (threadIdx.x == 0) {
        int r = 0;
        if (!a.infeasible[b])
            for (int k = 0; k < a.Rmax && r < Rs; ++k)
                if (a.rowflag[(size_t)b * a.Rmax + k] == 0) rowsel[r++] = k;
        R = r;
        a.wR[b] = r;
        a.wcnt[b] = r > 0 ? (2 * ntargets(a, b) + TPI - 1) / TPI : 0;
    }
    __syncthreads();
    const int ns = a.split_off ? a.split_off[b + 1] - a.split_off[b] : 0;
    const float* lo = a.lo + (size_t)b * n0;
    const float* hi = a.hi + (size_t)b * n0;
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
        const size_t base = ((size_t)b * Rs + r) * n0;
        double smax = 0.0, wsum = 0.0, sgm = 0.0;
        for (int j = lane; j < n0; j += 32) {
            const float g = sg * gp[j];
            a.wg[base + j] = g;
            a.wrg[base + j] = (g != 0.f) ? 1.f / g : 0.f;
            const double gd = (double)g, l0 = (double)lo[j], h0 = (double)hi[j];
            smax += fmax(gd * l0, gd * h0);
            wsum += fabs(gd) * (0.5 * (h0 - l0));
            sgm += fabs(gd) * fmax(fabs((double)a.root_lo[j]), fabs((double)a.root_hi[j]));
        }
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) {
            smax += __shfl_xor_sync(0xffffffffu, smax, off);
            wsum += __shfl_xor_sync(0xffffffffu, wsum, off);
            sgm += __shfl_xor_sync(0xffffffffu, sgm, off);
        }
        // fixed-point weights: scale so that the row total stays below 2^62
        const int sh = (wsum > 0.0) ? 61 - ilogb(wsum) : 0;
        for (int j = lane; j < n0; j += 32) {
            const double w = fabs((double)sg * (double)gp[j]) * (0.5 * ((double)hi[j] - (double)lo[j]));
            a.ww[base + j] = __double2ll_rn(ldexp(w, sh));
        }
        if (lane == 0) {
            const double T = 0.5 * (smax + (double)hh);
            a.wT[(size_t)b * Rs + r] = (T <= 0.0) ? LLONG_MIN : __double2ll_ru(ldexp(T, sh));
            a.wh[(size_t)b * Rs + r] = hh;
            a.wSg[(size_t)b * Rs + r] = sgm;
        }
    }
}

// Work-item offsets with the subdomains ordered by decreasing row count (longest tasks first).
__global__ void __launch_bounds__(1024) k_cc_scan(CCArgs a) {
    __shared__ int sc[1024], si[1024];
    __shared__ int placed, carry;
    const int B = a.B, tid = threadIdx.x, nt = blockDim.x;
    const int per = (B + nt - 1) / nt;
    if (tid == 0) { placed = 0; carry = 0; }
    __syncthreads();
    for (int v = a.Rs; v >= 1; --v) {
        int c = 0, s = 0;
        for (int i = 0; i < per; ++i) {
            const int b = tid * per + i;
            if (b < B && a.wR[b] == v) { ++c; s += a.wcnt[b]; }
        }
        sc[tid] = c;
        si[tid] = s;
        __syncthreads();
        for (int off = 1; off < nt; off <<= 1) {  // inclusive scans
            const int tc = tid >= off ? sc[tid - off] : 0;
            const int ts = tid >= off ? si[tid - off] : 0;
            __syncthreads();
            sc[tid] += tc;
            si[tid] += ts;
            __syncthreads();
        }
        int pos = placed + sc[tid] - c;
        int ib = carry + si[tid] - s;
        for (int i = 0; i < per; ++i) {
            const int b = tid * per + i;
            if (b < B && a.wR[b] == v) {
                a.order[pos] = b;
                a.ioff[pos] = ib;
                ib += a.wcnt[b];
                ++pos;
            }
        }
        __syncthreads();
        if (tid == 0) { placed += sc[nt - 1]; carry += si[nt - 1]; }
        __syncthreads();
    }
    for (int i = placed + tid; i < B; i += nt) { a.ioff[i] = carry; a.order[i] = -1; }
    if (tid == 0) {
        a.ioff[B] = carry;
        *a.nplaced = placed;
        *a.ticket = 0u;
    }
}

__global__ void __launch_bounds__(NWARP * 32, 2) k_complete(CCArgs a) {
    extern __shared__ __align__(16) unsigned char smem[];
    const int n0 = a.n0, Rs = a.Rs, B = a.B;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int n0r = (n0 + 31) & ~31;
    // shared: w64 [Rs][n0] | g [Rs][n0] | rg [Rs][n0] | lo [n0] | hi [n0] | keys [NWARP][n0r]
    long long* w64 = (long long*)smem;
    float* gs = (float*)(w64 + (size_t)Rs * n0);
    float* rg = gs + (size_t)Rs * n0;
    float* slo = rg + (size_t)Rs * n0;
    float* shi = slo + n0;
    unsigned* keys = (unsigned*)(shi + n0) + (size_t)warp * n0r;  // this warp's breakpoint keys
    __shared__ long long T64[RMAX_CC];
    __shared__ float hrow[RMAX_CC];
    __shared__ double Sg[RMAX_CC];
    __shared__ float sbeta[NWARP][RMAX_CC];  // per warp: multipliers of the current task
    __shared__ int sjprev[NWARP][RMAX_CC];   // per warp: element of the last selected breakpoint
    __shared__ int s_item, s_pos, s_R;
    __shared__ unsigned long long nsteps;
    if (threadIdx.x == 0) nsteps = 0;
    unsigned long long my_steps = 0;
    const unsigned KZERO = 0x80000000u;  // key(+0.0)
    const unsigned KINF = 0xff800000u;   // key(+inf)
    const int total = a.ioff[B];
    const int np = *a.nplaced;
    int cur_b = -1;
    for (;;) {
        __syncthreads();
        if (threadIdx.x == 0) {
            const int it = (int)atomicAdd(a.ticket, 1u);
            s_item = it;
            if (it < total) {
                int lo = 0, hi = np - 1;  // last position whose first item is <= it
                while (lo < hi) {
                    const int mid = (lo + hi + 1) >> 1;
                    if (a.ioff[mid] <= it) lo = mid; else hi = mid - 1;
                }
                s_pos = lo;
            }
        }
        __syncthreads();
        const int item = s_item;
        if (item >= total) break;
        const int pos = s_pos;
        const int b = a.order[pos];
        if (b != cur_b) {
            // stage the subdomain's rows and clipped box
            if (threadIdx.x == 0) s_R = a.wR[b];
            __syncthreads();
            const int R = s_R;
            const size_t base = (size_t)b * Rs * n0;
            for (int i = threadIdx.x; i < R * n0; i += blockDim.x) {
                w64[i] = a.ww[base + i];
                gs[i] = a.wg[base + i];
                rg[i] = a.wrg[base + i];
            }
            for (int i = threadIdx.x; i < n0; i += blockDim.x) {
                slo[i] = a.lo[(size_t)b * n0 + i];
                shi[i] = a.hi[(size_t)b * n0 + i];
            }
            if (threadIdx.x < R) {
                T64[threadIdx.x] = a.wT[(size_t)b * Rs + threadIdx.x];
                hrow[threadIdx.x] = a.wh[(size_t)b * Rs + threadIdx.x];
                Sg[threadIdx.x] = a.wSg[(size_t)b * Rs + threadIdx.x];
            }
            cur_b = b;
            __syncthreads();
        }
        const int R = s_R;
        const bool have_list = a.tgt_off != nullptr;
        const int t0 = have_list ? a.tgt_off[b] : 0;
        const int ntask = 2 * ntargets(a, b);
        const int first = (item - a.ioff[pos]) * TPI;
        const int last = min(first + TPI, ntask);
        for (int task = first + warp; task < last; task += NWARP) {
            const int ti = task >> 1, side = task & 1;
            const int c = have_list ? a.tgt_ids[t0 + ti] : ti;
            if (c < 0 || c >= a.U) { if (lane == 0) atomicOr(a.status, CV_DEV_TARGET); continue; }
            const size_t o = (size_t)b * a.U + c;
            if (a.mask[o] != 0) continue;
            const float* ap = side ? a.uA + (size_t)c * n0 : a.lA + (size_t)c * n0;
            const float sa = side ? -1.f : 1.f;
            const float c0 = side ? -a.uc[c] : a.lc[c];
            float* beta = sbeta[warp];
            int* jprev = sjprev[warp];
            if (lane < RMAX_CC) { beta[lane] = 0.f; jprev[lane] = -1; }
            __syncwarp();
            // with one row, a' = a in every sweep, so one pass already repeats bit for bit
            const int nsweeps = (R == 1) ? 1 : a.sweeps;
            for (int sw = 0; sw < nsweeps; ++sw) {
                bool changed = false;
                my_steps += R;
                for (int k = 0; k < R; ++k) {
                    const float* rk = rg + (size_t)k * n0;
                    const long long* wk = w64 + (size_t)k * n0;
                    const int jp = jprev[k];
                    // a' = a + sum_{p != k} beta_p g_p (fma chain in increasing p), key of q = -a' / g_k
                    auto key_of = [&](int j) -> unsigned {
                        float apr = sa * ap[j];
                        for (int p = 0; p < R; ++p)
                            if (p != k) apr = fmaf(beta[p], gs[(size_t)p * n0 + j], apr);
                        const float r = rk[j];
                        return (r != 0.f) ? fkey(-apr * r) : 0xffffffffu;
                    };
                    unsigned kp = 0xffffffffu;
                    if (jp >= 0) kp = __shfl_sync(0xffffffffu, key_of(jp), 0);
                    const bool warm = kp > KZERO && kp <= KINF;
                    // F(x) = sum of the weights of the breakpoints with key <= x (exact integers)
                    unsigned long long f0 = 0, ftot = 0, flt = 0, fle = 0;
                    if (warm) {
                        for (int j = lane; j < n0; j += 32) {
                            const unsigned kk = key_of(j);
                            keys[j] = kk;
                            const unsigned long long w = (unsigned long long)wk[j];
                            f0 += (kk <= KZERO) ? w : 0ull;
                            ftot += (kk <= KINF) ? w : 0ull;
                            flt += (kk < kp) ? w : 0ull;
                            fle += (kk <= kp) ? w : 0ull;
                        }
                    } else {
                        for (int j = lane; j < n0; j += 32) {
                            const unsigned kk = key_of(j);
                            keys[j] = kk;
                            const unsigned long long w = (unsigned long long)wk[j];
                            f0 += (kk <= KZERO) ? w : 0ull;
                            ftot += (kk <= KINF) ? w : 0ull;
                        }
                    }
                    __syncwarp();
                    const long long T = T64[k];
                    const long long F0 = warp_sum64(f0), Ftot = warp_sum64(ftot);
                    long long Flt = 0, Fle = 0;
                    if (warm) { Flt = warp_sum64(flt); Fle = warp_sum64(fle); }
                    float bn = 0.f;
                    int jn = -1;
                    if (F0 >= T || Ftot < T) {
                        // beta = 0 (slope at 0+ not positive; or a row infeasible on this machine)
                    } else if (warm && Flt < T && T <= Fle) {
                        bn = fkey_inv(kp);  // the same breakpoint as last time
                        jn = jp;
                    } else {
                        // bracket (lo, hi] with F(lo) < T <= F(hi)
                        unsigned lo = KZERO, hi = KINF;
                        long long Flo = F0, Fhi = Ftot;
                        if (warm) {
                            if (Fle < T) { lo = kp; Flo = Fle; }
                            else { hi = kp - 1; Fhi = Flt; }
                        }
                        // shrink to a single breakpoint key: each pass takes the min and max key in the
                        // bracket (done when equal) and splits at the pivot interpolated from the weight
                        // still needed (halving every other pass after the eighth)
                        unsigned ks = 0;
                        for (int it = 0; it < 96; ++it) {
                            unsigned cmin = 0xffffffffu, cmax = 0u;
                            for (int j = lane; j < n0; j += 32) {
                                const unsigned kk = keys[j];
                                if (kk > lo && kk <= hi) { cmin = min(cmin, kk); cmax = max(cmax, kk); }
                            }
                            cmin = __reduce_min_sync(0xffffffffu, cmin);
                            cmax = __reduce_max_sync(0xffffffffu, cmax);
                            if (cmin == cmax) { ks = cmin; break; }
                            lo = cmin - 1;  // F unchanged: no breakpoint in (lo, cmin)
                            hi = cmax;      // F unchanged: no breakpoint in (cmax, hi]
                            unsigned mid;
                            if (it >= 8 && (it & 1)) {
                                mid = lo + ((hi - lo) >> 1);
                            } else {
                                const float fr = (float)(T - Flo) / (float)(Fhi - Flo);
                                unsigned off = (unsigned)(fr * (float)(hi - lo));
                                off = min(max(off, 1u), hi - lo - 1);
                                mid = lo + off;
                            }
                            unsigned long long fm = 0;
                            for (int j = lane; j < n0; j += 32)
                                fm += (keys[j] <= mid) ? (unsigned long long)wk[j] : 0ull;
                            const long long Fm = warp_sum64(fm);
                            if (Fm >= T) { hi = mid; Fhi = Fm; }
                            else { lo = mid; Flo = Fm; }
                        }
                        bn = fkey_inv(ks);
                        if (!(bn > 0.f)) bn = 0.f;
                        // the element holding the selected breakpoint (lowest index among ties)
                        jn = -1;
                        for (int j0 = 0; j0 < n0 && jn < 0; j0 += 32) {
                            const int j = j0 + lane;
                            const unsigned bal = __ballot_sync(0xffffffffu, j < n0 && keys[j] == ks);
                            if (bal) jn = j0 + __ffs(bal) - 1;
                        }
                    }
                    const float bk = beta[k];
                    __syncwarp();
                    if (lane == 0) { jprev[k] = jn; beta[k] = bn; }
                    __syncwarp();
                    changed |= (bn != bk);
                }
                if (!changed) break;
            }
            // dual objective at beta, FP32 with its rounding bound
            float part = 0.f;
            for (int j = lane; j < n0; j += 32) {
                float v = sa * ap[j];
                for (int k = 0; k < R; ++k) v = fmaf(beta[k], gs[(size_t)k * n0 + j], v);
                part += fminf(v * slo[j], v * shi[j]);
            }
#pragma unroll
            for (int off = 16; off > 0; off >>= 1) part += __shfl_xor_sync(0xffffffffu, part, off);
            float cst = c0;
            double scale = (double)a.pscale[side ? a.U + c : c] + fabs((double)c0);
            for (int k = 0; k < R; ++k) {
                cst = fmaf(beta[k], hrow[k], cst);
                scale += (double)beta[k] * (Sg[k] + fabs((double)hrow[k]));
            }
            const double gam = (double)(R + (n0 + 31) / 32 + 12) * CV_U32;
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
            __syncwarp();
        }
    }
    if (a.steps && lane == 0 && my_steps) atomicAdd(&nsteps, my_steps);
    __syncthreads();
    if (a.steps && threadIdx.x == 0 && nsteps) atomicAdd(a.steps, nsteps);
}

// stability of the targets after clipping; l > u means the subdomain is empty
__global__ void k_cc_post(CCArgs a) {
    const int b = blockIdx.x;
    if (a.wR[b] == 0) return;
    const bool have_list = a.tgt_off != nullptr;
    const int t0 = have_list ? a.tgt_off[b] : 0;
    const int nt = ntargets(a, b);
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

cv_status launch_cc(const CCArgs& a, int* launches, cudaStream_t st) {
    const size_t n0r = (a.n0 + 31) & ~31;
    const size_t smem = (size_t)a.Rs * a.n0 * (8 + 4 + 4) + 2 * (size_t)a.n0 * 4 + (size_t)NWARP * n0r * 4;
    if (smem > 220 * 1024) {
        cv_set_error("complete clipping: input dimension too large for the shared-memory row cache");
        return CV_EUNSUPPORTED;
    }
    CV_CUDA(cudaFuncSetAttribute(k_complete, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    int dev = 0, sms = 0, per = 0;
    CV_CUDA(cudaGetDevice(&dev));
    CV_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    CV_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_complete, NWARP * 32, smem));
    if (per < 1) per = 1;
    k_complete<<<sms * per, NWARP * 32, smem, st>>>(a);
    CV_LAUNCH_CHECK("k_complete");
    ++*launches;
    return CV_OK;
}

}  // namespace

size_t cv_cc_workspace(int B, int Rmax, int n0) {
    const size_t Rs = Rmax < RMAX_CC ? Rmax : RMAX_CC;
    if (Rs == 0) return 0;
    const size_t b = B;
    size_t s = 0;
    s += cv_align256(b * Rs * n0 * 4) * 2;  // wg, wrg
    s += cv_align256(b * Rs * n0 * 8);      // ww
    s += cv_align256(b * Rs * 8) * 2;       // wT, wSg
    s += cv_align256(b * Rs * 4);           // wh
    s += cv_align256(b * 4) * 3;            // wR, wcnt, order
    s += cv_align256((b + 1) * 4);          // ioff
    s += 256 * 2;                           // nplaced, ticket
    return s;
}

cv_status cv_launch_complete(const cv_net* net, const cv_cache* cache, const cv_batch_in* in,
                             const cv_options* opt, const cv_ws_layout* lay, char* ws,
                             const float* lo_clip, const float* hi_clip, float* l, float* u,
                             int8_t* mask, uint8_t* infeasible, unsigned long long* step_counter,
                             int* launches, cudaStream_t st) {
    if (opt->sweeps <= 0 || lay->Rmax == 0 || cache->U == 0) return CV_OK;
    if (lay->Rmax > RMAX_CC) {
        cv_set_error("complete clipping: more than 8 constraint rows per subdomain is not supported by this build");
        return CV_EUNSUPPORTED;
    }
    CCArgs a;
    a.B = in->B; a.U = cache->U; a.n0 = cache->n0; a.H = cache->H; a.Rmax = lay->Rmax; a.sweeps = opt->sweeps;
    a.Rs = lay->Rmax < RMAX_CC ? lay->Rmax : RMAX_CC;
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
    // workspace carve (the layout of cv_cc_workspace)
    const size_t B = in->B, Rs = a.Rs, n0 = cache->n0;
    char* p = ws + lay->cc;
    a.wg = (float*)p; p += cv_align256(B * Rs * n0 * 4);
    a.wrg = (float*)p; p += cv_align256(B * Rs * n0 * 4);
    a.ww = (long long*)p; p += cv_align256(B * Rs * n0 * 8);
    a.wT = (long long*)p; p += cv_align256(B * Rs * 8);
    a.wSg = (double*)p; p += cv_align256(B * Rs * 8);
    a.wh = (float*)p; p += cv_align256(B * Rs * 4);
    a.wR = (int*)p; p += cv_align256(B * 4);
    a.wcnt = (int*)p; p += cv_align256(B * 4);
    a.order = (int*)p; p += cv_align256(B * 4);
    a.ioff = (int*)p; p += cv_align256((B + 1) * 4);
    a.nplaced = (int*)p; p += 256;
    a.ticket = (unsigned*)p;
    k_cc_prep<<<in->B, 256, 0, st>>>(a);
    CV_LAUNCH_CHECK("k_cc_prep");
    k_cc_scan<<<1, 1024, 0, st>>>(a);
    CV_LAUNCH_CHECK("k_cc_scan");
    *launches += 3;  // prep, scan, post
    cv_status s = launch_cc(a, launches, st);
    if (s) return s;
    k_cc_post<<<in->B, 256, 0, st>>>(a);
    CV_LAUNCH_CHECK("k_cc_post");
    return CV_OK;
}
