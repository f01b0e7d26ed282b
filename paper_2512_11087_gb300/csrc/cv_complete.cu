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
// (lo, hi] with F(lo) < T <= F(hi): the first pass over a large bracket takes F at two pivots
// drawn from a 32-breakpoint sample around the target rank and keeps the slice between them;
// each later pass takes the min and max breakpoint key inside the bracket (done when they
// coincide) and splits it at the pivot interpolated from the weight still needed (after eight
// passes, every other pass halves the range instead, which bounds the count); the previous
// sweep's breakpoint is tried first (coordinate ascent mostly re-selects it).
//
// Decision arithmetic: a'_j = a_j + sum_{p != k} beta_p g_pj as an FP32 fma chain over increasing p
// from the leading FP32 parts of the multipliers, q_j = (-a'_j) * fl(1/g_kj); breakpoints with q > 0
// are compared through the raw bits of q (for positive floats the unsigned order of the bits is the
// order of the values).  Weights are exact 64-bit fixed-point integers (w scaled by 2^s_k, s_k chosen
// so the row's total stays below 2^62), so every cumulative sum is exact and order independent;
// warp sums use three 21-bit redux.sync limbs.  With one row a' = a exactly and one pass is the whole
// ascent; the selected breakpoint is then within a few FP32 ulps of the exact one.  With two or more
// rows the FP32 decision of every row step is certified against the a-priori error of the keys: the
// elements whose breakpoints could be ordered differently in exact arithmetic are re-decided on
// float-float breakpoints, and the multipliers are kept as float-float sums (beta_hi + beta_lo), so
// the ascent follows the paper's FP64 sorted-breakpoint rule (only breakpoints equal to within about
// 2^-44 of their magnitude can be ordered differently).  A row step whose inputs (the other rows'
// multipliers) did not change since its last step is skipped, and a sweep that changes no multiplier
// ends the ascent: both would repeat the previous result exactly.  The bound is the dual objective at
// the leading parts of the final multipliers, evaluated in FP32 and padded by its rounding bound
// (any beta >= 0 gives a valid bound), or in FP64 when the padded value straddles 0 so that the
// stability decision is exact.  With every multiplier 0 it equals the re-concretised bound already
// stored, and is skipped.
//
// GB300 mapping (persistent scheduling of uneven work): k_cc_prep writes each subdomain's active
// rows (g, 1/g, fixed-point weights, threshold, total weight) to the workspace once; a
// single-block scan turns the per-subdomain task counts into work items (by default 256 (target,
// side) tasks for one row, 64 for two, 16 for more: longer tasks, smaller items; the cache holds
// the sizes, which cv_cc_items_set and the autotuner change), subdomains with more rows first; a
// persistent k_complete grid (two blocks of 12 warps per SM) takes items from an atomic ticket,
// stages the item's rows in shared memory, and its warps take the item's tasks one at a time from
// a shared counter.  The task body is compiled for each row count (multipliers in registers);
// subdomains with more than four rows run in a separate launch of one block per SM (more
// registers).  Each warp keeps its breakpoint keys in its own shared buffer; for even n0 the main
// launch's element loops take two adjacent coefficients per lane with packed FP32 arithmetic.
#include "cv_internal.cuh"

#include <climits>
#include <cstring>
#include <math.h>

namespace {

constexpr int RMAX_CC = 32;  // rows per subdomain handled by complete clipping
constexpr int RTPL = 4;     // row counts up to this run in the main launch (two blocks per SM)
// (target, side) tasks per work item: fewer for subdomains with more rows (longer tasks)
#ifndef CV_CC_NWARP
#define CV_CC_NWARP 12
#endif
constexpr int NWARP = CV_CC_NWARP;  // warps per block at most (two blocks per SM of 12 leave 84 registers a thread)
constexpr int NWARPW = 16;  // warps per block at most in the wide launch (one block per SM, 128 registers a thread)
constexpr int CAPC = 256;   // breakpoints a warp's compacted list holds
constexpr int SAMP_MIN = 64;     // brackets with more breakpoints start from sampled pivots
constexpr float SAMP_D = 0.10f;  // rank margin of the sampled pivots around the target fraction
constexpr int PF = 4;       // coefficients loaded ahead per lane in the element loops

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

// n / d for 0 < n <= d < 2^63 to about 2^-23 relative, without a 64-bit integer conversion (those
// run on the FP64 pipe): both are shifted until d fits in 24 bits and converted from 32 bits.
__device__ __forceinline__ float ratio64(long long n, long long d) {
    const int sh = max(0, 40 - __clzll(d));
    return __fdividef((float)(unsigned)((unsigned long long)n >> sh), (float)(unsigned)((unsigned long long)d >> sh));
}

struct CCArgs {
    int B, U, n0, H, Rmax, Rs, sweeps;
    int tpi[3];  // tasks per work item for subdomains with 1, 2 and more active rows
    // spec-plane mode (cv_spec_clip): the targets are the m spec rows' final planes of each subdomain
    int spec, m;
    const float* sA;      // [B x m x n0] final planes
    const float* sc;      // [B x m] their intercepts
    const float* sscale;  // [B x m] magnitude scale of each plane (error pad)
    float* slower;        // [B x m] spec lower bounds, raised in place
    const int8_t* rowflag;
    const float* lA; const float* lc; const float* uA; const float* uc;
    const int* slot_of; const float* pscale;
    const float* root_lo; const float* root_hi;
    const int* split_off; const int* split_ids;
    const int* row_off; const float* G; const float* h;
    const int* tgt_off; const int* tgt_ids;
    const float* lo; const float* hi;
    float* l; float* u; int8_t* mask; uint8_t* infeasible; int* status;
    unsigned long long* steps;  // optional counters: [0] executed row steps, [1] certified row steps,
                                // [2] of them with several candidates, [3] with a widened window,
                                // [4] left with the FP32 decision, [5] of them over the candidate limit
    const float* amax;    // [2U] max |A| of the cached lower / upper planes (error bounds of the keys)
    const float* samax;   // [B x m] max |A| of the final planes (spec-plane mode)
    // workspace
    float* wg; float* wrg; long long* ww;   // [B][Rs][n0]
    long long* wT; long long* wW;           // [B][Rs] threshold, total weight (fixed point)
    double* wSg; float* wh;                  // [B][Rs]
    float* wGm;                              // [B][Rs] max |g| of every active row
    float* wRm;                              // [B][Rs] max |fl(1/g)| of every active row
    int* wR;                                 // [B] active rows used
    int* wcnt;                               // [B] work items
    int* order;                              // [B] positions -> subdomains, more rows first
    int* ioff;                               // [B+1] first item of every position; [B] = total
    int* toff;                               // [B+1] first task of every position (wide launch)
    int* nplaced;                            // positions holding subdomains with work
    int* wide;                               // items of subdomains with more than RTPL rows (first)
    int* nwpos;                              // positions of subdomains with more than RTPL rows
    unsigned* ticket;                        // [2] tickets: wide-launch tasks, main-launch items
    int allwide;                             // 1: the wide launch takes every item (rows too large to stage)
};

__device__ __forceinline__ int tpi_of(const CCArgs& a, int R) { return a.tpi[R <= 1 ? 0 : (R == 2 ? 1 : 2)]; }

__device__ __forceinline__ int ntargets(const CCArgs& a, int b) {
    return a.tgt_off ? a.tgt_off[b + 1] - a.tgt_off[b] : a.U;
}

// tasks of a subdomain: both sides of every target, or one per spec row in spec-plane mode
__device__ __forceinline__ int ntasks(const CCArgs& a, int b) { return a.spec ? a.m : 2 * ntargets(a, b); }

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
        a.wcnt[b] = r > 0 ? (ntasks(a, b) + tpi_of(a, r) - 1) / tpi_of(a, r) : 0;
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
        float gmx = 0.f, rmx = 0.f;
        for (int j = lane; j < n0; j += 32) {
            const float g = sg * gp[j];
            gmx = fmaxf(gmx, fabsf(g));
            a.wg[base + j] = g;
            const float rg = (g != 0.f) ? 1.f / g : 0.f;
            rmx = fmaxf(rmx, fabsf(rg));
            a.wrg[base + j] = rg;
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
            gmx = fmaxf(gmx, __shfl_xor_sync(0xffffffffu, gmx, off));
            rmx = fmaxf(rmx, __shfl_xor_sync(0xffffffffu, rmx, off));
        }
        // fixed-point weights: scale so that the row total stays below 2^62
        const int sh = (wsum > 0.0) ? 61 - ilogb(wsum) : 0;
        unsigned long long wtot = 0;
        for (int j = lane; j < n0; j += 32) {
            const double w = fabs((double)sg * (double)gp[j]) * (0.5 * ((double)hi[j] - (double)lo[j]));
            const long long wi = __double2ll_rn(ldexp(w, sh));
            a.ww[base + j] = wi;
            wtot += (unsigned long long)wi;
        }
        const long long Wrow = warp_sum64(wtot);
        if (lane == 0) {
            a.wW[(size_t)b * Rs + r] = Wrow;
            const double T = 0.5 * (smax + (double)hh);
            a.wT[(size_t)b * Rs + r] = (T <= 0.0) ? LLONG_MIN : __double2ll_ru(ldexp(T, sh));
            a.wh[(size_t)b * Rs + r] = hh;
            a.wSg[(size_t)b * Rs + r] = sgm;
            a.wGm[(size_t)b * Rs + r] = gmx;
            a.wRm[(size_t)b * Rs + r] = rmx;
        }
    }
}

// Work-item offsets with the subdomains ordered by decreasing row count (longest tasks first).
__global__ void __launch_bounds__(1024) k_cc_scan(CCArgs a) {
    __shared__ int sc[1024], si[1024], sk[1024];
    __shared__ int placed, carry, tcarry;
    const int B = a.B, tid = threadIdx.x, nt = blockDim.x;
    const int per = (B + nt - 1) / nt;
    if (tid == 0) { placed = 0; carry = 0; tcarry = 0; *a.wide = 0; *a.nwpos = 0; }
    __syncthreads();
    for (int v = a.Rs; v >= 1; --v) {
        int c = 0, s = 0, k = 0;
        for (int i = 0; i < per; ++i) {
            const int b = tid * per + i;
            if (b < B && a.wR[b] == v) { ++c; s += a.wcnt[b]; k += ntasks(a, b); }
        }
        sc[tid] = c;
        si[tid] = s;
        sk[tid] = k;
        __syncthreads();
        for (int off = 1; off < nt; off <<= 1) {  // inclusive scans
            const int tc = tid >= off ? sc[tid - off] : 0;
            const int ts = tid >= off ? si[tid - off] : 0;
            const int tk = tid >= off ? sk[tid - off] : 0;
            __syncthreads();
            sc[tid] += tc;
            si[tid] += ts;
            sk[tid] += tk;
            __syncthreads();
        }
        int pos = placed + sc[tid] - c;
        int ib = carry + si[tid] - s;
        int tb = tcarry + sk[tid] - k;
        for (int i = 0; i < per; ++i) {
            const int b = tid * per + i;
            if (b < B && a.wR[b] == v) {
                a.order[pos] = b;
                a.ioff[pos] = ib;
                a.toff[pos] = tb;
                ib += a.wcnt[b];
                tb += ntasks(a, b);
                ++pos;
            }
        }
        __syncthreads();
        if (tid == 0) {
            placed += sc[nt - 1];
            carry += si[nt - 1];
            tcarry += sk[nt - 1];
            if (v == RTPL + 1) { *a.wide = carry; *a.nwpos = placed; }
        }
        __syncthreads();
    }
    for (int i = placed + tid; i < B; i += nt) { a.ioff[i] = carry; a.toff[i] = tcarry; a.order[i] = -1; }
    if (tid == 0) {
        a.ioff[B] = carry;
        a.toff[B] = tcarry;
        *a.nplaced = placed;
        a.ticket[0] = 0u;
        a.ticket[1] = 0u;
    }
}

// Shared memory of k_complete.  The dynamic part holds, in order: the breakpoint keys of every
// warp [nw][n0r], the staged subdomain's rows w64 [Rs][n0] (fixed-point weights), g [Rs][n0],
// fl(1/g) [Rs][n0] (0 where g = 0), and the compacted list elements of every warp [nw][CAPC].
// Every pointer into it is formed from these namespace-scope arrays with 32-bit offsets, so the
// compiler addresses them as shared memory.
extern __shared__ __align__(16) unsigned char cc_smem[];
__shared__ long long cc_T64[RMAX_CC];  // thresholds (fixed point)
__shared__ long long cc_W64[RMAX_CC];  // total weights (fixed point)
__shared__ float cc_hrow[RMAX_CC];     // row constants h
__shared__ double cc_Sg[RMAX_CC];      // magnitude of g against the root box
__shared__ float cc_SgH[RMAX_CC];      // Sg + |h| rounded up
__shared__ float cc_Gm[RMAX_CC];       // max |g| of every row
__shared__ float cc_Rm[RMAX_CC];       // max |fl(1/g)| of every row
// The wide launch's warps take tasks independently: each holds its subdomain's row constants itself.
__shared__ long long cc_wT64[NWARPW][RMAX_CC];
__shared__ long long cc_wW64[NWARPW][RMAX_CC];
__shared__ float cc_whrow[NWARPW][RMAX_CC];
__shared__ float cc_wSgH[NWARPW][RMAX_CC];
__shared__ float cc_wGm[NWARPW][RMAX_CC];
constexpr size_t CC_WCONST = (size_t)NWARPW * RMAX_CC * (8 + 8 + 4 + 4 + 4);  // their bytes
// row p's constants for the calling thread: the block's (main launch) or its warp's (wide launch)
template <bool WIDE> __device__ __forceinline__ long long ccT(int p) {
    if constexpr (WIDE) return cc_wT64[threadIdx.x >> 5][p]; else return cc_T64[p];
}
template <bool WIDE> __device__ __forceinline__ long long ccW(int p) {
    if constexpr (WIDE) return cc_wW64[threadIdx.x >> 5][p]; else return cc_W64[p];
}
template <bool WIDE> __device__ __forceinline__ float cch(int p) {
    if constexpr (WIDE) return cc_whrow[threadIdx.x >> 5][p]; else return cc_hrow[p];
}
template <bool WIDE> __device__ __forceinline__ float ccSgH(int p) {
    if constexpr (WIDE) return cc_wSgH[threadIdx.x >> 5][p]; else return cc_SgH[p];
}
template <bool WIDE> __device__ __forceinline__ float ccGm(int p) {
    if constexpr (WIDE) return cc_wGm[threadIdx.x >> 5][p]; else return cc_Gm[p];
}

struct CCView {
    float* blo;            // the staged subdomain's clipped box [n0] (lower ends)
    float* bhi;            // (upper ends)
    unsigned* keys;        // this warp's keys
    long long* w64;        // staged rows (main launch)
    float* gs;
    float* rg;
    unsigned short* cidx;  // this warp's list elements
    float* bsm;            // this warp's multiplier slots (wide launch): leading parts
    float* blsm;           // trailing parts
    int* jsm;
};

// Main launch: keys [nw][n0r] | w64 [RsS][n0] | g [RsS][n0] | 1/g [RsS][n0] | list [nw][CAPC] |
// multipliers' trailing parts and a copy of their leading parts [nw][2 RMAX_CC] | box [2][n0].
// Wide launch: keys [nw][n0r] | list [nw][CAPC] | multipliers [nw][RMAX_CC] | elements [nw][RMAX_CC] |
// multipliers' trailing parts [nw][RMAX_CC] (its warps read the box from global memory; blo / bhi
// are not used there).
__device__ __forceinline__ CCView cc_view(int n0, int RsS, bool wide) {
    const int n0r = (n0 + 31) & ~31;
    const int nw = blockDim.x >> 5, warp = threadIdx.x >> 5;
    CCView v;
    v.keys = (unsigned*)cc_smem + warp * n0r;
    if (!wide) {
        v.w64 = (long long*)((unsigned*)cc_smem + nw * n0r);
        v.gs = (float*)(v.w64 + RsS * n0);
        v.rg = v.gs + RsS * n0;
        v.cidx = (unsigned short*)(v.rg + RsS * n0) + warp * CAPC;
        v.bsm = nullptr;
        v.blsm = (float*)((unsigned short*)(v.rg + RsS * n0) + nw * CAPC) + warp * 2 * RMAX_CC;
        v.jsm = nullptr;
        v.blo = (float*)((unsigned short*)(v.rg + RsS * n0) + nw * CAPC) + nw * 2 * RMAX_CC;
    } else {
        unsigned short* list0 = (unsigned short*)((unsigned*)cc_smem + nw * n0r);
        v.cidx = list0 + warp * CAPC;
        float* b0 = (float*)(list0 + nw * CAPC);
        v.bsm = b0 + warp * RMAX_CC;
        v.jsm = (int*)(b0 + nw * RMAX_CC) + warp * RMAX_CC;
        v.blsm = (float*)((int*)(b0 + nw * RMAX_CC) + nw * RMAX_CC) + warp * RMAX_CC;
        v.blo = (float*)((int*)(b0 + nw * RMAX_CC) + nw * RMAX_CC) + nw * RMAX_CC;
        v.w64 = nullptr;
        v.gs = nullptr;
        v.rg = nullptr;
    }
    v.bhi = v.blo + n0;
    return v;
}

constexpr unsigned QINF = 0x7f800000u;  // bits of +inf; breakpoints q > 0 have bits in (0, QINF]

// Copies n floats from global src into the warp's shared buffer dst with cp.async, every copy in
// flight at once, and waits for them (16-byte pieces when src is 16-byte aligned and n % 4 == 0;
// dst is 16-byte aligned).  One L2 round trip per plane instead of one per element loop iteration.
__device__ __forceinline__ void cc_plane_to_smem(unsigned* dst, const float* src, int n, int lane) {
    const unsigned sdst = (unsigned)__cvta_generic_to_shared(dst);
    const size_t gsrc = __cvta_generic_to_global(src);
    if ((n & 3) == 0 && (gsrc & 15u) == 0) {
        for (int c = lane; c < (n >> 2); c += 32)
            asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(sdst + 16u * c), "l"(gsrc + 16u * c)
                         : "memory");
    } else {
        for (int c = lane; c < n; c += 32)
            asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(sdst + 4u * c), "l"(gsrc + 4u * c)
                         : "memory");
    }
    asm volatile("cp.async.commit_group;\n" ::: "memory");
    asm volatile("cp.async.wait_group 0;\n" ::: "memory");
    __syncwarp();
}

// Wide launch: a' = sa a + sum over the rows p of msk (increasing p) of beta_p g_p, formed over the
// plane in the warp's buffer buf, two rows per pass over the elements.  Each element gets the same fma
// chain, in the same order, as forming it element by element, so the bits are the same.  The loads
// of a pass do not depend on one another, so one L2 round trip covers PWA elements a lane, instead of
// one per row and element.  Returns the factor still to apply to the buffer: sa when msk is empty,
// else 1.  Lanes write only their own elements; the warp is synchronised on return.
constexpr int PWA = 4;
__device__ __forceinline__ float cc_accum_rows(float* buf, const float* gs, const float* bsm, unsigned msk,
                                               int n0, float sa, int lane) {
    float s0 = sa;
    while (msk) {
        const int p1 = __ffs(msk) - 1;
        msk &= msk - 1u;
        const bool two = msk != 0u;
        const int p2 = two ? __ffs(msk) - 1 : p1;
        if (two) msk &= msk - 1u;
        const float b1 = bsm[p1], b2 = bsm[p2];
        const float* g1 = gs + (size_t)p1 * n0;
        const float* g2 = gs + (size_t)p2 * n0;
#pragma unroll 1
        for (int j0 = lane; j0 < n0; j0 += 32 * PWA) {
            float x[PWA], y1[PWA], y2[PWA];
#pragma unroll
            for (int u = 0; u < PWA; ++u) {
                const int j = j0 + 32 * u;
                const int jj = min(j, n0 - 1);
                x[u] = j < n0 ? buf[j] : 0.f;
                y1[u] = __ldg(g1 + jj);
                y2[u] = __ldg(g2 + jj);
            }
#pragma unroll
            for (int u = 0; u < PWA; ++u) {
                const int j = j0 + 32 * u;
                float v = fmaf(b1, y1[u], s0 * x[u]);
                const float v2 = fmaf(b2, y2[u], v);
                v = two ? v2 : v;
                if (j < n0) buf[j] = v;
            }
        }
        s0 = 1.f;
    }
    __syncwarp();
    return s0;
}

// Rows of the task's subdomain: staged in shared memory (main launch) or read from the
// workspace (subdomains with more rows than the main launch stages).
struct CCRows {
    const float* gs;
    const float* rg;
    const long long* w64;
};

// Outcome of a certified row step (see cc_certify): the multiplier as beta_hi + beta_lo, its element,
// and counters (certified, several candidates, widened window, FP32 decision kept, of which over the
// candidate limit).
struct CertState {
    float bn, bln;
    int jn;
    unsigned cs[5];
};

// Certified decision of one row step of Algorithm 1 with R >= 2 rows (row k).  The FP32 search decided
// the crossing q* (element jn; dec = 1) or beta = 0 from F(0) >= T (dec = 0) on keys
// q_j = fl(-a'_j * fl(1/g_kj)), a' formed by an FP32 fma chain from the leading parts bh of the
// multipliers.  Each key lies within
//   E_j = 2u'|q_j| + (n + 1) u' S_j |fl(1/g_kj)|,  S_j = |a_j| + sum_{p != k} |bh_p g_pj|,  u' = 2^-24 * 1.001,
// of the exact breakpoint -(a_j + sum_{p != k} beta_p g_pj) / g_kj with the full multipliers bh + bl:
// n = the number of nonzero multipliers p != k (one fma rounding each), one more u' S_j for all the
// dropped trailing parts, two roundings in the product (with every other multiplier 0, a' = a exactly).
// The window [L, H] = [q* - E*, q* + E*] (the point 0 for dec = 0) is where the exact crossing can lie.
// A screening pass over the keys (S_j bounded by max|a| + sum_p |bh_p| max|g_p|, 1% margin) marks the
// elements whose interval might meet the window; each is then tested with its own S_j.  Candidates
// (interval meets the window) have their breakpoints recomputed in float-float arithmetic (error a few
// 2^-48 of S_j |1/g_kj|, inside the 0.1% margin of u'); exact zeros (S_j = 0) form one group at 0.  The
// elements surely below the window weigh F(< q*) (F(<= 0)) minus the candidates the FP32 keys put there.
// Walking the candidates in exact order (equal values by element) after that weight, the first to reach
// the threshold T is the exact crossing provided its breakpoint lies in the window: every element
// outside the window is then ordered against it.  Otherwise the window grows to it and a full pass
// repeats the selection (at most twice).  A crossing at or below 0 with 0 in the window is beta = 0.
// Left unsettled (more than CAPC candidates or the window still moving), the FP32 decision stands: still
// a valid multiplier.  The result is the decision of the sorted-breakpoint rule on exact breakpoints
// except between breakpoints equal to within about 2^-44 of their magnitude.
// Memory: keys (the warp's key buffer, every element's key), cidx (the warp's list buffer, free here),
// gs / rk / wk the staged rows, bh / bl the multipliers' leading and trailing parts (shared slots).
// Once more than 64 candidates' breakpoints are written over the key buffer, keys are recomputed from
// the target plane.
template <bool WIDE>
__device__ __forceinline__ void cc_certify(int n0, int R, int k, int lane, const float* gs, const float* rk,
                                        const long long* wk, unsigned* keys, unsigned short* cidx, const float* ap,
                                        float sa, const float* bh, const float* bl, float amx, long long T,
                                        long long Fdec, int dec, CertState* st) {
    const float cu1 = 5.9665e-08f;  // >= 2^-24 * 1.001
    const float tu = 1.1933e-07f;   // >= 2 * 2^-24 * 1.001
    float smx = amx;
    int nnz = 0;
    // rows p != k whose terms are formed: in the wide launch those with a nonzero multiplier (the
    // others add exactly nothing), in the main launch all of them
    unsigned nzm = 0u;
    for (int p = 0; p < R; ++p) {
        if (p == k) continue;
        const float b = bh[p];
        smx = __fmaf_ru(fabsf(b), ccGm<WIDE>(p), smx);
        nnz += b != 0.f;
        if (!WIDE || b != 0.f) nzm |= 1u << p;
    }
    const float Ru = nnz ? __fmul_ru((float)(nnz + 1), cu1) : 0.f;
    const float c1 = __fmul_ru(Ru, smx);
    const int jn0 = st->jn;
    const float qs = dec == 1 ? st->bn : 0.f;
    const float Es = dec == 1 ? __fmaf_ru(c1, fabsf(rk[jn0]), __fmul_ru(tu, qs)) : 0.f;
    float Lw = __fsub_rd(qs, Es), Hw = __fadd_ru(qs, Es);
    st->cs[0] = 1u; st->cs[1] = 0u; st->cs[2] = 0u; st->cs[3] = 0u; st->cs[4] = 0u;
    // the FP32 key of element j exactly as the key pass forms it
    auto key_calc = [&](int j) -> float {
        float x = sa * __ldg(ap + j);
        if constexpr (WIDE) {
            for (unsigned mm = nzm; mm; mm &= mm - 1u) {
                const int p = __ffs(mm) - 1;
                x = fmaf(bh[p], gs[p * n0 + j], x);
            }
        } else {
            for (int p = 0; p < R; ++p)
                if (p != k) x = fmaf(bh[p], gs[p * n0 + j], x);
        }
        return (-x) * rk[j];
    };
    bool keys_ok = true;  // the key buffer holds every element's key
    // With E' = c1 |1/g_kj| + tu |q_j| (every operation rounded up) >= E_j, an element whose interval
    // with E' lies wholly below the window is below it (class 1) and one wholly above is outside it
    // (class 0), exactly as classify finds with its own E_j <= E'; -1: the element needs its own test.
    // (g_kj = 0 gives weight 0: either class leaves the sums unchanged.)
    auto preclass = [&](int j, float q) -> int {
        const float Ep = __fmaf_ru(c1, fabsf(rk[j]), __fmul_ru(tu, fabsf(q)));
        if (__fadd_ru(q, Ep) < Lw) return 1;
        if (__fsub_rd(q, Ep) > Hw) return 0;
        return -1;
    };
    // the element's own interval against the window: 1 below, 2 candidate, 3 exact zero inside, 0 else
    auto classify = [&](int j, float q, float av) -> int {
        const float r = rk[j];
        if (r == 0.f) return 0;  // g_kj = 0: no breakpoint (weight 0)
        float S = fabsf(av);
        if constexpr (WIDE) {
            for (unsigned mm = nzm; mm; mm &= mm - 1u) {
                const int p = __ffs(mm) - 1;
                S = __fmaf_ru(fabsf(bh[p]), fabsf(gs[p * n0 + j]), S);
            }
        } else {
            for (int p = 0; p < R; ++p)
                if (p != k) S = __fmaf_ru(fabsf(bh[p]), fabsf(gs[p * n0 + j]), S);
        }
        if (S == 0.f) return 0.f < Lw ? 1 : (0.f <= Hw ? 3 : 0);
        const float E = __fmaf_ru(__fmul_ru(Ru, S), fabsf(r), __fmul_ru(tu, fabsf(q)));
        if (__fadd_ru(q, E) < Lw) return 1;
        return __fsub_rd(q, E) <= Hw ? 2 : 0;
    };
    // breakpoint of element j in float-float: -(sh + sl) / g_kj with sh + sl = a'_j.  The quotient is
    // refined once: qh from fl(1/g), the remainder qh g + sh by fma, the correction from it.
    auto ff_key = [&](int j, float av, float& kh, float& kl) {
        float sh = sa * av, sl = 0.f;
        auto term = [&](int p) {
            const float b1 = bh[p], b2 = bl[p], g = gs[p * n0 + j];
            const float pr = __fmul_rn(b1, g);
            float pe = __fmaf_rn(b1, g, -pr);  // exact error of the product
            pe = __fmaf_rn(b2, g, pe);
            const float t = __fadd_rn(sh, pr);
            const float bb = __fsub_rn(t, sh);
            const float er = __fadd_rn(__fsub_rn(sh, __fsub_rn(t, bb)), __fsub_rn(pr, bb));
            sh = t;
            sl = __fadd_rn(sl, __fadd_rn(er, pe));
        };
        if constexpr (WIDE) {  // (a zero leading part has a zero trailing part: those rows add nothing)
            for (unsigned mm = nzm; mm; mm &= mm - 1u) term(__ffs(mm) - 1);
        } else {
            for (int p = 0; p < R; ++p)
                if (p != k) term(p);
        }
        const float t = __fadd_rn(sh, sl);
        sl = __fsub_rn(sl, __fsub_rn(t, sh));
        sh = t;
        const float gk = gs[k * n0 + j], r = rk[j];
        const float qh = __fmul_rn(-sh, r);
        const float rem = __fmaf_rn(qh, gk, sh);  // qh g + sh
        const float ql = __fmul_rn(-__fadd_rn(rem, sl), r);
        kh = __fadd_rn(qh, ql);
        kl = __fsub_rn(ql, __fsub_rn(kh, qh));
    };
    // the crossing element's coefficient, loaded early (it is almost always the one candidate)
    const float a_jn = dec == 1 ? __ldg(ap + jn0) : 0.f;
    // screening bound (1% above the first test)
    const float sc1 = c1 * 1.01f, stu = tu * 1.01f, sEs = Es * 1.01f;
    const unsigned below_lanes = (1u << lane) - 1u;
    bool ok = false;
    float rh = 0.f, rl = 0.f;
    int rj = -1;
#pragma unroll 1
    for (int it = 0; it < 3 && !ok; ++it) {
        // 1. Classify the elements against the window.  it = 0: a screen over the keys marks the
        // elements to test (bits of a per-lane mask, 32 iterations at a time); each is tested with its
        // own bound, and the weight surely below is F(< q*) minus the candidates and zeros counted there.
        // Later passes (a widened window) test every element and sum the surely-below weight directly.
        // Candidates stay in registers, two per lane; a lane with more sends the pass to `spill`, which
        // repeats it listing every candidate in cidx.
        unsigned long long fb = 0ull, fz = 0ull;
        int c0 = -1, c1e = -1, nc = 0;
        float a0 = 0.f, a1 = 0.f;
        bool spill = false;
        int nloc = 0;
        // the element's class with the bookkeeping of this pass
        auto take = [&](int jj, float q, float av) -> int {
            const int cls = classify(jj, q, av);
            if (it == 0) {
                const bool counted = dec == 1 ? q < qs : q <= 0.f;
                if ((cls == 2 || cls == 3) && counted) fb += (unsigned long long)wk[jj];
            } else if (cls == 1) {
                fb += (unsigned long long)wk[jj];
            }
            if (cls == 3) fz += (unsigned long long)wk[jj];
            if (cls == 2) {
                if (nloc == 0) { c0 = jj; a0 = av; }
                else if (nloc == 1) { c1e = jj; a1 = av; }
                ++nloc;
            }
            return cls;
        };
        if (it == 0) {
            // With E_j <= c1 |1/g_kj| + tu |q_j| (c1 bounds Ru S_j for every j), an element can meet the
            // window only if |q_j - q*| <= c1 |1/g_kj| + tu |q_j| + E*: the screen tests that (1% above,
            // for its own roundings) with each element's own |1/g_kj|, 32 elements a lane at a time.
#pragma unroll 1
            for (int cb = 0; cb < n0; cb += 1024) {
                unsigned msk = 0u;  // bit i: element cb + 32 i + lane
                constexpr int SCRU = WIDE ? 8 : 2;  // (the wide launch reads 1/g from L2)
#pragma unroll SCRU
                for (int i = 0; i < 32; ++i) {
                    const int j = cb + 32 * i + lane;
                    const int jj = j < n0 ? j : n0 - 1;
                    const float q = __uint_as_float(keys[jj]);
                    const bool scr = fabsf(q - qs) <= fmaf(sc1, fabsf(rk[jj]), fmaf(stu, fabsf(q), sEs));
                    msk |= (unsigned)(j < n0 && scr) << i;
                }
                while (msk) {
                    const int i = __ffs(msk) - 1;
                    msk &= msk - 1u;
                    const int j = cb + 32 * i + lane;
                    take(j, __uint_as_float(keys[j]), j == jn0 ? a_jn : __ldg(ap + j));
                }
            }
        } else {
            // a widened window: every element, most of them settled by the global bound
#pragma unroll 1
            for (int j0 = 0; j0 < n0; j0 += 32) {
                const int j = j0 + lane;
                if (j >= n0) continue;
                const float q = keys_ok ? __uint_as_float(keys[j]) : key_calc(j);
                const int pc = preclass(j, q);
                if (pc == 1) fb += (unsigned long long)wk[j];
                else if (pc < 0) take(j, q, __ldg(ap + j));
            }
        }
        nc = __reduce_add_sync(0xffffffffu, (unsigned)nloc);
        spill = __any_sync(0xffffffffu, nloc > 2);
        if (spill) {
            // every candidate listed in cidx (a slow pass, for rows with many near-ties)
            fb = 0ull; fz = 0ull; c0 = -1; c1e = -1; nloc = 0;
            int ncl = 0;
#pragma unroll 1
            for (int j0 = 0; j0 < n0; j0 += 32) {
                const int j = j0 + lane;
                const bool v = j < n0;
                const int jj = v ? j : n0 - 1;
                const float q = keys_ok ? __uint_as_float(keys[jj]) : key_calc(jj);
                bool look = v;
                int pc = -1;
                if (it == 0) look = v && fabsf(q - qs) <= fmaf(sc1, fabsf(rk[jj]), fmaf(stu, fabsf(q), sEs));
                else if (v) pc = preclass(jj, q);
                if (pc == 1) fb += (unsigned long long)wk[jj];
                const int cls = (look && pc < 0) ? take(jj, q, __ldg(ap + jj)) : (pc == 1 ? 1 : 0);
                const unsigned bal = __ballot_sync(0xffffffffu, cls == 2);
                const int pos = ncl + __popc(bal & below_lanes);
                if (cls == 2 && pos < CAPC) cidx[pos] = (unsigned short)jj;
                ncl += __popc(bal);
            }
            nc = ncl;
        }
        __syncwarp();
        long long Fz = 0, Fb = 0;
        bool found = false;
        if (__any_sync(0xffffffffu, fz != 0ull)) Fz = warp_sum64(fz);
        if (__any_sync(0xffffffffu, fb != 0ull)) Fb = warp_sum64(fb);
        if (it == 0) Fb = Fdec - Fb;
        if (nc > 1) st->cs[1] = 1u;
        if (spill && (nc > CAPC || (nc > 64 && 2 * nc > ((n0 + 31) & ~31)))) {
            // Too many candidates to list: the crossing is found by bisection on the exact order
            // (breakpoint's leading part, trailing part, element) without storing them, each step a pass
            // that sums the weight of the candidates at or below a point (slow; rows with many near-ties).
            st->cs[4] = 1u;
            const bool it0 = it == 0;
            auto ordf = [](float f) -> unsigned {
                const unsigned u = __float_as_uint(f);
                return (u & 0x80000000u) ? ~u : (u | 0x80000000u);
            };
            auto unord = [](unsigned o) -> float { return __uint_as_float((o & 0x80000000u) ? (o & 0x7fffffffu) : ~o); };
            // weight of the elements at or below (X1, X2, X3) in the exact order, plus Fb
            auto count_le = [&](unsigned X1, unsigned X2, int X3) -> long long {
                unsigned long long f = 0ull;
                for (int j0 = 0; j0 < n0; j0 += 32) {
                    const int j = j0 + lane;
                    if (j >= n0) continue;
                    const float q = keys_ok ? __uint_as_float(keys[j]) : key_calc(j);
                    if (it0 && !(fabsf(q - qs) <= fmaf(sc1, fabsf(rk[j]), fmaf(stu, fabsf(q), sEs)))) continue;
                    if (!it0 && preclass(j, q) >= 0) continue;  // settled by the global bound: not a candidate
                    const float av = __ldg(ap + j);
                    if (classify(j, q, av) != 2) continue;
                    float kh, kl;
                    ff_key(j, av, kh, kl);
                    const unsigned o1 = ordf(kh), o2 = ordf(kl);
                    if (o1 < X1 || (o1 == X1 && (o2 < X2 || (o2 == X2 && j <= X3)))) f += (unsigned long long)wk[j];
                }
                long long F2 = Fb + warp_sum64(f);
                // the exact zeros: the point (0, 0, -1)
                const unsigned z = ordf(0.f);
                if (z < X1 || (z == X1 && (z < X2 || (z == X2 && -1 <= X3)))) F2 += Fz;
                return F2;
            };
            if (Fb >= T) {
                found = true;
                rh = -INFINITY; rl = 0.f; rj = -1;
            } else {
                // The same bisections, with each count taken from stored ordinals.  One pass computes
                // every candidate's exact breakpoint once and keeps the ordinal of its leading part over
                // the key buffer (NONC, above every pivot, for the other elements), so the first bisection
                // reads ordinals; the candidates tied at its result then get their trailing parts in the
                // list buffer for the other two.  Every count equals count_le's at the same point.
                constexpr unsigned NONC = 0xffffffffu;  // no finite breakpoint has this ordinal
                const unsigned z = ordf(0.f);           // the exact zeros' point (0, 0, -1)
#pragma unroll 1
                for (int j0 = 0; j0 < n0; j0 += 32) {
                    const int j = j0 + lane;
                    if (j >= n0) continue;
                    const float q = keys_ok ? __uint_as_float(keys[j]) : key_calc(j);
                    bool cand;
                    if (it0) cand = fabsf(q - qs) <= fmaf(sc1, fabsf(rk[j]), fmaf(stu, fabsf(q), sEs));
                    else cand = preclass(j, q) < 0;
                    unsigned o = NONC;
                    if (cand) {
                        const float av = __ldg(ap + j);
                        if (classify(j, q, av) == 2) {
                            float kh, kl;
                            ff_key(j, av, kh, kl);
                            o = ordf(kh);
                        }
                    }
                    keys[j] = o;  // (each lane rewrites only the elements it read)
                }
                keys_ok = false;
                __syncwarp();
                // weight of the candidates whose leading ordinal is at or below X1 (the count at
                // (X1, max, max)), plus Fb and the zeros
                auto count1 = [&](unsigned X1) -> long long {
                    unsigned long long f = 0ull;
#pragma unroll 1
                    for (int j0 = 0; j0 < n0; j0 += 32 * 4) {
                        unsigned kq[4];
                        unsigned long long wq[4];
#pragma unroll
                        for (int u = 0; u < 4; ++u) {
                            const int j = min(j0 + 32 * u + lane, n0 - 1);
                            kq[u] = keys[j];
                            wq[u] = (unsigned long long)wk[j];
                        }
#pragma unroll
                        for (int u = 0; u < 4; ++u)
                            if (j0 + 32 * u + lane < n0 && kq[u] <= X1) f += wq[u];
                    }
                    long long F2 = Fb + warp_sum64(f);
                    if (z <= X1) F2 += Fz;
                    return F2;
                };
                // invariants F(<= low end) < T <= F(<= high end); ordinal 0 lies below every key
                unsigned l1 = 0u, h1 = 0xffffffffu;
                while (h1 - l1 > 1u) {
                    const unsigned m1 = l1 + ((h1 - l1) >> 1);
                    if (count1(m1) >= T) h1 = m1; else l1 = m1;
                }
                // the candidates tied at h1: listed (at most CAPC), their trailing ordinals over their key
                // slots; the weight strictly below h1 summed on the way
                unsigned long long fl = 0ull;
                int ntie = 0;
#pragma unroll 1
                for (int j0 = 0; j0 < n0; j0 += 32) {
                    const int j = j0 + lane;
                    const bool v = j < n0;
                    const unsigned o = v ? keys[j] : NONC;
                    if (v && o < h1) fl += (unsigned long long)wk[j];
                    const bool tie = v && o == h1 && o != NONC;
                    const unsigned bal = __ballot_sync(0xffffffffu, tie);
                    const int pos = ntie + __popc(bal & below_lanes);
                    if (tie && pos < CAPC) cidx[pos] = (unsigned short)j;
                    ntie += __popc(bal);
                }
                __syncwarp();
                const long long Flow = Fb + warp_sum64(fl);
                unsigned l2 = 0u, h2 = 0xffffffffu;
                int l3 = -2, h3 = n0;
                if (ntie <= CAPC) {
                    for (int t = lane; t < ntie; t += 32) {
                        const int j = cidx[t];
                        float kh, kl;
                        ff_key(j, __ldg(ap + j), kh, kl);
                        keys[j] = ordf(kl);
                    }
                    __syncwarp();
                    // weight at or below (h1, X2, X3) from the list
                    auto count23 = [&](unsigned X2, int X3) -> long long {
                        unsigned long long f = 0ull;
                        for (int t = lane; t < ntie; t += 32) {
                            const int j = cidx[t];
                            const unsigned o2 = keys[j];
                            if (o2 < X2 || (o2 == X2 && j <= X3)) f += (unsigned long long)wk[j];
                        }
                        long long F2 = Flow + warp_sum64(f);
                        if (z < h1 || (z == h1 && (z < X2 || (z == X2 && -1 <= X3)))) F2 += Fz;
                        return F2;
                    };
                    while (h2 - l2 > 1u) {
                        const unsigned m2 = l2 + ((h2 - l2) >> 1);
                        if (count23(m2, INT_MAX) >= T) h2 = m2; else l2 = m2;
                    }
                    while (h3 - l3 > 1) {
                        const int m3 = l3 + ((h3 - l3) >> 1);
                        if (count23(h2, m3) >= T) h3 = m3; else l3 = m3;
                    }
                } else {
                    // more ties than the list holds: the counts recomputed from the rows
                    while (h2 - l2 > 1u) {
                        const unsigned m2 = l2 + ((h2 - l2) >> 1);
                        if (count_le(h1, m2, INT_MAX) >= T) h2 = m2; else l2 = m2;
                    }
                    while (h3 - l3 > 1) {
                        const int m3 = l3 + ((h3 - l3) >> 1);
                        if (count_le(h1, h2, m3) >= T) h3 = m3; else l3 = m3;
                    }
                }
                found = true;
                rh = unord(h1); rl = unord(h2); rj = h3;
            }
        }
        if (!found) {
        // 2. the candidates' breakpoints: per lane two in registers (slots 0, 1); in spill mode the first
        // 64 listed go to registers (lane t % 32, slot t / 32) and the rest over the key buffer
        // (keys[2t], keys[2t + 1]), after which keys are recomputed
        float ch0 = 0.f, cl0 = 0.f, ch1 = 0.f, cl1 = 0.f;
        int cj0 = c0, cj1 = c1e;
        if (spill) {
            cj0 = lane < nc ? (int)cidx[lane] : -1;
            cj1 = lane + 32 < nc ? (int)cidx[lane + 32] : -1;
            a0 = cj0 >= 0 ? __ldg(ap + cj0) : 0.f;
            a1 = cj1 >= 0 ? __ldg(ap + cj1) : 0.f;
        }
        if (cj0 >= 0) ff_key(cj0, a0, ch0, cl0);
        if (cj1 >= 0) ff_key(cj1, a1, ch1, cl1);
        if (spill && nc > 64) {
            __syncwarp();
            for (int t = lane + 64; t < nc; t += 32) {
                float h2, l2;
                const int j = cidx[t];
                ff_key(j, __ldg(ap + j), h2, l2);
                keys[2 * t] = __float_as_uint(h2);
                keys[2 * t + 1] = __float_as_uint(l2);
            }
            keys_ok = false;
            __syncwarp();
        }
        // 3. walk the candidates in exact order after Fb; the exact zeros form one group at 0
        long long F = Fb;
        if (F >= T) {
            found = true;  // the crossing lies below the window
            rh = -INFINITY; rl = 0.f; rj = -1;
        } else if (nc == 1 && Fz == 0) {
            // one candidate: no ordering to do
            const unsigned bal = __ballot_sync(0xffffffffu, cj0 >= 0);
            const int src = __ffs(bal) - 1;
            const float kh = __shfl_sync(0xffffffffu, ch0, src), kl = __shfl_sync(0xffffffffu, cl0, src);
            const int kj = __shfl_sync(0xffffffffu, cj0, src);
            F += wk[kj];
            if (F >= T) { found = true; rh = kh; rl = kl; rj = kj; }
        } else if (nc > 0 || Fz != 0) {
            unsigned taken = 0u;  // bit u: this lane's slot u (u >= 2: listed candidate lane + 32 u)
            bool tz = (Fz == 0);
#pragma unroll 1
            for (int s2 = 0; s2 <= nc && !found; ++s2) {
                float kh = INFINITY, kl = 0.f;
                int kj = INT_MAX, ku = -1;
                auto better = [&](float h2, float l2, int j2) {
                    return h2 < kh || (h2 == kh && (l2 < kl || (l2 == kl && j2 < kj)));
                };
                if (cj0 >= 0 && !(taken & 1u) && better(ch0, cl0, cj0)) { kh = ch0; kl = cl0; kj = cj0; ku = 0; }
                if (cj1 >= 0 && !(taken & 2u) && better(ch1, cl1, cj1)) { kh = ch1; kl = cl1; kj = cj1; ku = 1; }
                if (spill)
                    for (int u = 2, t = lane + 64; t < nc; ++u, t += 32) {
                        if ((taken >> u) & 1u) continue;
                        const float h2 = __uint_as_float(keys[2 * t]), l2 = __uint_as_float(keys[2 * t + 1]);
                        const int j2 = cidx[t];
                        if (better(h2, l2, j2)) { kh = h2; kl = l2; kj = j2; ku = u; }
                    }
                if (!tz && lane == 0 && better(0.f, 0.f, -1)) { kh = 0.f; kl = 0.f; kj = -1; ku = 31; }
                // element and lane in one word (elements < 65536)
                int tag = ((kj == INT_MAX ? 0xffff : (kj & 0xffff)) << 5) | lane;
#pragma unroll
                for (int off = 16; off > 0; off >>= 1) {
                    const float h2 = __shfl_xor_sync(0xffffffffu, kh, off);
                    const float l2 = __shfl_xor_sync(0xffffffffu, kl, off);
                    const int t2 = __shfl_xor_sync(0xffffffffu, tag, off);
                    if (h2 < kh || (h2 == kh && (l2 < kl || (l2 == kl && t2 < tag)))) { kh = h2; kl = l2; tag = t2; }
                }
                if (kh == INFINITY) break;  // none left
                const int src = tag & 31;
                kj = (tag >> 5) == 0xffff ? -1 : (tag >> 5);
                const int slot = __shfl_sync(0xffffffffu, ku, src);
                if (lane == src) {
                    if (slot == 31) tz = true;
                    else taken |= 1u << slot;
                }
                F += (slot == 31) ? Fz : wk[kj];
                if (F >= T) { found = true; rh = kh; rl = kl; rj = kj; }
            }
        }
        }
        if (!found) {
            // the crossing lies above the window
            st->cs[2] = 1u;
            Hw = INFINITY;
            continue;
        }
        // settled when the crossing's breakpoint lies in the window, or at or below 0 with 0 inside it
        const bool le0 = rh < 0.f || (rh == 0.f && rl <= 0.f);
        const bool inside = (rh > Lw || (rh == Lw && rl >= 0.f)) && (rh < Hw || (rh == Hw && rl <= 0.f));
        if (inside || (le0 && Lw <= 0.f && 0.f <= Hw)) {
            ok = true;
            break;
        }
        st->cs[2] = 1u;
        if (rh == -INFINITY) Lw = -INFINITY;
        else {
            Lw = fminf(Lw, nextafterf(rh, -INFINITY));  // |trailing part| <= half an ulp of the leading one
            Hw = fmaxf(Hw, nextafterf(rh, INFINITY));
        }
    }
    if (!ok) {
        st->cs[3] = 1u;  // the FP32 decision stands
        return;
    }
    if (rh < 0.f || (rh == 0.f && rl <= 0.f)) {
        st->bn = 0.f; st->bln = 0.f; st->jn = -1;
    } else {
        st->bn = rh; st->bln = rl; st->jn = rj;
    }
}

// One (target, side) task of complete clipping with Rn active rows.  RC is a compile-time bound on
// Rn: the main launch instantiates RC = Rn = 1..4 with the multipliers in registers; the wide
// launch instantiates RC = 8, 16, 32 for any Rn <= RC with the multipliers in the warp's shared
// slots bsm / jsm.  Breakpoint keys are the raw bits of q_j = (-a'_j) * fl(1/g_kj): for q > 0 (the
// search range) the unsigned order of the bits is the order of the values.
template <int RC, bool WIDE, bool SPEC>
__device__ __forceinline__ void cc_task(const CCArgs& a, const CCRows& rw, unsigned* keys, unsigned short* cidx,
                                        float* bsm, float* blsm, int* jsm, const float* blo, const float* bhi, int Rn,
                                        int b, int c, int side, int lane, unsigned long long& my_steps,
                                        unsigned (&my_cs)[5]) {
    // with two or more rows the FP32 decisions are certified (see cc_certify below)
    constexpr bool CERT = WIDE || RC >= 2;
    // elements a lane loads ahead in the scalar key pass (the wide launch reads its rows from L2)
    constexpr int PFK = WIDE ? 8 : PF;
    // and in the search passes over keys and weights
    constexpr int PFS = WIDE ? 4 : 1;
    const int n0 = a.n0;
    const int R = WIDE ? Rn : RC;
    // the target plane a.x + c0 (lower side; the upper side is the negated upper plane), or in
    // spec-plane mode spec row c's final plane
    const size_t o = SPEC ? (size_t)b * a.m + c : (size_t)b * a.U + c;
    const float* ap = SPEC ? a.sA + o * n0 : (side ? a.uA + (size_t)c * n0 : a.lA + (size_t)c * n0);
    const float sa = (!SPEC && side) ? -1.f : 1.f;
    const float c0 = SPEC ? a.sc[o] : (side ? -a.uc[c] : a.lc[c]);
    // multipliers as unevaluated sums beta_hi + beta_lo of two floats (the trailing part stays 0
    // with one row); keys and the dual value use the leading parts
    float beta[WIDE ? 1 : RC] = {};
    int jprev[WIDE ? 1 : RC];
    auto bget = [&](int p) -> float {
        if constexpr (WIDE) return bsm[p]; else return beta[p];
    };
    // trailing parts in the warp's shared slots (read only by the certification)
#pragma unroll
    for (int p = 0; p < RC; ++p) {
        if (WIDE && p >= R) break;
        if constexpr (WIDE) { bsm[p] = 0.f; jsm[p] = -1; } else { beta[p] = 0.f; jprev[p] = -1; }
        if (CERT) blsm[p] = 0.f;
    }
    // With one row, a' = a in every sweep, so one pass already repeats bit for bit.  More
    // generally a row step depends only on the other rows' multipliers: a row whose inputs have
    // not changed since its last step would repeat it exactly and is skipped (bit `k` of `dirty`
    // marks row k as having changed inputs), which leaves every multiplier as the full sweep
    // order gives it.
    const int nsweeps = (R == 1) ? 1 : a.sweeps;
    const unsigned all_rows = (R >= 32) ? 0xffffffffu : ((1u << R) - 1u);
    unsigned dirty = all_rows;
    for (int sw = 0; sw < nsweeps && dirty; ++sw) {
        bool changed = false;
#pragma unroll 1
        for (int k = 0; k < R; ++k) {
            if (!((dirty >> k) & 1u)) continue;
            dirty &= ~(1u << k);
            ++my_steps;
            const float* rk = rw.rg + k * n0;
            const long long* wk = rw.w64 + k * n0;
            float bk = 0.f, blk = 0.f;
            int jp = -1;
            if constexpr (WIDE) {
                bk = bsm[k]; jp = jsm[k];
            } else {
#pragma unroll
                for (int p = 0; p < RC; ++p)
                    if (p == k) { bk = beta[p]; jp = jprev[p]; }
            }
            if (CERT) blk = blsm[k];
            // q_j from a' = a + sum_{p != k} beta_p g_p (fma chain in increasing p).  The wide launch
            // skips the rows whose multiplier is 0: fma(0, g, x) = x (up to the sign of a zero, which
            // is never a breakpoint), so the keys are the same and only the nonzero rows are read.
            unsigned nzm = 0u;
            if constexpr (WIDE) {
                for (int p = 0; p < R; ++p)
                    if (p != k && bsm[p] != 0.f) nzm |= 1u << p;
            }
            auto q_of = [&](float av, int j) -> float {
                float apr = sa * av;
                if constexpr (WIDE) {
                    for (unsigned mm = nzm; mm; mm &= mm - 1u) {
                        const int p = __ffs(mm) - 1;
                        apr = fmaf(bsm[p], rw.gs[p * n0 + j], apr);
                    }
                } else {
#pragma unroll
                    for (int p = 0; p < RC; ++p) {
                        if (RC > 1) {
                            const float t = fmaf(bget(p), rw.gs[p * n0 + j], apr);
                            apr = (p != k) ? t : apr;
                        }
                    }
                }
                return (-apr) * rk[j];
            };
            // the target plane into the warp's key buffer; the key pass overwrites it with the keys
            cc_plane_to_smem(keys, ap, n0, lane);
            // previous breakpoint of this row (same value for every lane)
            float qp = 0.f;
            if (jp >= 0) {
                if constexpr (WIDE) {
                    // q_of at one element with the rows' coefficients loaded by one lane each (all in
                    // flight at once) and passed along the fma chain by shuffles: the same bits
                    const float gl = lane < R ? __ldg(rw.gs + (size_t)lane * n0 + jp) : 0.f;
                    float apr = sa * __uint_as_float(keys[jp]);
                    for (unsigned mm = nzm; mm; mm &= mm - 1u) {
                        const int p = __ffs(mm) - 1;
                        apr = fmaf(bsm[p], __shfl_sync(0xffffffffu, gl, p), apr);
                    }
                    qp = (-apr) * rk[jp];
                } else {
                    qp = q_of(__uint_as_float(keys[jp]), jp);
                }
            }
            __syncwarp();
            // wide launch: a' formed over the plane in the buffer first (the same bits as q_of forms),
            // so that the key pass below only scales it
            float skey = sa;
            if constexpr (WIDE) skey = cc_accum_rows((float*)keys, rw.gs, bsm, nzm, n0, sa, lane);
            auto qk_of = [&](float av, int j) -> float {
                if constexpr (WIDE) return (-(skey * av)) * rk[j];
                else return q_of(av, j);
            };
            const bool warm = qp > 0.f;
            const long long T = ccT<WIDE>(k);
            const long long W = ccW<WIDE>(k);
            // One pass over all n0 elements keeps the keys in the warp's buffer.  Without a previous
            // breakpoint it takes F(0) = sum_{q <= 0} w (the paired pass: W minus the weight of q > 0,
            // leaving the extent and size of the search range to the search); with one, F just below
            // and at it.  F(+inf) is the row's total weight W.  (Branch-free element loops: indices
            // past n0 are clamped and contribute nothing.)
            unsigned long long f0 = 0, flt = 0, fle = 0;
            unsigned mn = 0xffffffffu, mx = 0u, cnt = 0u;
            // extents (mn, mx, cnt) of the positive keys: the paired pass leaves them to the search
            bool ext = true;
            if (!WIDE && (n0 & 1) == 0) {
                // Two adjacent elements per lane with packed FP32 arithmetic.  x = -a' is built as
                // (-sa) a + sum_p (-beta_p) g_p with row k's own multiplier zeroed: negation is exact
                // and commutes with round-to-nearest, so q = x * fl(1/g) has the bits of (-a') * fl(1/g)
                // (up to the sign of a zero, and zero is never a breakpoint).
                float nb[WIDE ? 1 : RC];
#pragma unroll
                for (int p = 0; p < (WIDE ? 1 : RC); ++p) nb[p] = (p == k) ? 0.f : -bget(p);
                const float2 nsa2 = make_float2(-sa, -sa);
                auto q2_of = [&](float2 av, int j) -> float2 {
                    float2 x = __fmul2_rn(av, nsa2);
#pragma unroll
                    for (int p = 0; p < (WIDE ? 1 : RC); ++p)
                        if (RC > 1) x = __ffma2_rn(make_float2(nb[p], nb[p]), *(const float2*)(rw.gs + p * n0 + j), x);
                    return __fmul2_rn(x, *(const float2*)(rk + j));
                };
                const float2* ap2 = (const float2*)keys;  // the plane, overwritten pair by pair
                constexpr int P2 = 1;  // pairs per lane per iteration
                if (warm) {
#pragma unroll 1
                    for (int j0 = 2 * lane; j0 < n0; j0 += 64 * P2) {
                        float2 av[P2];
                        av[0] = ap2[min(j0, n0 - 2) >> 1];
#pragma unroll
                        for (int u = 0; u < P2; ++u) {
                            const int j = j0 + 64 * u;
                            const bool v = j < n0;
                            const int jj = v ? j : n0 - 2;
                            const float2 q = q2_of(av[u], jj);
                            if (v) *(uint2*)(keys + j) = make_uint2(__float_as_uint(q.x), __float_as_uint(q.y));
                            const longlong2 w = *(const longlong2*)(wk + jj);
                            if (v) {
                                if (q.x < qp) flt += (unsigned long long)w.x;
                                if (q.y < qp) flt += (unsigned long long)w.y;
                                if (q.x == qp) fle += (unsigned long long)w.x;
                                if (q.y == qp) fle += (unsigned long long)w.y;
                            }
                        }
                    }
                    fle += flt;
                } else {
                    ext = false;
#pragma unroll 1
                    for (int j0 = 2 * lane; j0 < n0; j0 += 64 * P2) {
                        float2 av[P2];
                        av[0] = ap2[min(j0, n0 - 2) >> 1];
#pragma unroll
                        for (int u = 0; u < P2; ++u) {
                            const int j = j0 + 64 * u;
                            const bool v = j < n0;
                            const int jj = v ? j : n0 - 2;
                            const float2 q = q2_of(av[u], jj);
                            if (v) *(uint2*)(keys + j) = make_uint2(__float_as_uint(q.x), __float_as_uint(q.y));
                            const longlong2 w = *(const longlong2*)(wk + jj);
                            if (v && q.x > 0.f) f0 += (unsigned long long)w.x;  // weight of q > 0 here: F(0) = W - it
                            if (v && q.y > 0.f) f0 += (unsigned long long)w.y;
                        }
                    }
                }
            } else {
                if (warm) {
#pragma unroll 1
                    for (int j0 = lane; j0 < n0; j0 += 32 * PFK) {
                        float av[PFK];
#pragma unroll
                        for (int u = 0; u < PFK; ++u) av[u] = __uint_as_float(keys[min(j0 + 32 * u, n0 - 1)]);
#pragma unroll
                        for (int u = 0; u < PFK; ++u) {
                            const int j = j0 + 32 * u;
                            const bool v = j < n0;
                            const int jj = v ? j : n0 - 1;
                            const float q = qk_of(av[u], jj);
                            if (v) keys[j] = __float_as_uint(q);
                            const unsigned long long w = v ? (unsigned long long)wk[jj] : 0ull;
                            flt += (q < qp) ? w : 0ull;
                            fle += (q <= qp) ? w : 0ull;
                        }
                    }
                } else {
#pragma unroll 1
                    for (int j0 = lane; j0 < n0; j0 += 32 * PFK) {
                        float av[PFK];
#pragma unroll
                        for (int u = 0; u < PFK; ++u) av[u] = __uint_as_float(keys[min(j0 + 32 * u, n0 - 1)]);
#pragma unroll
                        for (int u = 0; u < PFK; ++u) {
                            const int j = j0 + 32 * u;
                            const bool v = j < n0;
                            const int jj = v ? j : n0 - 1;
                            const float q = qk_of(av[u], jj);
                            const unsigned kk = __float_as_uint(q);
                            if (v) keys[j] = kk;
                            const unsigned long long w = v ? (unsigned long long)wk[jj] : 0ull;
                            const bool pos = v && q > 0.f;
                            f0 += (q <= 0.f) ? w : 0ull;
                            mn = min(mn, pos ? kk : 0xffffffffu);
                            mx = max(mx, pos ? kk : 0u);
                            cnt += pos ? 1u : 0u;
                        }
                    }
                }
            }
            __syncwarp();
            float bn = 0.f;
            int jn = -1;
            bool zdec = false;  // F(0) >= T: the FP32 decision is beta = 0
            long long Fdec = 0; // F(< q*) of the FP32 decision q* (F(<= 0) when it is beta = 0)
            // bracket (lo, hi] of key bits with F(lo) < T <= F(hi); mn, mx, cnt: extent and size of the
            // breakpoints inside it
            unsigned lo = 0u, hi = QINF;
            long long Flo = 0, Fhi = W;
            bool search = false;
            if (warm) {
                const long long Flt = warp_sum64(flt), Fle = warp_sum64(fle);
                if (Flt < T && T <= Fle) {
                    bn = qp;  // the same breakpoint as last time
                    jn = jp;
                    Fdec = Flt;
                } else {
                    // missed: F(0) and the extent of the side of qp that holds the answer
                    const unsigned kp = __float_as_uint(qp);
                    if (Fle < T) { lo = kp; Flo = Fle; }
                    else { hi = kp - 1u; Fhi = Flt; }
#pragma unroll 1
                    for (int j0 = lane; j0 < n0; j0 += 32 * PFS) {
                        unsigned kq[PFS];
                        unsigned long long wq[PFS];
#pragma unroll
                        for (int u = 0; u < PFS; ++u) {
                            const int j = j0 + 32 * u;
                            const int jj = min(j, n0 - 1);
                            kq[u] = keys[jj];
                            wq[u] = j < n0 ? (unsigned long long)wk[jj] : 0ull;
                        }
#pragma unroll
                        for (int u = 0; u < PFS; ++u) {
                            const unsigned kk = kq[u];
                            const unsigned long long w = wq[u];
                            f0 += (__uint_as_float(kk) <= 0.f) ? w : 0ull;
                            const bool in = j0 + 32 * u < n0 && kk > lo && kk <= hi;
                            mn = min(mn, in ? kk : 0xffffffffu);
                            mx = max(mx, in ? kk : 0u);
                            cnt += in ? 1u : 0u;
                        }
                    }
                    const long long F0 = warp_sum64(f0);
                    if (lo == 0u) Flo = F0;
                    search = !(F0 >= T || W < T);
                    zdec = F0 >= T;
                    Fdec = F0;
                }
            } else {
                const long long F0 = ext ? warp_sum64(f0) : W - warp_sum64(f0);
                Flo = F0;
                search = !(F0 >= T || W < T);  // else beta = 0: slope at 0+ not positive, or no crossing
                zdec = F0 >= T;
                Fdec = F0;
            }
            if (search) {
                unsigned cmin = __reduce_min_sync(0xffffffffu, mn);
                unsigned cmax = __reduce_max_sync(0xffffffffu, mx);
                unsigned ncnt = __reduce_add_sync(0xffffffffu, cnt);
                if (!ext) {
                    // not taken yet: every positive key, at most n0 of them
                    cmin = 1u; cmax = QINF; ncnt = (unsigned)n0;
                }
                // Shrink to a single key.  Each pass splits the bracket at a pivot interpolated from
                // the weight still needed (after eight passes every other pass halves it) and takes F
                // at the pivot and the extent and size of both halves.  Once the bracket holds at most
                // CAPC breakpoints, the pass also moves them (key and element) to the front of the
                // warp's buffer, and later passes read only that list.
                bool listed = false;
                int m = n0;
                unsigned ks = 0u;
                const unsigned below = (1u << lane) - 1u;
                if (cmin != cmax && ncnt > (unsigned)SAMP_MIN) {
                    // First pivots from a sample: each lane takes its first breakpoint inside the bracket
                    // among elements lane, lane+32, lane+64, lane+96.  With phi the fraction of the
                    // bracket's weight still needed, p1 is the largest sample whose weighted rank is at
                    // most phi - SAMP_D and p2 the smallest at least phi + SAMP_D.  One pass takes F at
                    // both and moves the breakpoints between them to the front of the buffer (key and
                    // element, at most CAPC); when the quantile lies there (most of the time) the later
                    // passes read only that list, else the overwritten keys are recomputed.  The
                    // pivots only steer the search: every decision still uses the exact sums.
                    unsigned sk = 0u;
                    float sw = 0.f;
                    const int shw = max(0, 40 - __clzll(Fhi - Flo));  // bracket weights fit 24 bits
#pragma unroll
                    for (int t = 0; t < 4; ++t) {
                        const int j = lane + 32 * t;
                        const int jj = j < n0 ? j : 0;
                        const unsigned kk = keys[jj];
                        const bool ok = sk == 0u && j < n0 && kk >= cmin && kk <= cmax;
                        if (ok) { sk = kk; sw = (float)(unsigned)((unsigned long long)wk[jj] >> shw); }
                    }
                    // weight of the samples at or below each lane's own
                    float cw = 0.f, tot = 0.f;
#pragma unroll
                    for (int s = 0; s < 32; ++s) {
                        const unsigned k2 = __shfl_sync(0xffffffffu, sk, s);
                        const float w2 = __shfl_sync(0xffffffffu, sw, s);
                        tot += w2;
                        cw += (k2 <= sk) ? w2 : 0.f;
                    }
                    const float phi = ratio64(T - Flo, Fhi - Flo);
                    const bool has = sk != 0u;
                    unsigned p1 = __reduce_max_sync(0xffffffffu, (has && cw <= (phi - SAMP_D) * tot) ? sk : 0u);
                    unsigned p2 = __reduce_min_sync(0xffffffffu, (has && cw >= (phi + SAMP_D) * tot) ? sk : 0xffffffffu);
                    if (p1 == 0u) p1 = cmin - 1u;
                    if (p2 == 0xffffffffu) p2 = cmax;
                    if (tot > 0.f && p1 < p2 && (p1 >= cmin || p2 < cmax)) {
                        // F at both pivots; the breakpoints between them move to the front of the buffer
                        // (at most CAPC of them)
                        // offsets from cmin: d <= span inside the bracket (keys below it wrap past span),
                        // d < e1 at or below p1, d < e2 at or below p2
                        const unsigned span = cmax - cmin, e1 = p1 + 1u - cmin, e2 = p2 + 1u - cmin;
                        unsigned long long f1 = 0, fM = 0;
                        unsigned c1 = 0u, emn = 0xffffffffu, emx = 0u;
                        int wpos = 0;
#pragma unroll 1
                        for (int j00 = 0; j00 < n0; j00 += 32 * PFS) {
                          unsigned kq[PFS];
                          unsigned long long wq[PFS];
#pragma unroll
                          for (int u = 0; u < PFS; ++u) {
                              const int j = j00 + 32 * u + lane;
                              const int jj = j < n0 ? j : 0;
                              kq[u] = keys[jj];
                              wq[u] = (unsigned long long)wk[jj];
                          }
#pragma unroll
                          for (int u = 0; u < PFS; ++u) {
                            const int j = j00 + 32 * u + lane;
                            const bool v = j < n0;
                            const unsigned kk = kq[u];
                            const unsigned long long w = wq[u];
                            const unsigned d = v ? kk - cmin : 0xffffffffu;
                            const bool L1 = d < e1;
                            const bool M = !L1 && d < e2;
                            const unsigned bal = __ballot_sync(0xffffffffu, M);
                            const int q = wpos + __popc(bal & below);
                            if (M && q < CAPC) cidx[q] = (unsigned short)j;
                            wpos += __popc(bal);
                            if (L1) { f1 += w; ++c1; }
                            if (M) fM += w;
                            emn = min(emn, d);
                            emx = max(emx, d <= span ? d : 0u);
                          }
                        }
                        __syncwarp();
                        const long long F1 = Flo + warp_sum64(f1);
                        const long long F2 = F1 + warp_sum64(fM);
                        const unsigned n1 = __reduce_add_sync(0xffffffffu, c1);
                        bool keep = false;
                        if (F1 >= T) {
                            Fhi = F1; cmax = p1; ncnt = n1;
                            cmin += __reduce_min_sync(0xffffffffu, emn);
                        } else if (F2 >= T) {
                            Flo = F1; Fhi = F2; cmin = p1 + 1u; cmax = p2; ncnt = (unsigned)wpos;
                            keep = ncnt <= (unsigned)CAPC;
                        } else {
                            // at most the rest of the bracket
                            Flo = F2; cmax = cmin + __reduce_max_sync(0xffffffffu, emx); cmin = p2 + 1u;
                            ncnt -= n1 + (unsigned)wpos;
                        }
                        if (keep) {
                            listed = true;
                            m = (int)ncnt;
                        }
                    }
                }
#pragma unroll 1
                for (int it = 0; it < 96; ++it) {
                    if (cmin == cmax) { ks = cmin; break; }
                    lo = cmin - 1u;  // F unchanged: no breakpoint in (lo, cmin)
                    hi = cmax;       // F unchanged: no breakpoint in (cmax, hi]
                    unsigned mid;
                    if (it >= 8 && (it & 1)) {
                        mid = lo + ((hi - lo) >> 1);
                    } else {
                        const float fr = ratio64(T - Flo, Fhi - Flo);
                        unsigned off = (unsigned)(fr * (float)(hi - lo));
                        off = min(max(off, 1u), hi - lo - 1u);
                        mid = lo + off;
                    }
                    const bool wr = listed || ncnt <= (unsigned)CAPC;
                    // F at the pivot; the largest key at or below it and the smallest above it (the
                    // other extreme of either half is the bracket's own, cmin or cmax).  Offsets
                    // d = key - cmin: inside the bracket d <= span (keys below it wrap past span), in
                    // the lower half d <= dm; d - (dm + 1) is smallest for the upper half's least key.
                    const unsigned span = cmax - cmin, dm = mid - cmin, dm1 = dm + 1u;
                    unsigned long long fm = 0;
                    unsigned mxL = 0u, mnR = 0xffffffffu, cl = 0u;
                    int wpos = 0;
#pragma unroll 1
                    for (int j00 = 0; j00 < m; j00 += 32 * PFS) {
                      // (in-place compaction writes only at or before the positions this chunk read)
                      int eq[PFS];
                      unsigned kq[PFS];
                      unsigned long long wq[PFS];
#pragma unroll
                      for (int u = 0; u < PFS; ++u) {
                          const int j = j00 + 32 * u + lane;
                          const bool v = j < m;
                          const int jj = v ? j : 0;
                          eq[u] = v ? (listed ? (int)cidx[jj] : jj) : 0;
                      }
#pragma unroll
                      for (int u = 0; u < PFS; ++u) {
                          kq[u] = keys[eq[u]];
                          wq[u] = (unsigned long long)wk[eq[u]];
                      }
#pragma unroll
                      for (int u = 0; u < PFS; ++u) {
                        const int j = j00 + 32 * u + lane;
                        const bool v = j < m;
                        const int e = eq[u];
                        const unsigned kk = kq[u];
                        const unsigned d = v ? kk - cmin : 0xffffffffu;
                        const bool in = d <= span;
                        if (wr) {
                            // in-place compaction: every write lands at or before the position read
                            const unsigned bal = __ballot_sync(0xffffffffu, in);
                            const int q = wpos + __popc(bal & below);
                            if (in) cidx[q] = (unsigned short)e;
                            wpos += __popc(bal);
                        }
                        const unsigned long long w = wq[u];
                        const bool L = d <= dm;
                        if (L) { fm += w; ++cl; }
                        mxL = max(mxL, L ? d : 0u);
                        mnR = min(mnR, d - dm1);
                      }
                    }
                    __syncwarp();
                    if (wr) { listed = true; m = wpos; }
                    const long long Fm = Flo + warp_sum64(fm);
                    const unsigned nl = __reduce_add_sync(0xffffffffu, cl);
                    if (Fm >= T) {
                        hi = mid; Fhi = Fm;
                        cmax = cmin + __reduce_max_sync(0xffffffffu, mxL);  // cmin stays
                        ncnt = nl;
                    } else {
                        lo = mid; Flo = Fm;
                        cmin = cmin + dm1 + __reduce_min_sync(0xffffffffu, mnR);  // cmax stays
                        ncnt -= nl;
                    }
                }
                bn = (ks != 0u) ? __uint_as_float(ks) : 0.f;
                Fdec = Flo;  // F(< ks): the bracket's lower end is ks - 1
                // the element holding the selected breakpoint (lowest index among ties)
                if (ks != 0u) {
                    if (listed) {
                        int jm = INT_MAX;
                        for (int j = lane; j < m; j += 32)
                            if (keys[cidx[j]] == ks) jm = min(jm, (int)cidx[j]);
                        jm = __reduce_min_sync(0xffffffffu, jm);
                        jn = (jm == INT_MAX) ? -1 : jm;
                    } else {
                        for (int j0 = 0; j0 < n0 && jn < 0; j0 += 32) {
                            const int j = j0 + lane;
                            const unsigned bal = __ballot_sync(0xffffffffu, j < n0 && keys[j] == ks);
                            if (bal) jn = j0 + __ffs(bal) - 1;
                        }
                    }
                }
            }
            float bln = 0.f;
            if constexpr (CERT) {
                const int dec = (jn >= 0 && bn > 0.f) ? 1 : (zdec ? 0 : 2);
                if (dec != 2) {
                    CertState cst;
                    cst.bn = bn; cst.bln = 0.f; cst.jn = jn;
                    const float amx = SPEC ? a.samax[o] : __ldg(a.amax + (side ? a.U + c : c));
                    if constexpr (WIDE) {
                        cc_certify<true>(n0, R, k, lane, rw.gs, rk, wk, keys, cidx, ap, sa, bsm, blsm, amx, T,
                                         Fdec, dec, &cst);
                    } else {
                        // the leading parts in the warp's shared slots after the trailing ones
#pragma unroll
                        for (int p = 0; p < RC; ++p) blsm[RMAX_CC + p] = beta[p];
                        __syncwarp();
                        cc_certify<false>(n0, R, k, lane, rw.gs, rk, wk, keys, cidx, ap, sa, blsm + RMAX_CC, blsm,
                                          amx, T, Fdec, dec, &cst);
                    }
                    bn = cst.bn; bln = cst.bln; jn = cst.jn;
#pragma unroll
                    for (int i = 0; i < 5; ++i) my_cs[i] += cst.cs[i];
                }
            }
            __syncwarp();  // the next step rewrites the key buffer
            if constexpr (WIDE) {
                bsm[k] = bn; jsm[k] = jn;  // every lane writes the same values
            } else {
#pragma unroll
                for (int p = 0; p < RC; ++p)
                    if (p == k) { beta[p] = bn; jprev[p] = jn; }
            }
            if (CERT) blsm[k] = bln;
            if (bn != bk || bln != blk) {
                changed = true;
                dirty |= all_rows & ~(1u << k);
            }
        }
        if (!changed) break;
    }
    // With every multiplier 0 the dual objective is the target's plane concretised over the clipped
    // box, which re-concretisation has already folded into l / u: nothing to update.
    bool any = false;
#pragma unroll
    for (int p = 0; p < RC; ++p) {
        if (WIDE && p >= R) break;
        any |= (bget(p) != 0.f);
    }
    if (!any) return;
    // dual objective at beta, FP32 with its rounding bound: the plane again in the key buffer (the keys
    // are no longer needed), the box as staged for the work item
    __syncwarp();
    cc_plane_to_smem(keys, ap, n0, lane);
    float* keys_f = (float*)keys;
    const float* apl = keys_f;
    const float* slo = blo;
    const float* shi = bhi;
    const float psc = SPEC ? a.sscale[o] : __ldg(a.pscale + (side ? a.U + c : c));
    const float cur = SPEC ? a.slower[o] : (side == 0 ? a.l[o] : -a.u[o]);
    float part = 0.f;
    unsigned nzv = 0u;  // rows with a nonzero multiplier (wide launch)
    float sval = sa;    // factor of the buffer: 1 once the wide launch has formed a' over it
    if constexpr (WIDE) {
        for (int p = 0; p < R; ++p)
            if (bsm[p] != 0.f) nzv |= 1u << p;
        sval = cc_accum_rows(keys_f, rw.gs, bsm, nzv, n0, sa, lane);
    }
    if (!WIDE && (n0 & 1) == 0) {
        // two adjacent elements per lane, packed FP32: each lane sums at most ceil(n0/64) terms per
        // component and one more to combine them, within the ceil(n0/32) the rounding bound allows
        const float2* ap2 = (const float2*)apl;
        const float2* slo2 = (const float2*)slo;
        const float2* shi2 = (const float2*)shi;
        const float2 sa2 = make_float2(sa, sa);
        float2 part2 = make_float2(0.f, 0.f);
#pragma unroll 1
        for (int j0 = 2 * lane; j0 < n0; j0 += 64 * 2) {
            float2 av[2], lv[2], hv[2];
#pragma unroll
            for (int u = 0; u < 2; ++u) {
                const int jj = min(j0 + 64 * u, n0 - 2);
                const bool in = j0 + 64 * u < n0;
                av[u] = ap2[jj >> 1];
                lv[u] = in ? slo2[jj >> 1] : make_float2(0.f, 0.f);
                hv[u] = in ? shi2[jj >> 1] : make_float2(0.f, 0.f);
            }
#pragma unroll
            for (int u = 0; u < 2; ++u) {
                const int jj = min(j0 + 64 * u, n0 - 2);
                float2 v = __fmul2_rn(av[u], sa2);
#pragma unroll
                for (int p = 0; p < (WIDE ? 1 : RC); ++p)
                    v = __ffma2_rn(make_float2(bget(p), bget(p)), *(const float2*)(rw.gs + p * n0 + jj), v);
                const float2 t1 = __fmul2_rn(v, lv[u]), t2 = __fmul2_rn(v, hv[u]);
                part2 = __fadd2_rn(part2, make_float2(fminf(t1.x, t2.x), fminf(t1.y, t2.y)));
            }
        }
        part = part2.x + part2.y;
    } else {
#pragma unroll 1
        for (int j0 = lane; j0 < n0; j0 += 32 * PF) {
            float av[PF], lv[PF], hv[PF];
#pragma unroll
            for (int u = 0; u < PF; ++u) {
                const int jj = min(j0 + 32 * u, n0 - 1);
                const bool in = j0 + 32 * u < n0;
                av[u] = apl[jj];
                lv[u] = in ? slo[jj] : 0.f;
                hv[u] = in ? shi[jj] : 0.f;
            }
#pragma unroll
            for (int u = 0; u < PF; ++u) {
                const int jj = min(j0 + 32 * u, n0 - 1);
                float v = sval * av[u];
                if constexpr (WIDE) {
                    // a' already formed over the buffer (zero multipliers add nothing)
                } else {
#pragma unroll
                    for (int p = 0; p < RC; ++p) v = fmaf(bget(p), rw.gs[p * n0 + jj], v);
                }
                part += fminf(v * lv[u], v * hv[u]);  // 0 past n0 (lv = hv = 0)
            }
        }
    }
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) part += __shfl_xor_sync(0xffffffffu, part, off);
    float cst = c0;
    // Rounding bound gam * scale, scale = sum_j S_j max(|lo_j|, |hi_j|) + |c0| + sum_p beta_p |h_p| with
    // S_j = |a_j| + sum_p beta_p |g_pj| (bounded through the root box: psc and Sg + |h| per row, in FP32
    // with every operation rounded up).  Operation count, in units of u = 2^-24 times scale:
    //  - v_j = a_j + sum_p beta_p g_pj: R fma roundings; the product with lo or hi: 1;
    //  - the sums: the packed path adds ceil(n0/64) terms per component, 1 to combine them and 5 shuffle
    //    levels; the scalar path ceil(n0/32) terms and 5 levels; cst = c0 + sum_p beta_p h_p: R fmas,
    //    disjoint terms of the same scale;
    //  - the dropped trailing parts of the multipliers change D by at most u * scale: 1.
    // So R + ceil(n0/32) + 7 suffices on both paths; gam takes R + ceil(n0/32) + 12 (second-order terms
    // are inside the factors 1.0001).  The final sum and the pad are rounded outward.
    float scale = __fadd_ru(psc, fabsf(c0));
#pragma unroll
    for (int p = 0; p < RC; ++p) {
        if (WIDE && p >= R) break;
        cst = fmaf(bget(p), cch<WIDE>(p), cst);
        scale = __fmaf_ru(bget(p), ccSgH<WIDE>(p), scale);
    }
    const float gam = __fmul_ru((float)(R + (n0 + 31) / 32 + 12), 5.9611e-08f);  // >= 2^-24 * 1.0001
    const float pad = __fmul_ru(__fmul_ru(gam, scale), 1.0001f);
    float val = __fsub_rd(__fadd_rd(part, cst), pad);
    const float valhi = __fadd_ru(__fadd_ru(part, cst), pad);
    if (val < 0.f && valhi >= 0.f && cur < 0.f) {
        // the stability decision is uncertain in FP32: evaluate D(beta) in FP64
        double d = 0.0;
        for (int j = lane; j < n0; j += 32) {
            double v = (double)(sa * __ldg(ap + j));  // (the wide launch's buffer holds a', not a)
#pragma unroll
            for (int p = 0; p < RC; ++p) {
                if (WIDE && p >= R) break;
                v += (double)bget(p) * (double)rw.gs[p * n0 + j];
            }
            d += fmin(v * (double)slo[j], v * (double)shi[j]);
        }
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) d += __shfl_xor_sync(0xffffffffu, d, off);
        d += (double)c0;
#pragma unroll
        for (int p = 0; p < RC; ++p) {
            if (WIDE && p >= R) break;
            d += (double)bget(p) * (double)cch<WIDE>(p);
        }
        // D at the leading parts differs from D at the full multipliers (the ascent's point) by at most
        // sum_p |beta_lo,p| (sum_j |g_pj| max(|lo_j|, |hi_j|) + |h_p|); charged so that the bound never
        // exceeds the value at the full multipliers (in the FP32 path the 12 u of slack in gam covers it)
        float tpad = 0.f;
        if (CERT) {
#pragma unroll
            for (int p = 0; p < RC; ++p) {
                if (WIDE && p >= R) break;
                tpad = __fmaf_ru(fabsf(blsm[p]), ccSgH<WIDE>(p), tpad);
            }
        }
        val = __double2float_rd(d - ldexp((double)scale, -40) - (double)tpad);
    }
    if (lane == 0) {
        if (SPEC) { if (val > a.slower[o]) a.slower[o] = val; }
        else if (side == 0) { if (val > a.l[o]) a.l[o] = val; }
        else { const float ub = -val; if (ub < a.u[o]) a.u[o] = ub; }
    }
}

// WIDE: the tasks of subdomains with more than RTPL rows, taken by each warp on its own (one block
// per SM, more registers); otherwise the rest, in work items shared by a block's warps.
template <bool WIDE, bool SPEC>
__global__ void __launch_bounds__((WIDE ? NWARPW : NWARP) * 32, WIDE ? 1 : 2) k_complete(CCArgs a) {
    const int n0 = a.n0, Rs = a.Rs, B = a.B;
    const int RsS = Rs < RTPL ? Rs : RTPL;  // rows staged by the main launch
    const int lane = threadIdx.x & 31;
    const CCView sv = cc_view(n0, RsS, WIDE);
    __shared__ int s_item, s_pos, s_R, s_next;
    __shared__ unsigned long long nsteps, ncs[5];
    if (threadIdx.x == 0) { nsteps = 0; ncs[0] = ncs[1] = ncs[2] = ncs[3] = ncs[4] = 0; }
    unsigned long long my_steps = 0;
    unsigned my_cs[5] = {0u, 0u, 0u, 0u, 0u};
    const int np = *a.nplaced;
    if constexpr (WIDE) {
        // Each warp takes (target, side) tasks one at a time from the wide launch's ticket, over the
        // subdomains in order of decreasing row count, holding its subdomain's row constants in its
        // own slots: no block barrier between tasks.  The rows and the box are read from L2.
        __syncthreads();  // the block's counters are initialised
        const int warp = threadIdx.x >> 5;
        const int npw = a.allwide ? np : *a.nwpos;
        const int total = a.toff[npw];
        const bool have_list = a.tgt_off != nullptr;
        int cb = -1, R = 0, tbeg = 0, tend = 0, t0 = 0;
        CCRows rw;
        rw.gs = nullptr; rw.rg = nullptr; rw.w64 = nullptr;
        const float* blo = nullptr;
        const float* bhi = nullptr;
        for (;;) {
            int t = 0;
            if (lane == 0) t = (int)atomicAdd(&a.ticket[0], 1u);
            t = __shfl_sync(0xffffffffu, t, 0);
            if (t >= total) break;
            if (t < tbeg || t >= tend) {
                int pos = 0;
                if (lane == 0) {
                    int lo = 0, hi = npw - 1;  // the last position whose first task is <= t
                    while (lo < hi) {
                        const int mid = (lo + hi + 1) >> 1;
                        if (a.toff[mid] <= t) lo = mid; else hi = mid - 1;
                    }
                    pos = lo;
                }
                pos = __shfl_sync(0xffffffffu, pos, 0);
                tbeg = a.toff[pos];
                tend = a.toff[pos + 1];
                const int b = a.order[pos];
                if (b != cb) {
                    R = a.wR[b];
                    if (lane < R) {
                        const size_t q = (size_t)b * Rs + lane;
                        cc_wT64[warp][lane] = a.wT[q];
                        cc_wW64[warp][lane] = a.wW[q];
                        cc_whrow[warp][lane] = a.wh[q];
                        cc_wSgH[warp][lane] = __double2float_ru(a.wSg[q] + fabs((double)a.wh[q]));
                        cc_wGm[warp][lane] = a.wGm[q];
                    }
                    __syncwarp();
                    cb = b;
                    const size_t base = (size_t)b * Rs * n0;
                    rw.gs = a.wg + base; rw.rg = a.wrg + base; rw.w64 = a.ww + base;
                    blo = a.lo + (size_t)b * n0;
                    bhi = a.hi + (size_t)b * n0;
                    t0 = have_list ? a.tgt_off[b] : 0;
                }
            }
            const int tl = t - tbeg;  // the task's index within its subdomain
            int c, side;
            if (SPEC) {
                c = tl;
                side = 0;
                if (a.slower[(size_t)cb * a.m + c] > 0.f) continue;  // proven already
            } else {
                const int ti = tl >> 1;
                side = tl & 1;
                c = have_list ? a.tgt_ids[t0 + ti] : ti;
                if (c < 0 || c >= a.U) {
                    if (lane == 0) atomicOr(a.status, CV_DEV_TARGET);
                    continue;
                }
                if (a.mask[(size_t)cb * a.U + c] != 0) continue;
            }
            if (R <= 8) cc_task<8, true, SPEC>(a, rw, sv.keys, sv.cidx, sv.bsm, sv.blsm, sv.jsm, blo, bhi, R, cb, c, side, lane, my_steps, my_cs);
            else if (R <= 16) cc_task<16, true, SPEC>(a, rw, sv.keys, sv.cidx, sv.bsm, sv.blsm, sv.jsm, blo, bhi, R, cb, c, side, lane, my_steps, my_cs);
            else cc_task<32, true, SPEC>(a, rw, sv.keys, sv.cidx, sv.bsm, sv.blsm, sv.jsm, blo, bhi, R, cb, c, side, lane, my_steps, my_cs);
            __syncwarp();
        }
    } else {
        const int ibeg = *a.wide;
        const int total = a.ioff[B];
        int cur_b = -1;
        for (;;) {
            __syncthreads();
            if (threadIdx.x == 0) {
                const int it = ibeg + (int)atomicAdd(&a.ticket[1], 1u);
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
                // stage the subdomain's row constants (and, in the main launch, its rows)
                if (threadIdx.x == 0) s_R = a.wR[b];
                __syncthreads();
                const int R = s_R;
                {
                    const size_t base = (size_t)b * Rs * n0;
                    for (int i = threadIdx.x; i < R * n0; i += blockDim.x) {
                        sv.w64[i] = a.ww[base + i];
                        sv.gs[i] = a.wg[base + i];
                        sv.rg[i] = a.wrg[base + i];
                    }
                }
                for (int i = threadIdx.x; i < n0; i += blockDim.x) {
                    sv.blo[i] = a.lo[(size_t)b * n0 + i];
                    sv.bhi[i] = a.hi[(size_t)b * n0 + i];
                }
                if (threadIdx.x < R) {
                    cc_T64[threadIdx.x] = a.wT[(size_t)b * Rs + threadIdx.x];
                    cc_W64[threadIdx.x] = a.wW[(size_t)b * Rs + threadIdx.x];
                    cc_hrow[threadIdx.x] = a.wh[(size_t)b * Rs + threadIdx.x];
                    cc_Sg[threadIdx.x] = a.wSg[(size_t)b * Rs + threadIdx.x];
                    cc_SgH[threadIdx.x] = __double2float_ru(cc_Sg[threadIdx.x] + fabs((double)cc_hrow[threadIdx.x]));
                    cc_Gm[threadIdx.x] = a.wGm[(size_t)b * Rs + threadIdx.x];
                    cc_Rm[threadIdx.x] = a.wRm[(size_t)b * Rs + threadIdx.x];
                }
                cur_b = b;
            }
            const int R = s_R;
            CCRows rw;
            rw.gs = sv.gs; rw.rg = sv.rg; rw.w64 = sv.w64;
            const bool have_list = a.tgt_off != nullptr;
            const int t0 = have_list ? a.tgt_off[b] : 0;
            const int ntask = SPEC ? a.m : 2 * ntargets(a, b);
            const int first = (item - a.ioff[pos]) * tpi_of(a, R);
            const int last = min(first + tpi_of(a, R), ntask);
            if (threadIdx.x == 0) s_next = first;
            __syncthreads();
            // the warps take the item's tasks one at a time from its counter
            for (;;) {
                int t = 0;
                if (lane == 0) t = atomicAdd(&s_next, 1);
                t = __shfl_sync(0xffffffffu, t, 0);
                if (t >= last) break;
                int c, side;
                if (SPEC) {
                    c = t;
                    side = 0;
                    if (a.slower[(size_t)b * a.m + c] > 0.f) continue;  // proven already
                } else {
                    const int ti = t >> 1;
                    side = t & 1;
                    c = have_list ? a.tgt_ids[t0 + ti] : ti;
                    if (c < 0 || c >= a.U) {
                        if (lane == 0) atomicOr(a.status, CV_DEV_TARGET);
                        continue;
                    }
                    if (a.mask[(size_t)b * a.U + c] != 0) continue;
                }
                {
                    switch (R) {
                        case 1: cc_task<1, false, SPEC>(a, rw, sv.keys, sv.cidx, nullptr, sv.blsm, nullptr, sv.blo, sv.bhi, 1, b, c, side, lane, my_steps, my_cs); break;
                        case 2: cc_task<2, false, SPEC>(a, rw, sv.keys, sv.cidx, nullptr, sv.blsm, nullptr, sv.blo, sv.bhi, 2, b, c, side, lane, my_steps, my_cs); break;
                        case 3: cc_task<3, false, SPEC>(a, rw, sv.keys, sv.cidx, nullptr, sv.blsm, nullptr, sv.blo, sv.bhi, 3, b, c, side, lane, my_steps, my_cs); break;
                        default: cc_task<4, false, SPEC>(a, rw, sv.keys, sv.cidx, nullptr, sv.blsm, nullptr, sv.blo, sv.bhi, 4, b, c, side, lane, my_steps, my_cs); break;
                    }
                }
                __syncwarp();
            }
        }
    }
    if (a.steps && lane == 0) {
        if (my_steps) atomicAdd(&nsteps, my_steps);
        for (int i = 0; i < 5; ++i)
            if (my_cs[i]) atomicAdd(&ncs[i], (unsigned long long)my_cs[i]);
    }
    __syncthreads();
    if (a.steps && threadIdx.x == 0) {
        if (nsteps) atomicAdd(a.steps, nsteps);
        for (int i = 0; i < 5; ++i)
            if (ncs[i]) atomicAdd(a.steps + 1 + i, ncs[i]);
    }
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

template <bool WIDE, bool SPEC>
cv_status launch_cc_one(const CCArgs& a, int* launches, cudaStream_t st) {
    const size_t n0r = (a.n0 + 31) & ~31;
    const size_t RsS = a.Rs < RTPL ? a.Rs : RTPL;
    // main: staged rows and box + per warp keys and list; wide: per warp keys, list and multiplier
    // slots (its row constants are static shared memory, CC_WCONST bytes)
    const size_t fixed = WIDE ? 0 : RsS * a.n0 * (8 + 4 + 4) + (size_t)a.n0 * 8;  // rows, box
    const size_t per_warp = n0r * 4 + CAPC * 2 + (WIDE ? (size_t)RMAX_CC * 12 : (size_t)RMAX_CC * 8);
    const size_t limit = 220 * 1024 - (WIDE ? CC_WCONST : 0);
    int nw = WIDE ? NWARPW : NWARP;
    while (nw > 1 && fixed + nw * per_warp > limit) --nw;
    const size_t smem = fixed + nw * per_warp;
    if (smem > limit || a.n0 > 65535) {
        cv_set_error("complete clipping: input dimension too large for the shared-memory row cache");
        return CV_EUNSUPPORTED;
    }
    CV_CUDA(cudaFuncSetAttribute(k_complete<WIDE, SPEC>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    int dev = 0, sms = 0, per = 0;
    CV_CUDA(cudaGetDevice(&dev));
    CV_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    CV_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_complete<WIDE, SPEC>, nw * 32, smem));
    if (per < 1) per = 1;
    k_complete<WIDE, SPEC><<<sms * per, nw * 32, smem, st>>>(a);
    CV_LAUNCH_CHECK("k_complete");
    ++*launches;
    return CV_OK;
}

template <bool SPEC>
cv_status launch_cc(const CCArgs& a0, int* launches, cudaStream_t st) {
    // The main launch stages up to RTPL rows of a subdomain (16 bytes per element) and the box in shared
    // memory; when that does not fit next to one warp's buffers (large inputs), the wide launch, which
    // reads the rows from the L2-resident workspace, takes every subdomain.
    CCArgs a = a0;
    const size_t n0r = (a.n0 + 31) & ~31;
    const size_t RsS = a.Rs < RTPL ? a.Rs : RTPL;
    const size_t main_min = RsS * a.n0 * 16 + (size_t)a.n0 * 8 + n0r * 4 + CAPC * 2 + (size_t)RMAX_CC * 8;
    a.allwide = main_min > 220 * 1024;
    if (a.allwide) return launch_cc_one<true, SPEC>(a, launches, st);
    if (a.Rs > RTPL) {
        cv_status s = launch_cc_one<true, SPEC>(a, launches, st);
        if (s) return s;
    }
    return launch_cc_one<false, SPEC>(a, launches, st);
}

// spec-plane mode: magnitude scale of every final plane against its subdomain's clipped box,
// sum_j |A_j| max(|lo_j|, |hi_j|) + |c|, an upper bound (FP32, every operation rounded up: the
// terms are non-negative) for the error pad of the dual value
__global__ void k_spec_scale(int m, int n0, const float* A, const float* c, const float* lo, const float* hi,
                             float* sscale, float* samax) {
    const size_t o = blockIdx.x;  // b * m + r
    const size_t b = o / (size_t)m;
    float mag = 0.f, amx = 0.f;
    for (int j = threadIdx.x; j < n0; j += blockDim.x) {
        const float av = fabsf(A[o * n0 + j]);
        mag = __fmaf_ru(av, fmaxf(fabsf(lo[b * n0 + j]), fabsf(hi[b * n0 + j])), mag);
        amx = fmaxf(amx, av);
    }
    __shared__ float red[32], redm[32];
    for (int off = 16; off > 0; off >>= 1) {
        mag = __fadd_ru(mag, __shfl_xor_sync(0xffffffffu, mag, off));
        amx = fmaxf(amx, __shfl_xor_sync(0xffffffffu, amx, off));
    }
    if ((threadIdx.x & 31) == 0) { red[threadIdx.x >> 5] = mag; redm[threadIdx.x >> 5] = amx; }
    __syncthreads();
    if (threadIdx.x == 0) {
        float t = 0.f, mm = 0.f;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) { t = __fadd_ru(t, red[w]); mm = fmaxf(mm, redm[w]); }
        sscale[o] = __fadd_ru(t, fabsf(c[o]));
        samax[o] = mm;
    }
}

}  // namespace

size_t cv_cc_workspace(int B, int Rmax, int n0) {
    const size_t Rs = Rmax < RMAX_CC ? Rmax : RMAX_CC;
    if (Rs == 0) return 0;
    const size_t b = B;
    size_t s = 0;
    s += cv_align256(b * Rs * n0 * 4) * 2;  // wg, wrg
    s += cv_align256(b * Rs * n0 * 8);      // ww
    s += cv_align256(b * Rs * 8) * 3;       // wT, wW, wSg
    s += cv_align256(b * Rs * 4) * 3;       // wh, wGm, wRm
    s += cv_align256(b * 4) * 3;            // wR, wcnt, order
    s += cv_align256((b + 1) * 4) * 2;      // ioff, toff
    s += 256 * 2;                           // nplaced / wide / nwpos, ticket
    return s;
}

cv_status cv_launch_complete(const cv_net* net, const cv_cache* cache, const cv_batch_in* in,
                             const cv_options* opt, const cv_ws_layout* lay, char* ws,
                             const float* lo_clip, const float* hi_clip, float* l, float* u,
                             int8_t* mask, uint8_t* infeasible, unsigned long long* step_counter,
                             int* launches, cudaStream_t st) {
    if (opt->sweeps <= 0 || lay->Rmax == 0 || cache->U == 0) return CV_OK;
    if (lay->Rmax > RMAX_CC) {
        cv_set_error("complete clipping: more than 32 constraint rows per subdomain are not supported");
        return CV_EUNSUPPORTED;
    }
    CCArgs a;
    a.B = in->B; a.U = cache->U; a.n0 = cache->n0; a.H = cache->H; a.Rmax = lay->Rmax; a.sweeps = opt->sweeps;
    a.Rs = lay->Rmax < RMAX_CC ? lay->Rmax : RMAX_CC;
    for (int i = 0; i < 3; ++i) a.tpi[i] = cache->cc_items[i];
    a.spec = 0; a.m = 0; a.sA = nullptr; a.sc = nullptr; a.sscale = nullptr; a.slower = nullptr;
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
    a.amax = cache->amax; a.samax = nullptr;
    // workspace carve (the layout of cv_cc_workspace)
    const size_t B = in->B, Rs = a.Rs, n0 = cache->n0;
    char* p = ws + lay->cc;
    a.wg = (float*)p; p += cv_align256(B * Rs * n0 * 4);
    a.wrg = (float*)p; p += cv_align256(B * Rs * n0 * 4);
    a.ww = (long long*)p; p += cv_align256(B * Rs * n0 * 8);
    a.wT = (long long*)p; p += cv_align256(B * Rs * 8);
    a.wW = (long long*)p; p += cv_align256(B * Rs * 8);
    a.wSg = (double*)p; p += cv_align256(B * Rs * 8);
    a.wh = (float*)p; p += cv_align256(B * Rs * 4);
    a.wGm = (float*)p; p += cv_align256(B * Rs * 4);
    a.wRm = (float*)p; p += cv_align256(B * Rs * 4);
    a.wR = (int*)p; p += cv_align256(B * 4);
    a.wcnt = (int*)p; p += cv_align256(B * 4);
    a.order = (int*)p; p += cv_align256(B * 4);
    a.ioff = (int*)p; p += cv_align256((B + 1) * 4);
    a.toff = (int*)p; p += cv_align256((B + 1) * 4);
    a.nplaced = (int*)p;
    a.wide = a.nplaced + 1;
    a.nwpos = a.nplaced + 2;
    p += 256;
    a.ticket = (unsigned*)p;
    k_cc_prep<<<in->B, 256, 0, st>>>(a);
    CV_LAUNCH_CHECK("k_cc_prep");
    k_cc_scan<<<1, 1024, 0, st>>>(a);
    CV_LAUNCH_CHECK("k_cc_scan");
    *launches += 3;  // prep, scan, post
    cv_status s = launch_cc<false>(a, launches, st);
    if (s) return s;
    k_cc_post<<<in->B, 256, 0, st>>>(a);
    CV_LAUNCH_CHECK("k_cc_post");
    return CV_OK;
}

cv_status cv_launch_spec_clip(const cv_net* net, const cv_cache* cache, const cv_batch_in* in, cv_batch_out* out,
                              const cv_options* opt, const cv_ws_layout* lay, char* ws, float* sscale,
                              unsigned long long* step_counter, int* launches, cudaStream_t st) {
    (void)net;
    if (opt->sweeps <= 0 || lay->Rmax == 0 || in->B == 0 || in->m == 0) return CV_OK;
    if (lay->Rmax > RMAX_CC) {
        cv_set_error("spec clipping: more than 32 constraint rows per subdomain are not supported");
        return CV_EUNSUPPORTED;
    }
    CCArgs a;
    memset(&a, 0, sizeof(a));
    a.B = in->B; a.U = cache->U; a.n0 = cache->n0; a.H = cache->H; a.Rmax = lay->Rmax; a.sweeps = opt->sweeps;
    a.Rs = lay->Rmax < RMAX_CC ? lay->Rmax : RMAX_CC;
    for (int i = 0; i < 3; ++i) a.tpi[i] = cache->cc_items[i];
    a.rowflag = (const int8_t*)(ws + lay->rowflag);
    a.lA = cache->lA; a.lc = cache->lc; a.uA = cache->uA; a.uc = cache->uc;
    a.slot_of = cache->slot_of; a.pscale = cache->pscale;
    a.root_lo = cache->root_lo; a.root_hi = cache->root_hi;
    a.split_off = in->split_off; a.split_ids = in->split_ids;
    a.row_off = in->row_off; a.G = in->G; a.h = in->h;
    a.tgt_off = nullptr; a.tgt_ids = nullptr;
    a.lo = out->lo_clip; a.hi = out->hi_clip;
    a.infeasible = out->infeasible; a.status = cache->net->status;
    a.spec = 1; a.m = in->m;
    a.sA = out->final_A; a.sc = out->final_c; a.sscale = sscale; a.slower = out->lower;
    a.amax = cache->amax;
    a.samax = sscale + (size_t)in->B * in->m;  // the scratch holds the scales, then the maxima
    a.steps = step_counter;
    const size_t B = in->B, Rs = a.Rs, n0 = cache->n0;
    char* p = ws + lay->cc;
    a.wg = (float*)p; p += cv_align256(B * Rs * n0 * 4);
    a.wrg = (float*)p; p += cv_align256(B * Rs * n0 * 4);
    a.ww = (long long*)p; p += cv_align256(B * Rs * n0 * 8);
    a.wT = (long long*)p; p += cv_align256(B * Rs * 8);
    a.wW = (long long*)p; p += cv_align256(B * Rs * 8);
    a.wSg = (double*)p; p += cv_align256(B * Rs * 8);
    a.wh = (float*)p; p += cv_align256(B * Rs * 4);
    a.wGm = (float*)p; p += cv_align256(B * Rs * 4);
    a.wRm = (float*)p; p += cv_align256(B * Rs * 4);
    a.wR = (int*)p; p += cv_align256(B * 4);
    a.wcnt = (int*)p; p += cv_align256(B * 4);
    a.order = (int*)p; p += cv_align256(B * 4);
    a.ioff = (int*)p; p += cv_align256((B + 1) * 4);
    a.toff = (int*)p; p += cv_align256((B + 1) * 4);
    a.nplaced = (int*)p;
    a.wide = a.nplaced + 1;
    a.nwpos = a.nplaced + 2;
    p += 256;
    a.ticket = (unsigned*)p;
    k_spec_scale<<<(unsigned)(B * in->m), 256, 0, st>>>(in->m, (int)n0, out->final_A, out->final_c, out->lo_clip,
                                                       out->hi_clip, sscale, sscale + B * in->m);
    CV_LAUNCH_CHECK("k_spec_scale");
    k_cc_prep<<<in->B, 256, 0, st>>>(a);
    CV_LAUNCH_CHECK("k_cc_prep");
    k_cc_scan<<<1, 1024, 0, st>>>(a);
    CV_LAUNCH_CHECK("k_cc_scan");
    *launches += 3;
    return launch_cc<true>(a, launches, st);
}
