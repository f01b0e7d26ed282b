// The activation branch-and-bound loop of Algorithm 5 (Clip-and-Verify for activation BaB) with
// every step on the GPU: Batch_Pick_Out, Batch_Split (cv_activation_split, BaBSR score with the
// weight of the Appendix's neuron selection heuristic), Top-K_Heuristic (cv_select_targets), the
// round (cv_bound_batch: Domain_Clipper, Domain_Update, Solve_Bound) and Domain_Filter.
//
// D_Unknown is a stack in device memory: per domain its split codes (CSR, offsets from 0), its
// clipped box, the bounds / mask / BaBSR weight of its cached neurons and its least spec lower
// bound.  The picked parents are the top P domains; their children's survivors are written back
// from the first picked position on, so the rest of the stack is never moved.  The host loop
// (native) reads two small counts per iteration: the children (the round's B) and the survivors.
//
// Kernels of this file: k_bab_inherit (block per child: the parent's mask with the new split fixed
// and the parent's weight), k_bab_tally (one block: stuck parents), k_bab_filter (one block: keep
// flags, positions by an ordered scan, counts, least lower bound), k_bab_push (block per child:
// the survivors onto the stack).  All stream the per-domain arrays once: HBM-bound and small next
// to the round.
#include "cv_internal.cuh"

#include <math.h>
#include <string.h>

#include <string>
#include <vector>

namespace {

// device counters of one call (int words; the last one holds float bits)
enum { ST_NCHILD = 0, ST_STUCK, ST_VER, ST_INF, ST_DEPTH, ST_PUSHED, ST_CODES, ST_LMIN, ST_N = 8 };

__global__ void k_bab_inherit(int U, const int* nchild, int base, const int* parent, const int* branched,
                              const int8_t* s_mask, const float* s_w, int8_t* c_mask, float* c_w) {
    const int ch = blockIdx.x;
    if (ch >= *nchild) return;
    const size_t pg = (size_t)(base + parent[ch]) * U, co = (size_t)ch * U;
    const int br = branched[ch];
    const int8_t side = (ch & 1) ? (int8_t)1 : (int8_t)-1;  // child 2k: z <= 0, child 2k + 1: z >= 0
    for (int c = threadIdx.x; c < U; c += blockDim.x) {
        c_mask[co + c] = (c == br) ? side : s_mask[pg + c];
        c_w[co + c] = s_w[pg + c];
    }
}

__device__ __forceinline__ int block_sum(int v, int* red) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    __syncthreads();
    if (lane == 0) red[warp] = v;
    __syncthreads();
    int t = 0;
    for (int w = 0; w < nw; ++w) t += red[w];
    return t;
}

__global__ void __launch_bounds__(1024) k_bab_tally(int P, const uint8_t* stuck, int* stat) {
    __shared__ int red[32];
    int n = 0;
    for (int i = threadIdx.x; i < P; i += blockDim.x) n += stuck[i] ? 1 : 0;
    n = block_sum(n, red);
    if (threadIdx.x == 0) stat[ST_STUCK] = n;
}

// One block over the n children (n = *nchild, or n_host when nchild is null): keep = not verified,
// not infeasible and below max_depth codes; exclusive positions of the kept ones and of their
// codes, in child order; the counts and the least spec lower bound of the kept ones.
__global__ void __launch_bounds__(1024) k_bab_filter(const int* nchild, int n_host, int m, int max_depth,
                                                     const int* c_off, const float* lower, const uint8_t* verified,
                                                     const uint8_t* infeasible, int* keep_pos, int* code_pos,
                                                     float* lmin, int* stat) {
    __shared__ int s_k[1024], s_c[1024], red[32];
    __shared__ float s_lm[32];
    const int n = nchild ? *nchild : n_host;
    const int tid = threadIdx.x, nt = blockDim.x;
    const int per = (n + nt - 1) / nt;
    int k = 0, cd = 0, nv = 0, ni = 0, nd = 0;
    float lm = INFINITY;
    for (int i = 0; i < per; ++i) {
        const int ch = tid * per + i;
        if (ch >= n) break;
        const int ns = c_off ? c_off[ch + 1] - c_off[ch] : 0;
        float v = INFINITY;
        for (int r = 0; r < m; ++r) v = fminf(v, lower[(size_t)ch * m + r]);
        lmin[ch] = v;
        const bool inf = infeasible[ch] != 0, ver = verified[ch] != 0;
        const bool kp = !inf && !ver && ns < max_depth;
        ni += inf;
        nv += ver && !inf;
        nd += !inf && !ver && !kp;
        if (kp) { ++k; cd += ns; lm = fminf(lm, v); }
    }
    s_k[tid] = k;
    s_c[tid] = cd;
    __syncthreads();
    for (int off = 1; off < nt; off <<= 1) {
        const int x = tid >= off ? s_k[tid - off] : 0;
        const int y = tid >= off ? s_c[tid - off] : 0;
        __syncthreads();
        s_k[tid] += x;
        s_c[tid] += y;
        __syncthreads();
    }
    int pk = s_k[tid] - k, pc = s_c[tid] - cd;
    for (int i = 0; i < per; ++i) {
        const int ch = tid * per + i;
        if (ch >= n) break;
        const int ns = c_off ? c_off[ch + 1] - c_off[ch] : 0;
        const bool kp = !infeasible[ch] && !verified[ch] && ns < max_depth;
        keep_pos[ch] = kp ? pk : -1;
        code_pos[ch] = pc;
        if (kp) { ++pk; pc += ns; }
    }
    const int tv = block_sum(nv, red), ti = block_sum(ni, red), td = block_sum(nd, red);
    // least lower bound of the kept children: warp minima, then one thread
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) lm = fminf(lm, __shfl_xor_sync(0xffffffffu, lm, o));
    if ((tid & 31) == 0) s_lm[tid >> 5] = lm;
    __syncthreads();
    if (tid == 0) {
        float f = INFINITY;
        for (int w = 0; w < (nt >> 5); ++w) f = fminf(f, s_lm[w]);
        stat[ST_VER] = tv;
        stat[ST_INF] = ti;
        stat[ST_DEPTH] = td;
        stat[ST_PUSHED] = s_k[nt - 1];
        stat[ST_CODES] = s_c[nt - 1];
        stat[ST_LMIN] = __float_as_int(f);
    }
}

struct Stack {
    int* off; int* ids; float* lo; float* hi; float* l; float* u; int8_t* mask; float* w; float* lmin;
};

// block per child: a kept child goes to stack position base + keep_pos, its codes after the codes
// of the domains below it
__global__ void k_bab_push(const int* nchild, int n_host, int n0, int U, int m, int base, const int* c_off,
                           const int* c_ids, const int* keep_pos, const int* code_pos, const float* lmin,
                           const float* lo, const float* hi, const float* l, const float* u, const int8_t* mask,
                           const float* w, Stack s) {
    const int ch = blockIdx.x;
    const int n = nchild ? *nchild : n_host;
    if (ch >= n) return;
    const int kp = keep_pos[ch];
    if (kp < 0) return;
    const int d = base + kp;
    const int c0 = c_off ? c_off[ch] : 0;
    const int ns = c_off ? c_off[ch + 1] - c0 : 0;
    const int s0 = s.off[base] + code_pos[ch];
    for (int q = threadIdx.x; q < ns; q += blockDim.x) s.ids[s0 + q] = c_ids[c0 + q];
    for (int i = threadIdx.x; i < n0; i += blockDim.x) {
        s.lo[(size_t)d * n0 + i] = lo[(size_t)ch * n0 + i];
        s.hi[(size_t)d * n0 + i] = hi[(size_t)ch * n0 + i];
    }
    for (int c = threadIdx.x; c < U; c += blockDim.x) {
        const size_t so = (size_t)d * U + c, co = (size_t)ch * U + c;
        s.l[so] = l[co];
        s.u[so] = u[co];
        s.mask[so] = mask[co];
        s.w[so] = w[co];
    }
    if (threadIdx.x == 0) {
        s.off[d + 1] = s0 + ns;
        s.lmin[d] = lmin[ch];
    }
}

}  // namespace

struct cv_bab {
    cv_net* net;
    const cv_cache* cache;
    int m, n0, U;
    const float* C;
    const float* t;
    cv_bab_params p;
    int count;               // domains on the stack
    std::vector<void*> allocs;
    Stack s;                 // capacity domains
    // children of one iteration (2 batch)
    int *c_off, *c_ids, *c_parent, *c_branched, *tgt_off, *tgt_ids, *keep_pos, *code_pos;
    float *c_lo, *c_hi, *c_l, *c_u, *c_w, *lmin;
    int8_t* c_mask;
    uint8_t *stuck, *zeros;
    // the round's outputs for 2 batch subdomains
    float *r_lower, *r_lo, *r_hi, *r_l, *r_u, *r_w;
    int8_t* r_mask;
    uint8_t *r_inf, *r_ver;
    void* ws_round; size_t ws_round_bytes;
    void* ws_split; size_t ws_split_bytes;
    void* ws_topk; size_t ws_topk_bytes;
    int* d_stat;
    int* h_stat;             // pinned mirror
};

namespace {

template <typename T>
cv_status bab_alloc(cv_bab* b, T** p, size_t n) {
    void* q = nullptr;
    const size_t bytes = cv_align256((n ? n : 1) * sizeof(T));
    if (cudaMalloc(&q, bytes) != cudaSuccess) {
        cv_set_error("cv_bab_create: cudaMalloc of " + std::to_string(bytes) + " bytes failed");
        return CV_ECUDA;
    }
    b->allocs.push_back(q);
    *p = (T*)q;
    return CV_OK;
}

void bab_free(cv_bab* b) {
    for (void* q : b->allocs) cudaFree(q);
    b->allocs.clear();
    if (b->h_stat) cudaFreeHost(b->h_stat);
    b->h_stat = nullptr;
}

cv_batch_in bab_round_in(const cv_bab* b, int B, const float* lo, const float* hi, bool children) {
    cv_batch_in in;
    memset(&in, 0, sizeof(in));
    in.B = B;
    in.lo = lo;
    in.hi = hi;
    in.m = b->m;
    in.C = b->C;
    in.t = b->t;
    if (children) {
        in.l_in = b->c_l;
        in.u_in = b->c_u;
        in.split_off = b->c_off;
        in.split_ids = b->c_ids;
        in.max_splits = b->p.max_depth;
        if (b->p.top_k >= 0) { in.tgt_off = b->tgt_off; in.tgt_ids = b->tgt_ids; }
    }
    return in;
}

cv_batch_out bab_round_out(const cv_bab* b) {
    cv_batch_out o;
    memset(&o, 0, sizeof(o));
    o.lower = b->r_lower; o.lo_clip = b->r_lo; o.hi_clip = b->r_hi; o.l = b->r_l; o.u = b->r_u;
    o.mask = b->r_mask; o.infeasible = b->r_inf; o.verified = b->r_ver; o.babsr_weight = b->r_w;
    return o;
}

// Domain_Filter of n bounded subdomains (device count nchild, or n_host) and the push from `base`
cv_status bab_filter_push(cv_bab* b, const int* nchild, int n_host, int nblocks, int base, const int* c_off,
                          const int* c_ids, cudaStream_t st) {
    k_bab_filter<<<1, 1024, 0, st>>>(nchild, n_host, b->m, b->p.max_depth, c_off, b->r_lower, b->r_ver, b->r_inf,
                                     b->keep_pos, b->code_pos, b->lmin, b->d_stat);
    CV_LAUNCH_CHECK("k_bab_filter");
    if (nblocks > 0) {
        k_bab_push<<<nblocks, 128, 0, st>>>(nchild, n_host, b->n0, b->U, b->m, base, c_off, c_ids, b->keep_pos,
                                            b->code_pos, b->lmin, b->r_lo, b->r_hi, b->r_l, b->r_u, b->r_mask,
                                            b->r_w, b->s);
        CV_LAUNCH_CHECK("k_bab_push");
    }
    CV_CUDA(cudaMemcpyAsync(b->h_stat, b->d_stat, ST_N * sizeof(int), cudaMemcpyDeviceToHost, st));
    CV_CUDA(cudaStreamSynchronize(st));
    return CV_OK;
}

void bab_fill_stats(const cv_bab* b, cv_bab_stats* o) {
    o->verified = b->h_stat[ST_VER];
    o->infeasible = b->h_stat[ST_INF];
    o->depth_limited = b->h_stat[ST_DEPTH];
    o->pushed = b->h_stat[ST_PUSHED];
    float f;
    memcpy(&f, &b->h_stat[ST_LMIN], sizeof(f));
    o->lower_min = f;
}

}  // namespace

extern "C" void cv_bab_params_default(cv_bab_params* p) {
    if (!p) return;
    p->batch = 1024;
    p->top_k = 20;
    p->capacity = 65536;
    p->max_depth = 32;
    cv_options_default(&p->opt);
    p->opt.sweeps = 10;
}

extern "C" cv_status cv_bab_create(cv_net* net, const cv_cache* cache, int m, const float* C, const float* t,
                                   const cv_bab_params* p, cv_bab** out) {
    if (!net || !cache || !C || !p || !out || cache->net != net) {
        cv_set_error("cv_bab_create: null argument or a cache of another network");
        return CV_EINVAL;
    }
    if (m < 1 || p->batch < 1 || p->max_depth < 1 || p->capacity < p->batch + 1 ||
        (long long)2 * p->batch * p->max_depth > INT_MAX / 2 || (long long)p->capacity * p->max_depth > INT_MAX) {
        cv_set_error("cv_bab_create: need m >= 1, batch >= 1, max_depth >= 1, capacity > batch (sizes within int)");
        return CV_EINVAL;
    }
    if (p->opt.sweeps > 0 && p->max_depth > 32) {
        cv_set_error("cv_bab_create: complete clipping takes at most 32 rows: max_depth <= 32 when sweeps > 0");
        return CV_EUNSUPPORTED;
    }
    *out = nullptr;
    cv_bab* b = new cv_bab();
    memset(&b->s, 0, sizeof(b->s));
    b->net = net; b->cache = cache; b->m = m; b->C = C; b->t = t; b->p = *p;
    b->p.opt.babsr_weight = 1;
    b->n0 = net->dims[0];
    b->U = cache->U;
    b->count = 0;
    b->h_stat = nullptr;
    const size_t D = (size_t)p->capacity, n0 = (size_t)b->n0, U = (size_t)(b->U > 0 ? b->U : 1);
    const size_t B2 = (size_t)2 * p->batch, mx = (size_t)p->max_depth;
    cv_status s = CV_OK;
    auto take = [&](auto** q, size_t n) { if (!s) s = bab_alloc(b, q, n); };
    take(&b->s.off, D + 1); take(&b->s.ids, D * mx); take(&b->s.lo, D * n0); take(&b->s.hi, D * n0);
    take(&b->s.l, D * U); take(&b->s.u, D * U); take(&b->s.mask, D * U); take(&b->s.w, D * U);
    take(&b->s.lmin, D);
    take(&b->c_off, B2 + 1); take(&b->c_ids, B2 * mx); take(&b->c_parent, B2); take(&b->c_branched, B2);
    take(&b->tgt_off, B2 + 1); take(&b->tgt_ids, B2 * U); take(&b->keep_pos, B2); take(&b->code_pos, B2);
    take(&b->c_lo, B2 * n0); take(&b->c_hi, B2 * n0); take(&b->c_l, B2 * U); take(&b->c_u, B2 * U);
    take(&b->c_w, B2 * U); take(&b->lmin, B2); take(&b->c_mask, B2 * U);
    take(&b->stuck, (size_t)p->batch); take(&b->zeros, (size_t)p->batch);
    take(&b->r_lower, B2 * m); take(&b->r_lo, B2 * n0); take(&b->r_hi, B2 * n0); take(&b->r_l, B2 * U);
    take(&b->r_u, B2 * U); take(&b->r_w, B2 * U); take(&b->r_mask, B2 * U); take(&b->r_inf, B2);
    take(&b->r_ver, B2); take(&b->d_stat, (size_t)ST_N);
    if (!s) {
        cv_batch_in in = bab_round_in(b, (int)B2, b->c_lo, b->c_hi, true);
        in.tgt_off = b->tgt_off; in.tgt_ids = b->tgt_ids;
        s = cv_bound_batch_workspace(net, cache, &in, &b->p.opt, &b->ws_round_bytes);
    }
    if (!s) s = cv_activation_split_workspace(p->batch, &b->ws_split_bytes);
    if (!s && b->U > 0) s = cv_select_targets_workspace((int)B2, b->U, &b->ws_topk_bytes);
    unsigned char* wr = nullptr; unsigned char* wsp = nullptr; unsigned char* wt = nullptr;
    take(&wr, b->ws_round_bytes); take(&wsp, b->ws_split_bytes); take(&wt, b->ws_topk_bytes);
    if (!s && cudaMallocHost((void**)&b->h_stat, ST_N * sizeof(int)) != cudaSuccess) {
        cv_set_error("cv_bab_create: cudaMallocHost failed");
        s = CV_ECUDA;
    }
    if (!s && (cudaMemset(b->zeros, 0, p->batch) != cudaSuccess || cudaMemset(b->s.off, 0, sizeof(int)) != cudaSuccess)) {
        cv_set_error("cv_bab_create: cudaMemset failed");
        s = CV_ECUDA;
    }
    if (s) { bab_free(b); delete b; return s; }
    b->ws_round = wr; b->ws_split = wsp; b->ws_topk = wt;
    *out = b;
    return CV_OK;
}

extern "C" void cv_bab_destroy(cv_bab* b) {
    if (!b) return;
    bab_free(b);
    delete b;
}

extern "C" cv_status cv_bab_init(cv_bab* b, int B0, const float* lo, const float* hi, void* stream,
                                 cv_bab_stats* stats) {
    if (!b || !lo || !hi || B0 < 1 || B0 > 2 * b->p.batch || B0 > b->p.capacity) {
        cv_set_error("cv_bab_init: null argument or B0 outside [1, min(2 batch, capacity)]");
        return CV_EINVAL;
    }
    cudaStream_t st = (cudaStream_t)stream;
    cv_batch_in in = bab_round_in(b, B0, lo, hi, false);
    cv_batch_out o = bab_round_out(b);
    cv_status s = cv_bound_batch(b->net, b->cache, &in, &o, &b->p.opt, b->ws_round, b->ws_round_bytes, stream);
    if (s) return s;
    CV_CUDA(cudaMemsetAsync(b->s.off, 0, sizeof(int), st));
    if ((s = bab_filter_push(b, nullptr, B0, B0, 0, nullptr, nullptr, st))) return s;
    b->count = b->h_stat[ST_PUSHED];
    if (stats) {
        memset(stats, 0, sizeof(*stats));
        stats->children = B0;
        bab_fill_stats(b, stats);
        stats->remaining = b->count;
    }
    return CV_OK;
}

extern "C" cv_status cv_bab_step(cv_bab* b, void* stream, cv_bab_stats* stats) {
    if (!b) { cv_set_error("cv_bab_step: null object"); return CV_EINVAL; }
    cudaStream_t st = (cudaStream_t)stream;
    cv_bab_stats o;
    memset(&o, 0, sizeof(o));
    o.lower_min = INFINITY;
    // Batch_Pick_Out: the top P domains; P also leaves room for two children each
    int P = b->count < b->p.batch ? b->count : b->p.batch;
    if (P > b->p.capacity - b->count) P = b->p.capacity - b->count;
    if (b->count == 0) {
        if (stats) *stats = o;
        return CV_OK;
    }
    if (P <= 0) { cv_set_error("cv_bab_step: the domain list is full"); return CV_EWORKSPACE; }
    const int base = b->count - P;
    const size_t n0 = (size_t)b->n0, U = (size_t)b->U;
    o.picked = P;
    if (b->U == 0) {  // nothing to branch on: every picked domain is stuck
        o.stuck = P;
        b->count = base;
        o.remaining = b->count;
        if (stats) *stats = o;
        return CV_OK;
    }
    // Batch_Split with the BaBSR score (the stored weight); offsets of the picked parents are absolute
    cv_status s = cv_activation_split(b->net, b->cache, P, b->s.off + base, b->s.ids, b->s.lo + base * n0,
                                      b->s.hi + base * n0, b->s.l + base * U, b->s.u + base * U,
                                      b->s.mask + base * U, b->s.w + base * U, b->zeros, b->zeros, b->c_off,
                                      b->c_ids, b->c_lo, b->c_hi, b->c_l, b->c_u, b->c_parent, b->c_branched,
                                      b->stuck, b->d_stat + ST_NCHILD, b->ws_split, b->ws_split_bytes, stream);
    if (s) return s;
    k_bab_inherit<<<2 * P, 128, 0, st>>>(b->U, b->d_stat + ST_NCHILD, base, b->c_parent, b->c_branched, b->s.mask,
                                         b->s.w, b->c_mask, b->c_w);
    CV_LAUNCH_CHECK("k_bab_inherit");
    k_bab_tally<<<1, 1024, 0, st>>>(P, b->stuck, b->d_stat);
    CV_LAUNCH_CHECK("k_bab_tally");
    CV_CUDA(cudaMemcpyAsync(b->h_stat, b->d_stat, 2 * sizeof(int), cudaMemcpyDeviceToHost, st));
    CV_CUDA(cudaStreamSynchronize(st));
    const int nch = b->h_stat[ST_NCHILD];
    o.stuck = b->h_stat[ST_STUCK];
    o.children = nch;
    if (nch > 0) {
        // Top-K_Heuristic on the children
        if (b->p.top_k >= 0) {
            s = cv_select_targets(b->net, b->cache, nch, b->c_l, b->c_u, b->c_mask, b->c_w, b->p.top_k, b->tgt_off,
                                  b->tgt_ids, b->ws_topk, b->ws_topk_bytes, stream);
            if (s) return s;
        }
        // Domain_Clipper, Domain_Update and Solve_Bound: one round on the children
        cv_batch_in in = bab_round_in(b, nch, b->c_lo, b->c_hi, true);
        cv_batch_out out = bab_round_out(b);
        s = cv_bound_batch(b->net, b->cache, &in, &out, &b->p.opt, b->ws_round, b->ws_round_bytes, stream);
        if (s) return s;
        // Domain_Filter, and the survivors back onto the stack from the first picked position
        if ((s = bab_filter_push(b, nullptr, nch, nch, base, b->c_off, b->c_ids, st))) return s;
        bab_fill_stats(b, &o);
    }
    b->count = base + o.pushed;
    o.remaining = b->count;
    if (stats) *stats = o;
    return CV_OK;
}

extern "C" cv_status cv_bab_run(cv_bab* b, int max_iters, void* stream, cv_bab_stats* total, int* iters) {
    if (!b || max_iters < 0) { cv_set_error("cv_bab_run: null object or negative max_iters"); return CV_EINVAL; }
    cv_bab_stats t;
    memset(&t, 0, sizeof(t));
    t.lower_min = INFINITY;
    t.remaining = b->count;
    int it = 0;
    cv_status s = CV_OK;
    while (it < max_iters && b->count > 0) {
        cv_bab_stats o;
        if ((s = cv_bab_step(b, stream, &o))) break;
        ++it;
        t.picked += o.picked; t.stuck += o.stuck; t.children += o.children; t.verified += o.verified;
        t.infeasible += o.infeasible; t.depth_limited += o.depth_limited; t.pushed += o.pushed;
        t.remaining = o.remaining;
        t.lower_min = o.lower_min;
    }
    if (total) *total = t;
    if (iters) *iters = it;
    return s;
}

extern "C" cv_status cv_bab_read(const cv_bab* b, int* count, int* split_off, int* split_ids, float* lower_min,
                                 void* stream) {
    if (!b) { cv_set_error("cv_bab_read: null object"); return CV_EINVAL; }
    cudaStream_t st = (cudaStream_t)stream;
    const int n = b->count;
    if (count) *count = n;
    std::vector<int> off((size_t)n + 1);
    CV_CUDA(cudaMemcpyAsync(off.data(), b->s.off, ((size_t)n + 1) * sizeof(int), cudaMemcpyDeviceToHost, st));
    CV_CUDA(cudaStreamSynchronize(st));
    if (split_off) memcpy(split_off, off.data(), ((size_t)n + 1) * sizeof(int));
    if (split_ids && off[n] > 0)
        CV_CUDA(cudaMemcpyAsync(split_ids, b->s.ids, (size_t)off[n] * sizeof(int), cudaMemcpyDeviceToHost, st));
    if (lower_min && n > 0)
        CV_CUDA(cudaMemcpyAsync(lower_min, b->s.lmin, (size_t)n * sizeof(float), cudaMemcpyDeviceToHost, st));
    CV_CUDA(cudaStreamSynchronize(st));
    return CV_OK;
}
