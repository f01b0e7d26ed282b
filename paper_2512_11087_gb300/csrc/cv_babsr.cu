// Activation branch and bound with the BaBSR intercept score (Appendix, neuron selection heuristic;
// Algorithm 5: Domain_Filter, Batch_Split on one ReLU, Top-K_Heuristic for complete clipping).
//
// Score of cached neuron c of a subdomain: -1 unless it is unstable (mask 0, l < 0 < u), else
//   max(0, -l) * max(0, u) / (u - l) * w,   w = max(0, -weight) (1 without weights)
// -- the intercept of the ReLU's upper line times the neuron's weight in the bound -- in FP32 with
// explicitly rounded operations in this order, so that every decision matches the oracle's.
//
// cv_activation_split (three launches): k_act_mark (block per parent: keep, best slot), a one-block
// scan (children and split-list positions), k_act_write (block per parent: two children's split
// lists, boxes and cached bounds).  cv_select_targets (three launches): k_topk_mark (block per
// subdomain: scores in shared memory, the unstable slots compacted in slot order so that every
// layer's are contiguous, each ranked among its layer's), a one-block scan, k_topk_write (ordered
// compaction into the CSR).  The ranking gives each unstable slot a warp, whose lanes compare it
// with 32 slots of its layer at a time.  The split streams the per-subdomain arrays once: HBM-bound.
#include "cv_internal.cuh"

#include <string>

namespace {

__device__ __forceinline__ float babsr_score(float l, float u, int8_t mask, const float* weight, size_t o) {
    if (mask != 0 || !(l < 0.f) || !(u > 0.f)) return -1.f;
    const float p = __fmul_rn(fmaxf(0.f, -l), fmaxf(0.f, u));
    float s = __fdiv_rn(p, __fsub_rn(u, l));
    if (weight) s = __fmul_rn(s, fmaxf(0.f, -weight[o]));
    return s;
}

// (s, i) outranks (t, j): a higher score, or an equal one and a lower slot
__device__ __forceinline__ bool outranks(float s, int i, float t, int j) { return s > t || (s == t && i < j); }

// one-block exclusive scan of two per-item counts; totals into t0, t1 (either may be null)
__global__ void __launch_bounds__(1024) k_scan2(int B, const int* c0, const int* c1, int* p0, int* p1, int* t0,
                                                int* t1) {
    __shared__ int s0[1024], s1[1024];
    const int tid = threadIdx.x, nt = blockDim.x;
    const int per = (B + nt - 1) / nt;
    int a = 0, z = 0;
    for (int i = 0; i < per; ++i) {
        const int b = tid * per + i;
        if (b < B) { a += c0[b]; z += c1 ? c1[b] : 0; }
    }
    s0[tid] = a;
    s1[tid] = z;
    __syncthreads();
    for (int off = 1; off < nt; off <<= 1) {
        const int x = tid >= off ? s0[tid - off] : 0;
        const int y = tid >= off ? s1[tid - off] : 0;
        __syncthreads();
        s0[tid] += x;
        s1[tid] += y;
        __syncthreads();
    }
    int q0 = s0[tid] - a, q1 = s1[tid] - z;
    for (int i = 0; i < per; ++i) {
        const int b = tid * per + i;
        if (b < B) {
            p0[b] = q0;
            if (p1) p1[b] = q1;
            q0 += c0[b];
            q1 += c1 ? c1[b] : 0;
        }
    }
    if (tid == 0) {
        if (t0) *t0 = s0[nt - 1];
        if (t1) *t1 = s1[nt - 1];
    }
}

// ---------------------------------------------------------------- split step
struct ActWs {
    int* kept;    // [B] 2 for a kept parent (its children), else 0
    int* codes;   // [B] split codes the parent's children hold together: 2 (parent's + 1)
    int* best;    // [B] branching slot
    int* cpos;    // [B] first child
    int* spos;    // [B] first split code of the first child
};

__global__ void k_act_mark(int B, int U, const int* split_off, const float* l, const float* u, const int8_t* mask,
                           const float* weight, const uint8_t* verified, const uint8_t* infeasible, uint8_t* stuck,
                           ActWs w) {
    const int b = blockIdx.x;
    __shared__ float rs[32];
    __shared__ int ri[32];
    const bool keep = !verified[b] && !infeasible[b];
    float bs = -1.f;
    int bi = 0x7fffffff;
    if (keep) {
        for (int c = threadIdx.x; c < U; c += blockDim.x) {
            const size_t o = (size_t)b * U + c;
            const float sc = babsr_score(l[o], u[o], mask[o], weight, o);
            if (sc > bs) { bs = sc; bi = c; }  // increasing slot: the first maximum (-1 never wins)
        }
    }
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
        const float os = __shfl_xor_sync(0xffffffffu, bs, off);
        const int oi = __shfl_xor_sync(0xffffffffu, bi, off);
        if (outranks(os, oi, bs, bi)) { bs = os; bi = oi; }
    }
    if (lane == 0) { rs[warp] = bs; ri[warp] = bi; }
    __syncthreads();
    if (threadIdx.x == 0) {
        float fs = -1.f;
        int fi = 0x7fffffff;
        for (int q = 0; q < nw; ++q)
            if (outranks(rs[q], ri[q], fs, fi)) { fs = rs[q]; fi = ri[q]; }
        const bool branch = keep && fi != 0x7fffffff && fs >= 0.f;
        const int ns = split_off ? split_off[b + 1] - split_off[b] : 0;
        stuck[b] = (keep && !branch) ? 1 : 0;
        w.kept[b] = branch ? 2 : 0;
        w.codes[b] = branch ? 2 * (ns + 1) : 0;
        w.best[b] = branch ? fi : -1;
    }
}

__global__ void k_act_write(int B, int U, int n0, const int* ids, const int* split_off, const int* split_ids,
                            const float* lo, const float* hi, const float* l, const float* u, ActWs w,
                            int* split_off_out, int* split_ids_out, float* lo_out, float* hi_out, float* l_out,
                            float* u_out, int* parent, int* branched) {
    const int b = blockIdx.x;
    if (!w.kept[b]) return;
    const int best = w.best[b], ch0 = w.cpos[b], sp = w.spos[b];
    const int k0 = split_off ? split_off[b] : 0;
    const int ns = split_off ? split_off[b + 1] - k0 : 0;
    const int code = ids[best] + 1;
    for (int side = 0; side < 2; ++side) {
        const int ch = ch0 + side;
        const int s0 = sp + side * (ns + 1);
        for (int q = threadIdx.x; q < ns; q += blockDim.x) split_ids_out[s0 + q] = split_ids[k0 + q];
        for (int i = threadIdx.x; i < n0; i += blockDim.x) {
            lo_out[(size_t)ch * n0 + i] = lo[(size_t)b * n0 + i];
            hi_out[(size_t)ch * n0 + i] = hi[(size_t)b * n0 + i];
        }
        for (int c = threadIdx.x; c < U; c += blockDim.x) {
            l_out[(size_t)ch * U + c] = l[(size_t)b * U + c];
            u_out[(size_t)ch * U + c] = u[(size_t)b * U + c];
        }
        if (threadIdx.x == 0) {
            split_ids_out[s0 + ns] = side ? code : -code;  // child 2k: z <= 0; child 2k+1: z >= 0
            split_off_out[ch + 1] = s0 + ns + 1;
            parent[ch] = b;
            branched[ch] = best;
        }
    }
}

// ---------------------------------------------------------------- top-k targets
struct NetLayers { int L1; int hoff[CV_MAX_LAYERS + 1]; };  // hidden layers 1..L1; hoff[L1] = H

__device__ __forceinline__ int layer_of(const NetLayers& nl, int g) {
    int i = 1;
    while (i < nl.L1 && g >= nl.hoff[i]) ++i;
    return i;
}

// block per subdomain; dynamic shared memory: scores [U] floats, then the unstable slots in order
// [U] ints and their layers [U] ints
__global__ void k_topk_mark(int U, int k, NetLayers nl, const int* ids, const float* l, const float* u,
                            const int8_t* mask, const float* weight, uint8_t* sel, int* count) {
    extern __shared__ float tk_smem[];
    float* sc = tk_smem;
    int* lst = (int*)(sc + U);
    int* lay = lst + U;
    __shared__ int s_n, s_wn[32], s_cnt;
    const int b = blockIdx.x;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    if (threadIdx.x == 0) { s_n = 0; s_cnt = 0; }
    __syncthreads();
    // scores, and the unstable slots compacted in slot order (a block-wide ordered ballot per chunk)
    for (int base = 0; base < U; base += blockDim.x) {
        const int c = base + threadIdx.x;
        float s = -1.f;
        if (c < U) {
            const size_t o = (size_t)b * U + c;
            s = babsr_score(l[o], u[o], mask[o], weight, o);
            sc[c] = s;
            sel[o] = 0;
        }
        const bool un = c < U && s >= 0.f;
        const unsigned bal = __ballot_sync(0xffffffffu, un);
        if (lane == 0) s_wn[warp] = __popc(bal);
        __syncthreads();
        int pos = s_n + __popc(bal & ((1u << lane) - 1u));
        for (int q = 0; q < warp; ++q) pos += s_wn[q];
        if (un) { lst[pos] = c; lay[pos] = layer_of(nl, ids[c]); }
        __syncthreads();
        if (threadIdx.x == 0)
            for (int q = 0; q < nw; ++q) s_n += s_wn[q];
        __syncthreads();
    }
    const int n = s_n;
    // first and last list position of every layer (the list follows the slots, so the layers)
    __shared__ int s_first[CV_MAX_LAYERS + 1], s_last[CV_MAX_LAYERS + 1];
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
        const int li = lay[i];
        if (i == 0 || lay[i - 1] != li) s_first[li] = i;
        if (i == n - 1 || lay[i + 1] != li) s_last[li] = i;
    }
    __syncthreads();
    // a warp per unstable slot: its lanes count the slots of the same layer that outrank it, 32 at a
    // time, until k are found
    int mine = 0;
    for (int i = warp; i < n; i += nw) {
        const int c = lst[i], li = lay[i];
        const float s = sc[c];
        const int a = s_first[li], z = s_last[li];
        int rank = 0;
        for (int j0 = a; j0 <= z && rank < k; j0 += 32) {
            const int j = j0 + lane;
            const bool o = j <= z && j != i && outranks(sc[lst[j]], lst[j], s, c);
            rank += __popc(__ballot_sync(0xffffffffu, o));
        }
        if (rank < k && lane == 0) { sel[(size_t)b * U + c] = 1; ++mine; }
    }
    atomicAdd(&s_cnt, mine);
    __syncthreads();
    if (threadIdx.x == 0) count[b] = s_cnt;
}

__global__ void k_topk_write(int U, const uint8_t* sel, const int* off, int* tgt_ids) {
    __shared__ int s_n, s_wn[32];
    const int b = blockIdx.x;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    if (threadIdx.x == 0) s_n = 0;
    __syncthreads();
    for (int base = 0; base < U; base += blockDim.x) {
        const int c = base + threadIdx.x;
        const bool on = c < U && sel[(size_t)b * U + c];
        const unsigned bal = __ballot_sync(0xffffffffu, on);
        if (lane == 0) s_wn[warp] = __popc(bal);
        __syncthreads();
        int pos = s_n + __popc(bal & ((1u << lane) - 1u));
        for (int q = 0; q < warp; ++q) pos += s_wn[q];
        if (on) tgt_ids[off[b] + pos] = c;
        __syncthreads();
        if (threadIdx.x == 0)
            for (int q = 0; q < nw; ++q) s_n += s_wn[q];
        __syncthreads();
    }
}

size_t act_ws_bytes(int B) { return 5 * cv_align256((size_t)(B > 0 ? B : 1) * sizeof(int)); }
size_t topk_ws_bytes(int B, int U) {
    return cv_align256((size_t)(B > 0 ? B : 1) * (U > 0 ? U : 1)) + cv_align256((size_t)(B > 0 ? B : 1) * sizeof(int));
}

}  // namespace

extern "C" cv_status cv_activation_split_workspace(int B, size_t* bytes) {
    if (B < 0 || !bytes) { cv_set_error("cv_activation_split_workspace: negative B or null bytes"); return CV_EINVAL; }
    *bytes = act_ws_bytes(B);
    return CV_OK;
}

extern "C" cv_status cv_activation_split(const cv_net* net, const cv_cache* cache, int B, const int* split_off,
                                         const int* split_ids, const float* lo, const float* hi, const float* l,
                                         const float* u, const int8_t* mask, const float* weight,
                                         const uint8_t* verified, const uint8_t* infeasible, int* split_off_out,
                                         int* split_ids_out, float* lo_out, float* hi_out, float* l_out,
                                         float* u_out, int* parent, int* branched, uint8_t* stuck, int* n_children,
                                         void* workspace, size_t workspace_bytes, void* stream) {
    if (!net || !cache || cache->net != net) { cv_set_error("cv_activation_split: bad net or cache"); return CV_EINVAL; }
    if (B < 0) { cv_set_error("cv_activation_split: B < 0"); return CV_EINVAL; }
    if (!split_off_out || !n_children) { cv_set_error("cv_activation_split: null split_off_out or n_children"); return CV_EINVAL; }
    cudaStream_t st = (cudaStream_t)stream;
    if (B == 0) {
        CV_CUDA(cudaMemsetAsync(split_off_out, 0, sizeof(int), st));
        CV_CUDA(cudaMemsetAsync(n_children, 0, sizeof(int), st));
        return CV_OK;
    }
    const int U = cache->U, n0 = cache->n0;
    if (U < 1 || !lo || !hi || !l || !u || !mask || !verified || !infeasible || !split_ids_out || !lo_out ||
        !hi_out || !l_out || !u_out || !parent || !branched || !stuck || !workspace || (split_off && !split_ids)) {
        cv_set_error("cv_activation_split: null argument or a cache without unstable neurons");
        return CV_EINVAL;
    }
    if (workspace_bytes < act_ws_bytes(B)) {
        cv_set_error("cv_activation_split: workspace smaller than cv_activation_split_workspace()");
        return CV_EWORKSPACE;
    }
    ActWs w;
    char* p = (char*)workspace;
    const size_t step = cv_align256((size_t)B * sizeof(int));
    w.kept = (int*)p; p += step;
    w.codes = (int*)p; p += step;
    w.best = (int*)p; p += step;
    w.cpos = (int*)p; p += step;
    w.spos = (int*)p;
    k_act_mark<<<B, 256, 0, st>>>(B, U, split_off, l, u, mask, weight, verified, infeasible, stuck, w);
    CV_LAUNCH_CHECK("k_act_mark");
    k_scan2<<<1, 1024, 0, st>>>(B, w.kept, w.codes, w.cpos, w.spos, n_children, nullptr);
    CV_LAUNCH_CHECK("k_scan2");
    CV_CUDA(cudaMemsetAsync(split_off_out, 0, sizeof(int), st));
    k_act_write<<<B, 256, 0, st>>>(B, U, n0, cache->ids, split_off, split_ids, lo, hi, l, u, w, split_off_out,
                                   split_ids_out, lo_out, hi_out, l_out, u_out, parent, branched);
    CV_LAUNCH_CHECK("k_act_write");
    return CV_OK;
}

extern "C" cv_status cv_select_targets_workspace(int B, int U, size_t* bytes) {
    if (B < 0 || U < 0 || !bytes) { cv_set_error("cv_select_targets_workspace: bad argument"); return CV_EINVAL; }
    *bytes = topk_ws_bytes(B, U);
    return CV_OK;
}

extern "C" cv_status cv_select_targets(const cv_net* net, const cv_cache* cache, int B, const float* l,
                                       const float* u, const int8_t* mask, const float* weight, int k, int* tgt_off,
                                       int* tgt_ids, void* workspace, size_t workspace_bytes, void* stream) {
    if (!net || !cache || cache->net != net) { cv_set_error("cv_select_targets: bad net or cache"); return CV_EINVAL; }
    if (B < 0 || k < 0) { cv_set_error("cv_select_targets: B < 0 or k < 0"); return CV_EINVAL; }
    if (!tgt_off) { cv_set_error("cv_select_targets: null tgt_off"); return CV_EINVAL; }
    cudaStream_t st = (cudaStream_t)stream;
    const int U = cache->U;
    if (B == 0 || U == 0) {
        CV_CUDA(cudaMemsetAsync(tgt_off, 0, sizeof(int) * (size_t)(B + 1), st));
        return CV_OK;
    }
    if (!l || !u || !mask || !tgt_ids || !workspace) { cv_set_error("cv_select_targets: null argument"); return CV_EINVAL; }
    if (workspace_bytes < topk_ws_bytes(B, U)) {
        cv_set_error("cv_select_targets: workspace smaller than cv_select_targets_workspace()");
        return CV_EWORKSPACE;
    }
    const size_t smem = (size_t)U * (4 + 4 + 4);
    if (smem > 200 * 1024) { cv_set_error("cv_select_targets: more than 17066 cached neurons"); return CV_EUNSUPPORTED; }
    NetLayers nl;
    nl.L1 = net->L - 1;
    int acc = 0;
    for (int i = 1; i <= nl.L1 && i <= CV_MAX_LAYERS; ++i) { nl.hoff[i] = acc + net->dims[i]; acc += net->dims[i]; }
    // hoff[i] here: first global id after hidden layer i (ids below it belong to layers <= i)
    uint8_t* sel = (uint8_t*)workspace;
    int* count = (int*)((char*)workspace + cv_align256((size_t)B * U));
    CV_CUDA(cudaFuncSetAttribute(k_topk_mark, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    k_topk_mark<<<B, 256, smem, st>>>(U, k, nl, cache->ids, l, u, mask, weight, sel, count);
    CV_LAUNCH_CHECK("k_topk_mark");
    k_scan2<<<1, 1024, 0, st>>>(B, count, nullptr, tgt_off, nullptr, tgt_off + B, nullptr);
    CV_LAUNCH_CHECK("k_scan2");
    k_topk_write<<<B, 256, 0, st>>>(U, sel, tgt_off, tgt_ids);
    CV_LAUNCH_CHECK("k_topk_write");
    return CV_OK;
}
