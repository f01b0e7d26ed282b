// C-ABI entry points of one bounding round (cv_bound_batch and its helpers): argument
// validation, workspace layout, and the launch sequence a2..a8 on the caller's stream.
#include "cv_internal.cuh"

#include <climits>
#include <string.h>

#include <string>


static thread_local std::string g_err;

void cv_set_error(const std::string& msg) { g_err = msg; }

cv_status cv_cuda_fail(cudaError_t e, const char* what) {
    g_err = std::string(what) + ": " + cudaGetErrorString(e);
    return e == cudaErrorMemoryAllocation ? CV_ENOMEM : CV_ECUDA;
}

extern "C" const char* cv_last_error(void) { return g_err.c_str(); }

extern "C" void cv_options_default(cv_options* o) {
    if (!o) return;
    o->relaxed = 1;
    o->sweeps = 0;
    o->precision = CV_PREC_FP32;
    o->alpha_mode = CV_ALPHA_ADAPTIVE;
    o->enforce_splits = 1;
    o->timer = nullptr;
    o->babsr_weight = 0;
}

cv_status cv_ws_plan(const cv_net* net, const cv_cache* cache, int B, int m, int max_splits,
                     int max_rows, int precision, cv_ws_layout* lay, int babsr_weight) {
    memset(lay, 0, sizeof(*lay));
    lay->Rmax = max_splits + max_rows;
    lay->R = B * m;
    lay->ncb = cv_bwd_ncb_max(net);
    const size_t R = (size_t)lay->R, Rm = (size_t)B * lay->Rmax, ncb = lay->ncb;
    size_t off = 0;
    auto take = [&](size_t bytes) { size_t o = off; off = cv_align256(off + (bytes ? bytes : 1)); return o; };
    lay->rowflag = take(Rm);
    lay->vmin = take(Rm * sizeof(double));
    lay->rowdesc = take((size_t)2 * (cache->U > 0 ? cache->U : 1) * sizeof(float));
    lay->lam0 = take(R * net->wmax * sizeof(float));
    lay->lam1 = take(R * net->wmax * sizeof(float));
    lay->part_bias = take(R * ncb * sizeof(double));
    lay->part_pad = take(R * ncb * sizeof(double));
    lay->part_f = take(R * ncb * sizeof(double));
    lay->part_fmag = take(R * ncb * sizeof(double));
    lay->acc_bias = take(R * sizeof(double));
    lay->acc_pad = take(R * sizeof(double));
    lay->cc = take(cv_cc_workspace(B, lay->Rmax, net->dims[0]));
    if (precision == CV_PREC_BF16X8) {
        lay->tc_slices = take(cv_tc_slices_bytes(net, lay->R));
        lay->tc_exp = take(R * sizeof(int));
        lay->tc_tab = take((size_t)3 * B * net->wmax * sizeof(float));
        lay->tc_box = take(cv_tc_box_bytes(cache, B));
        lay->tc_bexp = take((size_t)B * sizeof(int));
        lay->tc_bsum = take((size_t)B * sizeof(float));
    }
    if (babsr_weight && m > 0 && cache->U > 0) lay->pbuf = take(R * net->wmax * sizeof(float));
    lay->total = off;
    return CV_OK;
}

static cv_status validate(const cv_net* net, const cv_cache* cache, const cv_batch_in* in, const cv_options* opt,
                          bool pointers = true) {
    if (!net || !cache || !in || !opt) { cv_set_error("null net / cache / input / options"); return CV_EINVAL; }
    if (cache->net != net) { cv_set_error("cache was built for another network"); return CV_EINVAL; }
    if (in->B < 0 || in->m < 0 || in->max_splits < 0 || in->max_rows < 0) {
        cv_set_error("negative B, m, max_splits or max_rows");
        return CV_EINVAL;
    }
    // sizes the kernels index with 32-bit integers
    if ((long long)in->max_splits + in->max_rows > INT_MAX || (long long)in->B * in->m > INT_MAX ||
        (long long)in->B * ((long long)in->max_splits + in->max_rows) > INT_MAX) {
        cv_set_error("B, m, max_splits + max_rows too large (B x m and B x (max_splits + max_rows) must fit in int)");
        return CV_EINVAL;
    }
    if (opt->relaxed < CV_RELAX_OFF || opt->relaxed > CV_RELAX_SEQUENTIAL_ORDERED || opt->sweeps < 0 ||
        opt->alpha_mode < 0 || opt->alpha_mode > 2 ||
        (opt->precision != CV_PREC_FP32 && opt->precision != CV_PREC_BF16X8) ||
        (opt->babsr_weight != 0 && opt->babsr_weight != 1)) {
        cv_set_error("bad options");
        return CV_EINVAL;
    }
    if (!pointers) return CV_OK;
    if (in->B > 0 && (!in->lo || !in->hi)) { cv_set_error("lo/hi required"); return CV_EINVAL; }
    if (in->m > 0 && !in->C) { cv_set_error("C required when m > 0"); return CV_EINVAL; }
    if (!in->split_off && in->split_ids) { cv_set_error("split_ids without split_off"); return CV_EINVAL; }
    if (in->split_off && !in->split_ids && in->max_splits > 0) { cv_set_error("split_ids required when max_splits > 0"); return CV_EINVAL; }
    if (in->row_off && (!in->G || !in->h) && in->max_rows > 0) { cv_set_error("row_off needs G and h"); return CV_EINVAL; }
    if ((in->tgt_off == nullptr) != (in->tgt_ids == nullptr)) { cv_set_error("tgt_off and tgt_ids go together"); return CV_EINVAL; }
    if ((in->l_in == nullptr) != (in->u_in == nullptr)) { cv_set_error("l_in and u_in go together"); return CV_EINVAL; }
    if (!in->split_off && in->max_splits > 0) { cv_set_error("max_splits > 0 without splits"); return CV_EINVAL; }
    if (!in->row_off && in->max_rows > 0) { cv_set_error("max_rows > 0 without rows"); return CV_EINVAL; }
    return CV_OK;
}

extern "C" cv_status cv_bound_batch_workspace(const cv_net* net, const cv_cache* cache, const cv_batch_in* in,
                                              const cv_options* opt, size_t* bytes) {
    cv_status s = validate(net, cache, in, opt, false);
    if (s) return s;
    if (!bytes) { cv_set_error("null bytes"); return CV_EINVAL; }
    cv_ws_layout lay;
    cv_ws_plan(net, cache, in->B, in->m, in->max_splits, in->max_rows, opt->precision, &lay, opt->babsr_weight);
    *bytes = lay.total;
    return CV_OK;
}

namespace {
__global__ void k_verified(int B, int m, const float* lower, const uint8_t* infeasible, uint8_t* verified) {
    int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= B) return;
    bool v = infeasible[b] != 0;
    if (!v) {
        v = true;
        for (int r = 0; r < m; ++r) v = v && (lower[(size_t)b * m + r] > 0.f);
    }
    verified[b] = v ? 1 : 0;
}
// one block: the least spec lower bound over the feasible subdomains and over the unverified ones,
// and the verified / infeasible counts (an ordered tree of minima: the result is exact)
__global__ void __launch_bounds__(1024) k_round_summary(int B, int m, const float* lower, const uint8_t* verified,
                                                        const uint8_t* infeasible, float* bounds, int* counts) {
    __shared__ float s0[32], s1[32];
    __shared__ int c0[32], c1[32];
    float a = INFINITY, z = INFINITY;
    int nv = 0, ni = 0;
    for (int b = threadIdx.x; b < B; b += blockDim.x) {
        if (infeasible[b]) { ++ni; continue; }
        float v = INFINITY;
        for (int r = 0; r < m; ++r) v = fminf(v, lower[(size_t)b * m + r]);
        a = fminf(a, v);
        if (verified[b]) ++nv;
        else z = fminf(z, v);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        a = fminf(a, __shfl_xor_sync(0xffffffffu, a, o));
        z = fminf(z, __shfl_xor_sync(0xffffffffu, z, o));
        nv += __shfl_xor_sync(0xffffffffu, nv, o);
        ni += __shfl_xor_sync(0xffffffffu, ni, o);
    }
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (lane == 0) { s0[warp] = a; s1[warp] = z; c0[warp] = nv; c1[warp] = ni; }
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int w = 1; w < (int)(blockDim.x >> 5); ++w) {
            a = fminf(a, s0[w]); z = fminf(z, s1[w]); nv += c0[w]; ni += c1[w];
        }
        bounds[0] = a; bounds[1] = z;
        counts[0] = nv; counts[1] = ni;
    }
}
}  // namespace

extern "C" cv_status cv_round_summary(int B, int m, const float* lower, const uint8_t* verified,
                                      const uint8_t* infeasible, float* bounds, int* counts, void* stream) {
    if (B < 0 || m < 0 || !bounds || !counts || (B > 0 && (!verified || !infeasible || (m > 0 && !lower)))) {
        cv_set_error("cv_round_summary: negative size or null pointer");
        return CV_EINVAL;
    }
    k_round_summary<<<1, 1024, 0, (cudaStream_t)stream>>>(B, m, lower, verified, infeasible, bounds, counts);
    CV_LAUNCH_CHECK("k_round_summary");
    return CV_OK;
}

extern "C" cv_status cv_bound_batch(cv_net* net, const cv_cache* cache, const cv_batch_in* in, cv_batch_out* out,
                                    const cv_options* opt, void* workspace, size_t workspace_bytes, void* stream) {
    cv_status s = validate(net, cache, in, opt);
    if (s) return s;
    if (!out) { cv_set_error("null output"); return CV_EINVAL; }
    const int B = in->B, m = in->m, U = cache->U;
    if (B == 0) return CV_OK;
    if (!out->lo_clip || !out->hi_clip || !out->infeasible || !out->verified || (m > 0 && !out->lower) ||
        (U > 0 && (!out->l || !out->u || !out->mask))) {
        cv_set_error("required output pointer is null");
        return CV_EINVAL;
    }
    if (opt->babsr_weight && U > 0 && !out->babsr_weight) {
        cv_set_error("cv_options.babsr_weight = 1 needs cv_batch_out.babsr_weight");
        return CV_EINVAL;
    }
    if (opt->precision == CV_PREC_BF16X8 && !cv_tc_supported(cache)) {
        cv_set_error("CV_PREC_BF16X8: the tensor-core weights of a layer were not prepared (K above 65536)");
        return CV_EUNSUPPORTED;
    }
    cv_ws_layout lay;
    cv_ws_plan(net, cache, B, m, in->max_splits, in->max_rows, opt->precision, &lay, opt->babsr_weight);
    if (!workspace || workspace_bytes < lay.total) {
        cv_set_error("workspace too small: need " + std::to_string(lay.total) + " bytes");
        return CV_EWORKSPACE;
    }
    if (((uintptr_t)workspace & 255) != 0) { cv_set_error("workspace must be 256-byte aligned"); return CV_EINVAL; }
    char* ws = (char*)workspace;
    cudaStream_t st = (cudaStream_t)stream;
    cv_timer* tm = opt->timer;
    int launches = 0;
    unsigned long long* steps = nullptr;
    if (tm) {
        CV_CUDA(cudaMemsetAsync(tm->d_steps, 0, CV_TIMER_COUNTERS * sizeof(unsigned long long), st));
        CV_CUDA(cudaEventRecord(tm->ev[0], st));
        steps = tm->d_steps;
    }

    CV_CUDA(cudaMemsetAsync(out->infeasible, 0, B, st));
    if ((s = cv_launch_rows(net, cache, in, &lay, ws, out->infeasible, st))) return s;
    launches += lay.Rmax > 0;
    if ((s = cv_launch_relaxed(net, cache, in, opt, &lay, ws, out->lo_clip, out->hi_clip, out->infeasible, st))) return s;
    launches += 1;
    if (tm) CV_CUDA(cudaEventRecord(tm->ev[1], st));
    if ((s = cv_launch_reconc(net, cache, in, opt, &lay, ws, out->lo_clip, out->hi_clip, out->l, out->u, out->mask,
                              out->infeasible, st)))
        return s;
    launches += U > 0 ? (opt->precision == CV_PREC_BF16X8 ? 4 : 3) : 0;
    if (tm) CV_CUDA(cudaEventRecord(tm->ev[2], st));
    if ((s = cv_launch_complete(net, cache, in, opt, &lay, ws, out->lo_clip, out->hi_clip, out->l, out->u, out->mask,
                                out->infeasible, steps, &launches, st)))
        return s;
    if (tm) CV_CUDA(cudaEventRecord(tm->ev[3], st));
    // BaBSR weight: zero first (m = 0 leaves it so), then one reduction after each hidden layer
    float* wgt = (opt->babsr_weight && U > 0) ? out->babsr_weight : nullptr;
    if (wgt) CV_CUDA(cudaMemsetAsync(wgt, 0, (size_t)B * U * sizeof(float), st));
    if (m == 0) wgt = nullptr;
    if (m > 0 && opt->precision == CV_PREC_BF16X8) {
        s = cv_backward_tc(net, cache, lay.R, m, in->C, in->t, out->l, out->u, out->mask, U, in->alpha,
                           opt->alpha_mode, out->lo_clip, out->hi_clip, out->infeasible, out->lower, out->err_bound,
                           out->final_A, out->final_c, (float*)(ws + lay.lam0), (float*)(ws + lay.lam1),
                           (uint16_t*)(ws + lay.tc_slices), (int*)(ws + lay.tc_exp), (float*)(ws + lay.tc_tab),
                           (double*)(ws + lay.part_bias),
                           (double*)(ws + lay.part_pad), (double*)(ws + lay.part_f), (double*)(ws + lay.part_fmag),
                           (double*)(ws + lay.acc_bias), (double*)(ws + lay.acc_pad), &launches, st,
                           wgt ? (float*)(ws + lay.pbuf) : nullptr, wgt);
        if (s) return s;
    } else if (m > 0) {
        float* kpv[CV_MAX_LAYERS + 1];  // every layer's product goes to the one buffer, reduced in turn
        for (int i = 0; i <= CV_MAX_LAYERS; ++i) kpv[i] = wgt ? (float*)(ws + lay.pbuf) : nullptr;
        s = cv_backward_t<float>(net, lay.R, m, net->L, 1, m, nullptr, in->C, in->t, cache->root_l, cache->root_u,
                            cache->root_state, cache->slot_of, out->l, out->u, out->mask, U, in->alpha,
                            opt->alpha_mode, cache->V, out->lo_clip, out->hi_clip, out->infeasible, out->lower,
                            nullptr, out->err_bound, out->final_A, out->final_c, nullptr, nullptr,
                            (float*)(ws + lay.lam0), (float*)(ws + lay.lam1), (double*)(ws + lay.part_bias),
                            (double*)(ws + lay.part_pad), (double*)(ws + lay.part_f),
                            (double*)(ws + lay.part_fmag), (double*)(ws + lay.acc_bias),
                            (double*)(ws + lay.acc_pad), wgt ? kpv : nullptr, st, wgt);
        if (s) return s;
        launches += 1 + 2 * net->L + (wgt ? net->L - 1 : 0);
    }
    k_verified<<<(B + 255) / 256, 256, 0, st>>>(B, m, out->lower, out->infeasible, out->verified);
    CV_LAUNCH_CHECK("k_verified");
    launches += 1;
    if (tm) {
        CV_CUDA(cudaEventRecord(tm->ev[4], st));
        tm->launches = launches;
        tm->used = true;
    }
    return CV_OK;
}

extern "C" cv_status cv_timer_create(cv_timer** out) {
    if (!out) { cv_set_error("cv_timer_create: null"); return CV_EINVAL; }
    cv_timer* t = new cv_timer();
    memset(t, 0, sizeof(*t));
    for (int i = 0; i <= CV_N_PHASES; ++i) CV_CUDA(cudaEventCreate(&t->ev[i]));
    CV_CUDA(cudaMalloc(&t->d_steps, CV_TIMER_COUNTERS * sizeof(unsigned long long)));
    CV_CUDA(cudaMemset(t->d_steps, 0, CV_TIMER_COUNTERS * sizeof(unsigned long long)));
    *out = t;
    return CV_OK;
}

extern "C" void cv_timer_destroy(cv_timer* t) {
    if (!t) return;
    for (int i = 0; i <= CV_N_PHASES; ++i) cudaEventDestroy(t->ev[i]);
    cudaFree(t->d_steps);
    delete t;
}

extern "C" cv_status cv_timer_read(cv_timer* t, float* ms, int* launches, long long* cc_steps) {
    if (!t) { cv_set_error("cv_timer_read: null"); return CV_EINVAL; }
    if (!t->used) { cv_set_error("cv_timer_read: no timed call yet"); return CV_EINVAL; }
    CV_CUDA(cudaEventSynchronize(t->ev[CV_N_PHASES]));
    if (ms)
        for (int i = 0; i < CV_N_PHASES; ++i) CV_CUDA(cudaEventElapsedTime(&ms[i], t->ev[i], t->ev[i + 1]));
    if (launches) *launches = t->launches;
    if (cc_steps) {
        unsigned long long v = 0;
        CV_CUDA(cudaMemcpy(&v, t->d_steps, sizeof(v), cudaMemcpyDeviceToHost));
        *cc_steps = (long long)v;
    }
    return CV_OK;
}

extern "C" cv_status cv_timer_read_cc(cv_timer* t, long long stats[5]) {
    if (!t || !stats) { cv_set_error("cv_timer_read_cc: null"); return CV_EINVAL; }
    if (!t->used) { cv_set_error("cv_timer_read_cc: no timed call yet"); return CV_EINVAL; }
    unsigned long long v[CV_TIMER_COUNTERS];
    CV_CUDA(cudaEventSynchronize(t->ev[CV_N_PHASES]));
    CV_CUDA(cudaMemcpy(v, t->d_steps, sizeof(v), cudaMemcpyDeviceToHost));
    for (int i = 0; i < 5; ++i) stats[i] = (long long)v[1 + i];
    return CV_OK;
}

// ---------------------------------------------------------------- CUDA graph of a round
struct cv_graph {
    cudaGraph_t graph;
    cudaGraphExec_t exec;
};

extern "C" cv_status cv_graph_capture(cv_net* net, const cv_cache* cache, const cv_batch_in* in, cv_batch_out* out,
                                      const cv_options* opt, void* workspace, size_t workspace_bytes,
                                      cv_graph** graph) {
    if (!graph || !opt) { cv_set_error("cv_graph_capture: null argument"); return CV_EINVAL; }
    *graph = nullptr;
    cv_options o = *opt;
    o.timer = nullptr;
    cudaStream_t st = nullptr;
    CV_CUDA(cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking));
    cudaError_t e = cudaStreamBeginCapture(st, cudaStreamCaptureModeRelaxed);
    if (e != cudaSuccess) { cudaStreamDestroy(st); return cv_cuda_fail(e, "cudaStreamBeginCapture"); }
    cv_status s = cv_bound_batch(net, cache, in, out, &o, workspace, workspace_bytes, st);
    cudaGraph_t g = nullptr;
    e = cudaStreamEndCapture(st, &g);
    cudaStreamDestroy(st);
    if (s) { if (g) cudaGraphDestroy(g); return s; }
    if (e != cudaSuccess) { if (g) cudaGraphDestroy(g); return cv_cuda_fail(e, "cudaStreamEndCapture"); }
    cudaGraphExec_t x = nullptr;
    e = cudaGraphInstantiate(&x, g, 0);
    if (e != cudaSuccess) { cudaGraphDestroy(g); return cv_cuda_fail(e, "cudaGraphInstantiate"); }
    cv_graph* r = new cv_graph();
    r->graph = g;
    r->exec = x;
    *graph = r;
    return CV_OK;
}

extern "C" cv_status cv_graph_launch(cv_graph* graph, void* stream) {
    if (!graph) { cv_set_error("cv_graph_launch: null graph"); return CV_EINVAL; }
    CV_CUDA(cudaGraphLaunch(graph->exec, (cudaStream_t)stream));
    return CV_OK;
}

extern "C" void cv_graph_destroy(cv_graph* graph) {
    if (!graph) return;
    cudaGraphExecDestroy(graph->exec);
    cudaGraphDestroy(graph->graph);
    delete graph;
}

// ---------------------------------------------------------------- scheduler tuning

extern "C" cv_status cv_cc_items_set(cv_cache* cache, const int items[3]) {
    if (!cache || !items) { cv_set_error("cv_cc_items_set: null argument"); return CV_EINVAL; }
    for (int c = 0; c < 3; ++c)
        if (items[c] < 1 || items[c] > 4096) {
            cv_set_error("cv_cc_items_set: tasks per item must lie in [1, 4096]");
            return CV_EINVAL;
        }
    for (int c = 0; c < 3; ++c) cache->cc_items[c] = items[c];
    return CV_OK;
}

extern "C" cv_status cv_cc_items_get(const cv_cache* cache, int items[3]) {
    if (!cache || !items) { cv_set_error("cv_cc_items_get: null argument"); return CV_EINVAL; }
    for (int c = 0; c < 3; ++c) items[c] = cache->cc_items[c];
    return CV_OK;
}

extern "C" cv_status cv_autotune_cc(cv_net* net, cv_cache* cache, const cv_batch_in* in, cv_batch_out* out,
                                    const cv_options* opt, void* workspace, size_t workspace_bytes, void* stream,
                                    int best[3], float* best_ms) {
    if (!net || !cache || !in || !out || !opt) { cv_set_error("cv_autotune_cc: null argument"); return CV_EINVAL; }
    if (opt->sweeps <= 0) { cv_set_error("cv_autotune_cc: sweeps = 0, no complete clipping to tune"); return CV_EINVAL; }
    static const int cand[3][5] = {{128, 256, 512, 1024, 0}, {32, 64, 128, 256, 0}, {8, 16, 32, 64, 128}};
    cv_timer* timer = nullptr;
    cv_status s = cv_timer_create(&timer);
    if (s) return s;
    cv_options o = *opt;
    o.timer = timer;
    int cur[3], keep[3], orig[3];
    for (int c = 0; c < 3; ++c) cur[c] = keep[c] = orig[c] = cache->cc_items[c];
    float best_t = 0.f;
    bool have = false;
    // time one setting: the faster of two rounds
    auto time_it = [&](const int it[3], float* t) -> cv_status {
        for (int c = 0; c < 3; ++c) cache->cc_items[c] = it[c];
        float tb = 0.f;
        for (int rep = 0; rep < 2; ++rep) {
            cv_status e = cv_bound_batch(net, cache, in, out, &o, workspace, workspace_bytes, stream);
            if (e) return e;
            float ms[CV_N_PHASES];
            if ((e = cv_timer_read(timer, ms, nullptr, nullptr))) return e;
            if (rep == 0 || ms[2] < tb) tb = ms[2];
        }
        *t = tb;
        return CV_OK;
    };
    float t0 = 0.f;
    s = time_it(cur, &t0);  // the first rounds also warm the caches and the code
    if (!s) s = time_it(cur, &t0);
    if (!s) { best_t = t0; have = true; }
    for (int c = 0; c < 3 && !s; ++c) {
        for (int i = 0; i < 5 && !s; ++i) {
            const int v = cand[c][i];
            if (v == 0 || v == cur[c]) continue;
            int trial[3] = {cur[0], cur[1], cur[2]};
            trial[c] = v;
            float t = 0.f;
            s = time_it(trial, &t);
            if (!s && t < best_t) { best_t = t; for (int q = 0; q < 3; ++q) keep[q] = trial[q]; }
        }
        for (int q = 0; q < 3; ++q) cur[q] = keep[q];
    }
    cv_timer_destroy(timer);
    for (int c = 0; c < 3; ++c) cache->cc_items[c] = s ? orig[c] : keep[c];  // unchanged on an error
    if (s) return s;
    if (best) for (int c = 0; c < 3; ++c) best[c] = keep[c];
    if (best_ms) *best_ms = have ? best_t : 0.f;
    return CV_OK;
}

// ---------------------------------------------------------------- complete clipping of the spec planes

namespace {
// layout of cv_spec_clip's workspace: row status and minima, the complete-clipping region, scales
struct SpecWs { size_t rowflag, vmin, cc, sscale, total; };
SpecWs spec_ws(const cv_cache* cache, const cv_batch_in* in) {
    SpecWs w;
    const size_t Rm = (size_t)in->B * (size_t)(in->max_splits + in->max_rows);
    size_t off = 0;
    auto take = [&](size_t bytes) { size_t o = off; off = cv_align256(off + (bytes ? bytes : 1)); return o; };
    w.rowflag = take(Rm);
    w.vmin = take(Rm * sizeof(double));
    w.cc = take(cv_cc_workspace(in->B, in->max_splits + in->max_rows, cache->n0));
    w.sscale = take((size_t)2 * in->B * in->m * sizeof(float));  // plane scales, then plane maxima
    w.total = off;
    return w;
}
}  // namespace

extern "C" cv_status cv_spec_clip_workspace(const cv_net* net, const cv_cache* cache, const cv_batch_in* in,
                                            size_t* bytes) {
    cv_options o;
    cv_options_default(&o);
    cv_status s = validate(net, cache, in, &o, false);
    if (s) return s;
    if (!bytes) { cv_set_error("null bytes"); return CV_EINVAL; }
    *bytes = spec_ws(cache, in).total;
    return CV_OK;
}

extern "C" cv_status cv_spec_clip(cv_net* net, const cv_cache* cache, const cv_batch_in* in, cv_batch_out* out,
                                  const cv_options* opt, void* workspace, size_t workspace_bytes, void* stream) {
    cv_status s = validate(net, cache, in, opt);
    if (s) return s;
    if (!out) { cv_set_error("null output"); return CV_EINVAL; }
    if (opt->sweeps <= 0) { cv_set_error("cv_spec_clip: sweeps = 0, nothing to do"); return CV_EINVAL; }
    const int B = in->B, m = in->m;
    if (B == 0 || m == 0) return CV_OK;
    if (!out->lo_clip || !out->hi_clip || !out->infeasible || !out->verified || !out->lower || !out->final_A ||
        !out->final_c) {
        cv_set_error("cv_spec_clip: needs lo_clip, hi_clip, infeasible, verified, lower, final_A and final_c");
        return CV_EINVAL;
    }
    const SpecWs w = spec_ws(cache, in);
    if (!workspace || workspace_bytes < w.total) {
        cv_set_error("workspace too small: need " + std::to_string(w.total) + " bytes");
        return CV_EWORKSPACE;
    }
    if (((uintptr_t)workspace & 255) != 0) { cv_set_error("workspace must be 256-byte aligned"); return CV_EINVAL; }
    char* ws = (char*)workspace;
    cudaStream_t st = (cudaStream_t)stream;
    cv_ws_layout lay;
    memset(&lay, 0, sizeof(lay));
    lay.Rmax = in->max_splits + in->max_rows;
    lay.R = B * m;
    lay.rowflag = w.rowflag;
    lay.vmin = w.vmin;
    lay.cc = w.cc;
    lay.total = w.total;
    int launches = 0;
    cv_timer* tm = opt->timer;
    if (tm) {
        CV_CUDA(cudaMemsetAsync(tm->d_steps, 0, CV_TIMER_COUNTERS * sizeof(unsigned long long), st));
        for (int i = 0; i <= CV_N_PHASES; ++i) CV_CUDA(cudaEventRecord(tm->ev[i], st));
    }
    // the active rows, as the round's pre-check found them on the input box (infeasible flags the
    // round already set are set again; none is cleared)
    if ((s = cv_launch_rows(net, cache, in, &lay, ws, out->infeasible, st))) return s;
    if ((s = cv_launch_spec_clip(net, cache, in, out, opt, &lay, ws, (float*)(ws + w.sscale),
                                 tm ? tm->d_steps : nullptr, &launches, st)))
        return s;
    k_verified<<<(B + 255) / 256, 256, 0, st>>>(B, m, out->lower, out->infeasible, out->verified);
    CV_LAUNCH_CHECK("k_verified");
    if (tm) {
        // the whole call counts as the complete-clipping phase
        for (int i = 3; i <= CV_N_PHASES; ++i) CV_CUDA(cudaEventRecord(tm->ev[i], st));
        tm->launches = launches + 2;
        tm->used = true;
    }
    return CV_OK;
}
