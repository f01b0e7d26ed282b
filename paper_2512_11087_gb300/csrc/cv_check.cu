// Device-side validation of a batch (cv_batch_check): the checks the per-round calls cannot make on
// the host without reading the caller's device inputs back.  Problems are collected as bits in the
// network's check word (the word after the device status word) and read back once.
#include "cv_internal.cuh"

#include <math.h>

#include <string>

namespace {

constexpr int CHK_CSR = 1, CHK_SPLIT = 2, CHK_NONFINITE = 4, CHK_TARGET = 8, CHK_EMPTY = 32, CHK_ALPHA = 64;

// one block per subdomain: CSR counts and codes, target slots, the box, inherited bounds, slopes
__global__ void k_check_sub(cv_cache cc, cv_batch_in in, int* word) {
    const int b = blockIdx.x;
    const int n0 = cc.n0, U = cc.U, H = cc.H;
    int bits = 0;
    bool splits_ok = false, tgts_ok = false;
    int s0 = 0, s1 = 0, t0 = 0, t1 = 0;
    if (in.split_off) {
        s0 = in.split_off[b];
        s1 = in.split_off[b + 1];
        splits_ok = s0 >= 0 && s1 >= s0 && s1 - s0 <= in.max_splits;
        if (!splits_ok) bits |= CHK_CSR;
    }
    if (in.row_off) {
        const int r0 = in.row_off[b], r1 = in.row_off[b + 1];
        if (r0 < 0 || r1 < r0 || r1 - r0 > in.max_rows) bits |= CHK_CSR;
    }
    if (in.tgt_off) {
        t0 = in.tgt_off[b];
        t1 = in.tgt_off[b + 1];
        tgts_ok = t0 >= 0 && t1 >= t0;
        if (!tgts_ok) bits |= CHK_CSR;
    }
    if (splits_ok)
        for (int s = s0 + (int)threadIdx.x; s < s1; s += blockDim.x) {
            const int code = in.split_ids[s];
            if (code == 0 || code == INT_MIN || (code > 0 ? code : -code) - 1 >= H) bits |= CHK_SPLIT;
        }
    if (tgts_ok)
        for (int t = t0 + (int)threadIdx.x; t < t1; t += blockDim.x) {
            const int c = in.tgt_ids[t];
            if (c < 0 || c >= U) bits |= CHK_TARGET;
        }
    for (int j = threadIdx.x; j < n0; j += blockDim.x) {
        const float l = in.lo[(size_t)b * n0 + j], h = in.hi[(size_t)b * n0 + j];
        if (!isfinite(l) || !isfinite(h)) bits |= CHK_NONFINITE;
        else if (l > h) bits |= CHK_EMPTY;
    }
    if (in.l_in)
        for (int c = threadIdx.x; c < U; c += blockDim.x)
            if (isnan(in.l_in[(size_t)b * U + c]) || isnan(in.u_in[(size_t)b * U + c])) bits |= CHK_NONFINITE;
    if (in.alpha) {
        const size_t n = (size_t)in.m * H;
        for (size_t i = threadIdx.x; i < n; i += blockDim.x) {
            const float v = in.alpha[(size_t)b * n + i];
            if (isnan(v)) bits |= CHK_NONFINITE;
            else if (v < 0.f || v > 1.f) bits |= CHK_ALPHA;
        }
    }
    if (bits) atomicOr(word, bits);
}

// the shared arrays: extra rows (as many as row_off[B] says), spec rows and thresholds
__global__ void k_check_flat(cv_cache cc, cv_batch_in in, int nL, int* word) {
    const size_t tid = (size_t)blockIdx.x * blockDim.x + threadIdx.x, nt = (size_t)gridDim.x * blockDim.x;
    int bits = 0;
    if (in.row_off) {
        const int rows = in.row_off[in.B];
        if (rows >= 0) {
            const size_t n = (size_t)rows * cc.n0;
            for (size_t i = tid; i < n; i += nt)
                if (!isfinite(in.G[i])) bits |= CHK_NONFINITE;
            for (size_t i = tid; i < (size_t)rows; i += nt)
                if (!isfinite(in.h[i])) bits |= CHK_NONFINITE;
        }
    }
    if (in.C)
        for (size_t i = tid; i < (size_t)in.m * nL; i += nt)
            if (!isfinite(in.C[i])) bits |= CHK_NONFINITE;
    if (in.t)
        for (size_t i = tid; i < (size_t)in.m; i += nt)
            if (!isfinite(in.t[i])) bits |= CHK_NONFINITE;
    if (bits) atomicOr(word, bits);
}

}  // namespace

extern "C" cv_status cv_batch_check(cv_net* net, const cv_cache* cache, const cv_batch_in* in, int* code,
                                    void* stream) {
    if (code) *code = 0;
    if (!net || !cache || !in) { cv_set_error("cv_batch_check: null net / cache / input"); return CV_EINVAL; }
    if (cache->net != net) { cv_set_error("cv_batch_check: cache was built for another network"); return CV_EINVAL; }
    if (in->B < 0 || in->m < 0 || in->max_splits < 0 || in->max_rows < 0) {
        cv_set_error("cv_batch_check: negative B, m, max_splits or max_rows");
        return CV_EINVAL;
    }
    if (in->B > 0 && (!in->lo || !in->hi)) { cv_set_error("cv_batch_check: lo/hi required"); return CV_EINVAL; }
    if ((in->tgt_off == nullptr) != (in->tgt_ids == nullptr) || (in->l_in == nullptr) != (in->u_in == nullptr) ||
        (in->split_off && !in->split_ids) || (in->row_off && (!in->G || !in->h))) {
        cv_set_error("cv_batch_check: incomplete CSR or bound arguments");
        return CV_EINVAL;
    }
    if (in->B == 0) return CV_OK;
    cudaStream_t st = (cudaStream_t)stream;
    int* word = net->status + 1;
    CV_CUDA(cudaMemsetAsync(word, 0, sizeof(int), st));
    k_check_sub<<<in->B, 128, 0, st>>>(*cache, *in, word);
    CV_LAUNCH_CHECK("k_check_sub");
    k_check_flat<<<64, 256, 0, st>>>(*cache, *in, net->dims[net->L], word);
    CV_LAUNCH_CHECK("k_check_flat");
    int h = 0;
    CV_CUDA(cudaMemcpyAsync(&h, word, sizeof(int), cudaMemcpyDeviceToHost, st));
    CV_CUDA(cudaStreamSynchronize(st));
    if (code) *code = h;
    if (!h) return CV_OK;
    std::string msg = "cv_batch_check:";
    if (h & CHK_CSR) msg += " CSR offsets decreasing or a count above max_splits / max_rows;";
    if (h & CHK_SPLIT) msg += " split code 0 or beyond the hidden neurons;";
    if (h & CHK_NONFINITE) msg += " non-finite value (box bound, NaN bound or slope, G, h, C or t);";
    if (h & CHK_TARGET) msg += " target slot outside [0, U);";
    if (h & CHK_EMPTY) msg += " lo > hi;";
    if (h & CHK_ALPHA) msg += " slope outside [0, 1];";
    cv_set_error(msg);
    return (h & CHK_NONFINITE) ? CV_ENAN : CV_EINVAL;
}
