// Gradient of the spec bounds with respect to the lower relaxation slopes alpha (a9), and the Adam
// ascent step that optimises them (alpha-CROWN, the "optimized" alpha of the paper's ReLU
// relaxation Lemma; Adam with lr 0.1 decayed by 0.98 per iteration in its experiments appendix).
//
// Forward: the back-substitution of cv_bound_batch's spec step with the given alpha, keeping the
// layer products P^(i) = Lam^(i) W^(i) (i = 2..L) and Lam_0 = P^(1).  Reverse sweep, with the
// relaxation choices of the forward held fixed (P >= 0 selects the lower relaxation):
//   dLam_0          = g_f (xhat - sign(Lam_0) eps)                     (concretisation)
//   dLam^(h)        = dP^(h) W^(h)^T + g_f b^(h)                       (P^(h) = Lam^(h) W^(h))
//   d alpha^(h)_j   = dLam^(h)_j P^(h+1)_j   (unstable neuron, lower relaxation selected)
//   dP^(h+1)_j      = dLam^(h)_j d_j + g_f e_j                         (Lam^(h) = P^(h+1) d, bias += P e)
// with dP^(1) := dLam_0.  Each reverse step is an NT contraction [R x n_{h-1}] x W^(h)^T on CUDA
// cores with the relaxation epilogue fused.  The gradient is not a bound: it carries no pad.
#include "cv_internal.cuh"

#include <math.h>
#include <string.h>

namespace {

constexpr int BM = 64, BN = 64, BK = 16;

__global__ void k_adj_start(int R, int n0, int m, const float* lam0, const float* lo, const float* hi,
                            const float* grad_f, float* out) {
    const size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= (size_t)R * n0) return;
    const int r = (int)(i / n0), q = (int)(i % n0);
    const int sub = r / m;
    const float gf = grad_f ? grad_f[r] : 1.f;
    const float l0 = lo[(size_t)sub * n0 + q], h0 = hi[(size_t)sub * n0 + q];
    const float xh = 0.5f * (l0 + h0), ep = 0.5f * (h0 - l0);
    const float v = lam0[i];
    out[i] = gf * (xh - (v > 0.f ? ep : (v < 0.f ? -ep : 0.f)));
}

struct AdjArgs {
    const float* A;      // dP^(h) [R x K]
    const float* W;      // W^(h) [N x K]
    const float* b;      // b^(h) [N]
    int R, K, N, m, H, U, hoff, last;
    const float* P;      // P^(h+1) [R x N] (the forward product whose sign chose the relaxation)
    const int* slot_of; const float* l; const float* u; const int8_t* mask;
    const float* root_l; const float* root_u; const int8_t* root_state;
    const float* alpha;  // [B x m x H]
    const float* grad_f; // [R] or NULL
    float* out;          // dP^(h+1) [R x N] (unless last)
    float* grad_alpha;   // [B x m x H]
    const int8_t* bsign; // [B x H] split signs, or NULL (no split multipliers)
    float* grad_beta;    // [B x m x H]: d / d beta = -sign dLam^(h) at split neurons
};

__global__ void __launch_bounds__(256) k_adj_layer(AdjArgs a) {
    __shared__ float As[BK][BM + 4];
    __shared__ float Ws[BK][BN + 4];
    const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
    const int r0 = blockIdx.y * BM, j0 = blockIdx.x * BN;
    float acc[4][4];
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = 0.f;
    for (int k0 = 0; k0 < a.K; k0 += BK) {
#pragma unroll
        for (int e = 0; e < 4; ++e) {
            const int idx = tid * 4 + e;
            const int rr = idx >> 4, kk = idx & 15;
            const int gk = k0 + kk;
            As[kk][rr] = (r0 + rr < a.R && gk < a.K) ? a.A[(size_t)(r0 + rr) * a.K + gk] : 0.f;
            Ws[kk][rr] = (j0 + rr < a.N && gk < a.K) ? a.W[(size_t)(j0 + rr) * a.K + gk] : 0.f;
        }
        __syncthreads();
#pragma unroll
        for (int kk = 0; kk < BK; ++kk) {
            float av[4], wv[4];
#pragma unroll
            for (int i = 0; i < 4; ++i) av[i] = As[kk][ty * 4 + i];
#pragma unroll
            for (int j = 0; j < 4; ++j) wv[j] = Ws[kk][tx * 4 + j];
#pragma unroll
            for (int i = 0; i < 4; ++i)
#pragma unroll
                for (int j = 0; j < 4; ++j) acc[i][j] = fmaf(av[i], wv[j], acc[i][j]);
        }
        __syncthreads();
    }
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        const int r = r0 + ty * 4 + i;
        if (r >= a.R) continue;
        const int sub = r / a.m;
        const float gf = a.grad_f ? a.grad_f[r] : 1.f;
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const int q = j0 + tx * 4 + j;
            if (q >= a.N) continue;
            const float dl = acc[i][j] + gf * a.b[q];  // dLam^(h)_q
            const int g = a.hoff + q;
            const int slot = a.slot_of[g];
            float lb, ub; int st;
            if (slot >= 0) {
                const size_t o = (size_t)sub * a.U + slot;
                lb = a.l[o]; ub = a.u[o]; st = a.mask[o];
            } else {
                lb = a.root_l[g]; ub = a.root_u[g]; st = a.root_state[g];
            }
            const float p = a.P[(size_t)r * a.N + q];
            float d, e;
            const size_t ga = ((size_t)sub * a.m + (r % a.m)) * a.H + g;
            if (st > 0) { d = 1.f; e = 0.f; }
            else if (st < 0) { d = 0.f; e = 0.f; }
            else if (p >= 0.f) {
                d = a.alpha[ga];
                e = 0.f;
                a.grad_alpha[ga] = dl * p;
            } else {
                const float s = ub / (ub - lb);
                d = s;
                e = -s * lb;
            }
            if (a.bsign) {
                const int sg = a.bsign[(size_t)sub * a.H + g];
                if (sg) a.grad_beta[ga] = (float)(-sg) * dl;
            }
            if (!a.last) a.out[(size_t)r * a.N + q] = dl * d + gf * e;
        }
    }
}

// One element of the Adam ascent step, the result clamped to [lo, hi].
__device__ __forceinline__ void adam_one(float& x, float& m1v, float& m2v, float gi, float lr, float b1, float b2,
                                         float c1, float c2, float eps, float lo, float hi) {
    const float a1 = b1 * m1v + (1.f - b1) * gi;
    const float a2 = b2 * m2v + (1.f - b2) * gi * gi;
    m1v = a1;
    m2v = a2;
    const float step = lr * (a1 / c1) / (sqrtf(a2 / c2) + eps);
    x = fminf(fmaxf(x + step, lo), hi);
}

// The Adam step over n elements (HBM-bound): four elements a thread as 16-byte accesses when all four
// arrays are 16-byte aligned (a grid-stride loop), then the remaining elements one at a time.
__global__ void k_adam_range(long long n, float* x, float* m1, float* m2, const float* g, float lr, float b1,
                             float b2, float c1, float c2, float eps, float lo, float hi) {
    const long long stride = (long long)gridDim.x * blockDim.x;
    const long long tid = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const bool al = (((uintptr_t)x | (uintptr_t)m1 | (uintptr_t)m2 | (uintptr_t)g) & 15) == 0;
    const long long n4 = al ? n / 4 : 0;
    for (long long v = tid; v < n4; v += stride) {
        float4 X = ((float4*)x)[v], A = ((float4*)m1)[v], M = ((float4*)m2)[v];
        const float4 G = ((const float4*)g)[v];
        adam_one(X.x, A.x, M.x, G.x, lr, b1, b2, c1, c2, eps, lo, hi);
        adam_one(X.y, A.y, M.y, G.y, lr, b1, b2, c1, c2, eps, lo, hi);
        adam_one(X.z, A.z, M.z, G.z, lr, b1, b2, c1, c2, eps, lo, hi);
        adam_one(X.w, A.w, M.w, G.w, lr, b1, b2, c1, c2, eps, lo, hi);
        ((float4*)x)[v] = X;
        ((float4*)m1)[v] = A;
        ((float4*)m2)[v] = M;
    }
    for (long long i = 4 * n4 + tid; i < n; i += stride) {
        float xv = x[i], a = m1[i], b = m2[i];
        adam_one(xv, a, b, g[i], lr, b1, b2, c1, c2, eps, lo, hi);
        m1[i] = a;
        m2[i] = b;
        x[i] = xv;
    }
}

// threads for n elements, four a thread
inline unsigned adam_blocks(long long n) { return (unsigned)((n / 4 + 255) / 256 + 1); }

struct AlphaLayout {
    size_t lamA, lamB, pb, pp, pf, pm, ab, ap, lam0, keep[CV_MAX_LAYERS + 1], gA, gB;
    size_t tc_slices, tc_exp, tc_tab, total;  // tensor-core path
};

void alpha_plan(const cv_net* net, int B, int m, AlphaLayout* L) {
    memset(L, 0, sizeof(*L));
    const size_t R = (size_t)B * m;
    const int ncb = cv_bwd_ncb_max(net);
    size_t off = 0;
    auto take = [&](size_t bytes) { size_t o = off; off = cv_align256(off + (bytes ? bytes : 1)); return o; };
    L->lamA = take(R * net->wmax * 4);
    L->lamB = take(R * net->wmax * 4);
    L->pb = take(R * ncb * 8);
    L->pp = take(R * ncb * 8);
    L->pf = take(R * ncb * 8);
    L->pm = take(R * ncb * 8);
    L->ab = take(R * 8);
    L->ap = take(R * 8);
    L->lam0 = take(R * net->dims[0] * 4);
    for (int i = 2; i <= net->L; ++i) L->keep[i] = take(R * net->dims[i - 1] * 4);
    L->gA = take(R * net->wmax * 4);
    L->gB = take(R * net->wmax * 4);
    // digit slices of R rows for the forward (K = n_i, i >= 1) and the reverse sweep (K = n_{h-1},
    // down to n_0): every width of the network, rounded up to the 64-wide K tile
    L->tc_slices = take((size_t)3 * R * (size_t)((net->wmax + 63) / 64 * 64) * sizeof(uint16_t));
    L->tc_exp = take(R * sizeof(int));
    L->tc_tab = take((size_t)3 * B * net->wmax * sizeof(float));
    L->total = off;
}

}  // namespace

extern "C" cv_status cv_alpha_grad_workspace(const cv_net* net, int B, int m, size_t* bytes) {
    if (!net || !bytes || B < 0 || m < 0) { cv_set_error("cv_alpha_grad_workspace: bad arguments"); return CV_EINVAL; }
    AlphaLayout L;
    alpha_plan(net, B, m, &L);
    *bytes = L.total;
    return CV_OK;
}

extern "C" cv_status cv_alpha_grad(cv_net* net, const cv_cache* cache, const cv_alpha_in* in, float* lower,
                                   float* grad_alpha, void* workspace, size_t workspace_bytes, void* stream) {
    if (!net || !cache || !in || !grad_alpha || cache->net != net) {
        cv_set_error("cv_alpha_grad: bad arguments");
        return CV_EINVAL;
    }
    const int B = in->B, m = in->m, U = cache->U, H = net->H;
    if (B < 0 || m <= 0 || !in->lo || !in->hi || !in->C || !in->alpha ||
        (U > 0 && (!in->l || !in->u || !in->mask))) {
        cv_set_error("cv_alpha_grad: missing input");
        return CV_EINVAL;
    }
    if (in->precision != CV_PREC_FP32 && in->precision != CV_PREC_BF16X8) {
        cv_set_error("cv_alpha_grad: unknown precision");
        return CV_EINVAL;
    }
    if (in->beta && (!in->split_sign || !in->grad_beta)) {
        cv_set_error("cv_alpha_grad: beta needs split_sign and grad_beta");
        return CV_EINVAL;
    }
    if (in->precision == CV_PREC_BF16X8 && !cv_tc_supported(cache)) {
        cv_set_error("cv_alpha_grad: the tensor-core weights of a layer were not prepared");
        return CV_EUNSUPPORTED;
    }
    if (B == 0) return CV_OK;
    AlphaLayout L;
    alpha_plan(net, B, m, &L);
    if (!workspace || workspace_bytes < L.total) {
        cv_set_error("cv_alpha_grad: workspace too small: need " + std::to_string(L.total) + " bytes");
        return CV_EWORKSPACE;
    }
    if (((uintptr_t)workspace & 255) != 0) {
        cv_set_error("cv_alpha_grad: workspace must be 256-byte aligned");
        return CV_EINVAL;
    }
    char* ws = (char*)workspace;
    cudaStream_t st = (cudaStream_t)stream;
    const int R = B * m, n0 = net->dims[0];
    float* keep[CV_MAX_LAYERS + 1] = {nullptr};
    for (int i = 2; i <= net->L; ++i) keep[i] = (float*)(ws + L.keep[i]);
    float* lam0 = (float*)(ws + L.lam0);
    const bool tc = in->precision == CV_PREC_BF16X8;
    cv_status s;
    int launches = 0;
    if (tc) {
        // the forward on tensor cores (the bound of cv_bound_batch's split-BF16 path), keeping P^(i)
        // and Lam_0; lower is written unless NULL
        s = cv_backward_tc(net, cache, R, m, in->C, in->t, in->l, in->u, in->mask, U, in->alpha, CV_ALPHA_ADAPTIVE,
                           in->lo, in->hi, nullptr, lower, nullptr, lam0, nullptr, (float*)(ws + L.lamA),
                           (float*)(ws + L.lamB), (uint16_t*)(ws + L.tc_slices), (int*)(ws + L.tc_exp),
                           (float*)(ws + L.tc_tab), (double*)(ws + L.pb), (double*)(ws + L.pp),
                           (double*)(ws + L.pf), (double*)(ws + L.pm), (double*)(ws + L.ab), (double*)(ws + L.ap),
                           &launches, st, nullptr, nullptr, keep, in->beta, in->split_sign);
    } else {
        s = cv_backward_t<float>(net, R, m, net->L, 1, m, nullptr, in->C, in->t, cache->root_l, cache->root_u,
                                 cache->root_state, cache->slot_of, in->l, in->u, in->mask, U, in->alpha,
                                 CV_ALPHA_ADAPTIVE, cache->V, in->lo, in->hi, nullptr, lower, nullptr,
                                 nullptr, lam0, nullptr, nullptr, nullptr, (float*)(ws + L.lamA),
                                 (float*)(ws + L.lamB), (double*)(ws + L.pb), (double*)(ws + L.pp),
                                 (double*)(ws + L.pf), (double*)(ws + L.pm), (double*)(ws + L.ab),
                                 (double*)(ws + L.ap), keep, st, nullptr, in->beta, in->split_sign);
    }
    if (s) return s;
    const int8_t* bsign = in->beta ? in->split_sign : nullptr;
    if (bsign) CV_CUDA(cudaMemsetAsync(in->grad_beta, 0, (size_t)B * m * H * sizeof(float), st));
    CV_CUDA(cudaMemsetAsync(grad_alpha, 0, (size_t)B * m * H * sizeof(float), st));
    float* gA = (float*)(ws + L.gA);
    float* gB = (float*)(ws + L.gB);
    {
        const size_t n = (size_t)R * n0;
        k_adj_start<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(R, n0, m, lam0, in->lo, in->hi, in->grad_f, gA);
        CV_LAUNCH_CHECK("k_adj_start");
    }
    if (tc)
        return cv_alpha_reverse_tc(net, cache, R, m, in->l, in->u, in->mask, in->alpha, in->grad_f, keep, gA, gB,
                                   (uint16_t*)(ws + L.tc_slices), (int*)(ws + L.tc_exp), grad_alpha, &launches, st,
                                   bsign, in->grad_beta);
    for (int h = 1; h <= net->L - 1; ++h) {
        AdjArgs a;
        a.A = gA; a.W = net->W[h]; a.b = net->b[h];
        a.R = R; a.K = net->dims[h - 1]; a.N = net->dims[h]; a.m = m; a.H = H; a.U = U;
        a.hoff = net->hoff[h]; a.last = (h == net->L - 1);
        a.P = keep[h + 1];
        a.slot_of = cache->slot_of; a.l = in->l; a.u = in->u; a.mask = in->mask;
        a.root_l = cache->root_l; a.root_u = cache->root_u; a.root_state = cache->root_state;
        a.alpha = in->alpha; a.grad_f = in->grad_f;
        a.out = gB; a.grad_alpha = grad_alpha;
        a.bsign = bsign; a.grad_beta = in->grad_beta;
        dim3 grd((a.N + BN - 1) / BN, (R + BM - 1) / BM);
        k_adj_layer<<<grd, 256, 0, st>>>(a);
        CV_LAUNCH_CHECK("k_adj_layer");
        float* t = gA; gA = gB; gB = t;
    }
    return CV_OK;
}

namespace {


// thread per split code: +(g+1) -> +1, -(g+1) -> -1 at [b, g]
__global__ void k_split_signs(int B, int H, const int* split_off, const int* split_ids, int8_t* sign, int* status) {
    const int b = blockIdx.x;
    if (b >= B) return;
    const int k0 = split_off[b], k1 = split_off[b + 1];
    for (int k = k0 + threadIdx.x; k < k1; k += blockDim.x) {
        const int code = split_ids[k];
        const int g = (code > 0 ? code : -code) - 1;
        if (code == 0 || g >= H) { atomicOr(status, CV_DEV_SPLIT_RANGE); continue; }
        sign[(size_t)b * H + g] = code > 0 ? (int8_t)1 : (int8_t)-1;
    }
}

}  // namespace

extern "C" cv_status cv_split_signs(cv_net* net, int B, const int* split_off, const int* split_ids, int8_t* sign,
                                    void* stream) {
    if (!net || B < 0 || (B > 0 && !sign) || (split_off && !split_ids)) {
        cv_set_error("cv_split_signs: bad arguments");
        return CV_EINVAL;
    }
    cudaStream_t st = (cudaStream_t)stream;
    const int H = net->H;
    if (B == 0 || H == 0) return CV_OK;
    CV_CUDA(cudaMemsetAsync(sign, 0, (size_t)B * H, st));
    if (!split_off) return CV_OK;
    k_split_signs<<<B, 64, 0, st>>>(B, H, split_off, split_ids, sign, net->status);
    CV_LAUNCH_CHECK("k_split_signs");
    return CV_OK;
}

extern "C" cv_status cv_adam_range(float* x, float* m1, float* m2, const float* grad, long long n, int t, float lr,
                                   float beta1, float beta2, float eps, float lo, float hi, void* stream) {
    if (!x || !m1 || !m2 || !grad || n < 0 || t < 1 || !(lo <= hi)) {
        cv_set_error("cv_adam_range: bad arguments");
        return CV_EINVAL;
    }
    if (n == 0) return CV_OK;
    const float c1 = 1.f - powf(beta1, (float)t), c2 = 1.f - powf(beta2, (float)t);
    k_adam_range<<<adam_blocks(n), 256, 0, (cudaStream_t)stream>>>(n, x, m1, m2, grad, lr, beta1, beta2, c1, c2, eps,
                                                                    lo, hi);
    CV_LAUNCH_CHECK("k_adam_range");
    return CV_OK;
}

extern "C" cv_status cv_alpha_adam(float* alpha, float* m1, float* m2, const float* grad, long long n, int t,
                                   float lr, float beta1, float beta2, float eps, void* stream) {
    if (!alpha || !m1 || !m2 || !grad || n < 0 || t < 1) { cv_set_error("cv_alpha_adam: bad arguments"); return CV_EINVAL; }
    if (n == 0) return CV_OK;
    const float c1 = 1.f - powf(beta1, (float)t), c2 = 1.f - powf(beta2, (float)t);
    k_adam_range<<<adam_blocks(n), 256, 0, (cudaStream_t)stream>>>(n, alpha, m1, m2, grad, lr, beta1, beta2, c1, c2,
                                                                    eps, 0.f, 1.f);
    CV_LAUNCH_CHECK("k_adam_range");
    return CV_OK;
}
