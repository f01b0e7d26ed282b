// Network and root-cache objects: cv_net_create / cv_cache_build / cv_cache_create.
//
// The root cache is the "Get_Constraints" / "Init_Clipper" step of the paper's Algorithm 5
// (Section 3.4, cache and reuse): CROWN over every hidden layer k = 1..L-1 in turn, each a
// back-substitution of +/- identity rows through layers k..1 with the relaxations of the
// layers below, concretised over the root box.  It runs once per property, so it runs in FP64
// (cv_backward_t<double>) and only the stored planes and bounds are FP32.  The planes of the
// root-unstable neurons are kept; every later round re-concretises them over its clipped box.
#include "cv_internal.cuh"

#include <math.h>
#include <stdlib.h>
#include <string.h>

#include <vector>


namespace {

// V[j] = sum_q |W[j,q]| zmag[q] + |b[j]|, rounded up (pad weights)
__global__ void k_padweights(int no, int ni, const float* W, const float* b, const float* zmag, float* V) {
    const int j = blockIdx.x * blockDim.y + threadIdx.y;
    if (j >= no) return;
    double s = 0.0;
    for (int q = threadIdx.x; q < ni; q += 32) s += (double)fabsf(W[(size_t)j * ni + q]) * (double)zmag[q];
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) s += __shfl_xor_sync(0xffffffffu, s, off);
    if (threadIdx.x == 0) V[j] = __double2float_ru((s + fabs((double)b[j])) * (1.0 + 1e-12));
}

__global__ void k_absmax(int n, const float* a, const float* b, float* out) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) out[i] = fmaxf(fabsf(a[i]), fabsf(b[i]));
}

// Layer k bounds from the FP64 backward results (rows < nk: lower planes, rows >= nk: lower planes
// of -z).  The FP64 planes are stored as FP32: A is rounded to nearest and the intercept absorbs the
// rounding, c' = c - sum_q |A_q - fl(A_q)| max(|lo_q|,|hi_q|) (rounded down), so the stored plane
// is valid over the root box.  Bounds are kept in FP64 for the deeper layers and rounded outward.
__global__ void k_root_bounds(int nk, int n0, const double* lower64, const double* lam0, const double* bias_raw,
                              const double* pad_raw, const float* xmag, double* l64, double* u64, float* l_all,
                              float* u_all, int8_t* st_all, float* zmag, float* lA, float* lc, float* uA, float* uc) {
    const int j = blockIdx.x;
    if (j >= nk) return;
    double dl = 0.0, du = 0.0, ml = 0.0, mu = 0.0;
    for (int q = threadIdx.x; q < n0; q += blockDim.x) {
        const double a = lam0[(size_t)j * n0 + q];
        const double b = -lam0[(size_t)(j + nk) * n0 + q];
        const float af = (float)a, bf = (float)b;
        lA[(size_t)j * n0 + q] = af;
        uA[(size_t)j * n0 + q] = bf;
        dl += fabs(a - (double)af) * (double)xmag[q];
        du += fabs(b - (double)bf) * (double)xmag[q];
        ml += fabs(a) * (double)xmag[q];
        mu += fabs(b) * (double)xmag[q];
    }
    __shared__ double red[4][32];
    for (int off = 16; off > 0; off >>= 1) {
        dl += __shfl_xor_sync(0xffffffffu, dl, off);
        du += __shfl_xor_sync(0xffffffffu, du, off);
        ml += __shfl_xor_sync(0xffffffffu, ml, off);
        mu += __shfl_xor_sync(0xffffffffu, mu, off);
    }
    const int w = threadIdx.x >> 5;
    if ((threadIdx.x & 31) == 0) { red[0][w] = dl; red[1][w] = du; red[2][w] = ml; red[3][w] = mu; }
    __syncthreads();
    if (threadIdx.x == 0) {
        double sdl = 0, sdu = 0, sml = 0, smu = 0;
        for (int i = 0; i < (int)(blockDim.x >> 5); ++i) { sdl += red[0][i]; sdu += red[1][i]; sml += red[2][i]; smu += red[3][i]; }
        const double l = lower64[j];
        const double u = -lower64[j + nk];
        l64[j] = l;
        u64[j] = u;
        l_all[j] = __double2float_rd(l);
        u_all[j] = __double2float_ru(u);
        st_all[j] = (l >= 0.0) ? 1 : ((u <= 0.0) ? -1 : 0);
        zmag[j] = __double2float_ru(fmax(fabs(l), fabs(u)));
        const double cl = bias_raw[j] - pad_raw[j];
        const double cu = -bias_raw[j + nk] + pad_raw[j + nk];
        lc[j] = __double2float_rd(cl - sdl - ldexp(fabs(cl) + sdl + sml, -45));
        uc[j] = __double2float_ru(cu + sdu + ldexp(fabs(cu) + sdu + smu, -45));
    }
}

// concretisation operand rows and magnitude scales
__global__ void k_build_pc(int U, int n0, const float* lA, const float* lc, const float* uA, const float* uc,
                           const float* xmag, float* PC, float* PCc, float* pscale, float* amax) {
    const int c = blockIdx.x;  // 0..2U-1
    if (c >= 2 * U) return;
    const bool up = c >= U;
    const int s = up ? c - U : c;
    const float* A = up ? uA : lA;
    double mag = 0.0;
    float vmax = 0.f;
    for (int q = threadIdx.x; q < n0; q += blockDim.x) {
        const float v = A[(size_t)s * n0 + q];
        vmax = fmaxf(vmax, fabsf(v));
        const float pos = fmaxf(v, 0.f), neg = fminf(v, 0.f);
        // lower: [A+ | A-] against [lo | hi];  upper: [A- | A+]
        PC[(size_t)c * 2 * n0 + q] = up ? neg : pos;
        PC[(size_t)c * 2 * n0 + n0 + q] = up ? pos : neg;
        mag += (double)fabsf(v) * (double)xmag[q];
    }
    __shared__ double red[32];
    __shared__ float redm[32];
    for (int off = 16; off > 0; off >>= 1) {
        mag += __shfl_xor_sync(0xffffffffu, mag, off);
        vmax = fmaxf(vmax, __shfl_xor_sync(0xffffffffu, vmax, off));
    }
    if ((threadIdx.x & 31) == 0) { red[threadIdx.x >> 5] = mag; redm[threadIdx.x >> 5] = vmax; }
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        float m = 0.f;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) { t += red[w]; m = fmaxf(m, redm[w]); }
        amax[c] = m;
        const float cc = up ? uc[s] : lc[s];
        PCc[c] = cc;
        pscale[c] = __double2float_ru((t + fabs((double)cc)) * (1.0 + 1e-12));
    }
}

__global__ void k_slot_of(int H, int U, const int* ids, int* slot_of) {
    int g = blockIdx.x * blockDim.x + threadIdx.x;
    if (g < H) slot_of[g] = -1;
}
__global__ void k_slot_set(int U, const int* ids, int* slot_of) {
    int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c < U) slot_of[ids[c]] = c;
}

template <typename T>
cv_status dalloc(T** p, size_t n) {
    if (n == 0) n = 1;
    cudaError_t e = cudaMalloc((void**)p, n * sizeof(T));
    if (e != cudaSuccess) { *p = nullptr; return cv_cuda_fail(e, "cudaMalloc"); }
    return CV_OK;
}

void cache_free(cv_cache* c) {
    if (!c) return;
    cudaFree(c->ids); cudaFree(c->slot_of); cudaFree(c->lA); cudaFree(c->lc); cudaFree(c->uA);
    cudaFree(c->uc); cudaFree(c->PC); cudaFree(c->PCc); cudaFree(c->pscale); cudaFree(c->amax); cudaFree(c->root_l);
    cudaFree(c->root_u); cudaFree(c->root_state); cudaFree(c->root_lo); cudaFree(c->root_hi);
    for (int i = 0; i <= CV_MAX_LAYERS; ++i) cudaFree(c->V[i]);
    cv_tc_release(c);
    delete c;
}

}  // namespace

// ---------------------------------------------------------------- network
static void conv_dense(const cv_layer_desc& d, std::vector<float>& W, std::vector<float>& b) {
    const int ni = d.in_c * d.in_h * d.in_w, no = d.out_c * d.out_h * d.out_w;
    W.assign((size_t)no * ni, 0.f);
    b.assign(no, 0.f);
    for (int oc = 0; oc < d.out_c; ++oc)
        for (int oy = 0; oy < d.out_h; ++oy)
            for (int ox = 0; ox < d.out_w; ++ox) {
                const int r = (oc * d.out_h + oy) * d.out_w + ox;
                b[r] = d.bias[oc];
                for (int ic = 0; ic < d.in_c; ++ic)
                    for (int ky = 0; ky < d.k; ++ky) {
                        const int iy = oy * d.stride - d.pad + ky;
                        if (iy < 0 || iy >= d.in_h) continue;
                        for (int kx = 0; kx < d.k; ++kx) {
                            const int ix = ox * d.stride - d.pad + kx;
                            if (ix < 0 || ix >= d.in_w) continue;
                            W[(size_t)r * ni + (ic * d.in_h + iy) * d.in_w + ix] +=
                                d.weight[(((size_t)oc * d.in_c + ic) * d.k + ky) * d.k + kx];
                        }
                    }
            }
}

extern "C" cv_status cv_net_create(const cv_layer_desc* layers, int n_layers, cv_net** out) {
    if (!layers || !out || n_layers < 1 || n_layers > CV_MAX_LAYERS) {
        cv_set_error("cv_net_create: bad arguments");
        return CV_EINVAL;
    }
    *out = nullptr;
    cv_net* n = new cv_net();
    memset(n, 0, sizeof(*n));
    n->L = n_layers;
    cudaGetDevice(&n->device);
    for (int i = 0; i < n_layers; ++i) {
        const cv_layer_desc& d = layers[i];
        if (!d.weight || !d.bias || (d.kind != CV_LAYER_DENSE && d.kind != CV_LAYER_CONV2D)) {
            delete n;
            cv_set_error("cv_net_create: layer " + std::to_string(i) + ": null weight/bias or unknown kind");
            return CV_EINVAL;
        }
        int ni, no;
        if (d.kind == CV_LAYER_DENSE) { ni = d.in_c; no = d.out_c; }
        else {
            ni = d.in_c * d.in_h * d.in_w; no = d.out_c * d.out_h * d.out_w;
            if (d.k <= 0 || d.stride <= 0 || d.pad < 0 ||
                (d.in_h + 2 * d.pad - d.k) / d.stride + 1 != d.out_h ||
                (d.in_w + 2 * d.pad - d.k) / d.stride + 1 != d.out_w) {
                delete n;
                cv_set_error("cv_net_create: conv layer " + std::to_string(i) + ": inconsistent shape");
                return CV_ESHAPE;
            }
        }
        if (ni <= 0 || no <= 0 || (i > 0 && ni != n->dims[i])) {
            delete n;
            cv_set_error("cv_net_create: layer " + std::to_string(i) + ": width mismatch");
            return CV_ESHAPE;
        }
        n->dims[i] = ni;
        n->dims[i + 1] = no;
    }
    int ho = 0;
    n->wmax = 0;
    for (int i = 0; i <= n_layers; ++i) n->wmax = n->dims[i] > n->wmax ? n->dims[i] : n->wmax;
    for (int i = 1; i <= n_layers; ++i) {
        n->hoff[i] = ho;
        if (i < n_layers) ho += n->dims[i];
    }
    n->H = ho;
    for (int i = 1; i <= n_layers; ++i) {
        const cv_layer_desc& d = layers[i - 1];
        std::vector<float> W, b;
        const float* Wp = d.weight;
        const float* bp = d.bias;
        if (d.kind == CV_LAYER_CONV2D) { conv_dense(d, W, b); Wp = W.data(); bp = b.data(); }
        size_t nw = (size_t)n->dims[i] * n->dims[i - 1];
        if (dalloc(&n->W[i], nw) || dalloc(&n->b[i], (size_t)n->dims[i])) { cv_net_destroy(n); return CV_ENOMEM; }
        cudaMemcpy(n->W[i], Wp, nw * sizeof(float), cudaMemcpyHostToDevice);
        cudaMemcpy(n->b[i], bp, n->dims[i] * sizeof(float), cudaMemcpyHostToDevice);
    }
    // the device status word and, after it, cv_batch_check's result word
    if (dalloc(&n->status, 2)) { cv_net_destroy(n); return CV_ENOMEM; }
    CV_CUDA(cudaMemset(n->status, 0, 2 * sizeof(int)));
    CV_CUDA(cudaDeviceSynchronize());
    *out = n;
    return CV_OK;
}

extern "C" void cv_net_destroy(cv_net* n) {
    if (!n) return;
    for (int i = 0; i <= CV_MAX_LAYERS; ++i) { cudaFree(n->W[i]); cudaFree(n->b[i]); }
    cudaFree(n->status);
    delete n;
}

extern "C" cv_status cv_net_dims(const cv_net* n, int* n_layers, int* dims, int* n_hidden) {
    if (!n) { cv_set_error("cv_net_dims: null net"); return CV_EINVAL; }
    if (n_layers) *n_layers = n->L;
    if (dims) for (int i = 0; i <= n->L; ++i) dims[i] = n->dims[i];
    if (n_hidden) *n_hidden = n->H;
    return CV_OK;
}

extern "C" cv_status cv_device_status(cv_net* n, void* stream, int* code) {
    if (!n) { cv_set_error("cv_device_status: null net"); return CV_EINVAL; }
    cudaStream_t st = (cudaStream_t)stream;
    CV_CUDA(cudaStreamSynchronize(st));
    int h = 0;
    CV_CUDA(cudaMemcpy(&h, n->status, sizeof(int), cudaMemcpyDeviceToHost));
    CV_CUDA(cudaMemset(n->status, 0, sizeof(int)));
    if (code) *code = h;
    if (h) {
        cv_set_error("a kernel flagged a bad input (device status " + std::to_string(h) + ")");
        return CV_EDEVICE;
    }
    return CV_OK;
}

// ---------------------------------------------------------------- cache
// Derived tables: slot_of, PC/PCc/pscale (concretisation operand), V (pad weights).
// Needs: U, ids, planes, root_l/u/state, root box.
static cv_status finish_cache(cv_cache* c, cudaStream_t st) {
    const cv_net* n = c->net;
    const int H = n->H, U = c->U, n0 = c->n0;
    if (dalloc(&c->slot_of, H) || dalloc(&c->PC, (size_t)2 * U * 2 * n0) || dalloc(&c->PCc, 2 * U) ||
        dalloc(&c->pscale, 2 * U) || dalloc(&c->amax, 2 * U))
        return CV_ENOMEM;
    k_slot_of<<<(H + 255) / 256, 256, 0, st>>>(H, U, c->ids, c->slot_of);
    if (U > 0) k_slot_set<<<(U + 255) / 256, 256, 0, st>>>(U, c->ids, c->slot_of);
    float* xmag = nullptr;
    if (dalloc(&xmag, n0)) return CV_ENOMEM;
    k_absmax<<<(n0 + 255) / 256, 256, 0, st>>>(n0, c->root_lo, c->root_hi, xmag);
    if (U > 0)
        k_build_pc<<<2 * U, 256, 0, st>>>(U, n0, c->lA, c->lc, c->uA, c->uc, xmag, c->PC, c->PCc, c->pscale, c->amax);
    // V^(i) = |W^(i)| zmag^(i-1) + |b^(i)|; zmag^(0) = xmag, zmag^(i) = max(|l|,|u|) of layer i
    float* zmag = nullptr;
    if (dalloc(&zmag, H > 0 ? H : 1)) { cudaFree(xmag); return CV_ENOMEM; }
    if (H > 0) k_absmax<<<(H + 255) / 256, 256, 0, st>>>(H, c->root_l, c->root_u, zmag);
    for (int i = 1; i <= n->L; ++i) {
        if (!c->V[i] && dalloc(&c->V[i], n->dims[i])) { cudaFree(xmag); cudaFree(zmag); return CV_ENOMEM; }
        const float* zm = (i == 1) ? xmag : zmag + n->hoff[i - 1];
        dim3 blk(32, 8);
        k_padweights<<<(n->dims[i] + 7) / 8, blk, 0, st>>>(n->dims[i], n->dims[i - 1], n->W[i], n->b[i], zm, c->V[i]);
    }
    CV_LAUNCH_CHECK("cache tables");
    cv_status s = cv_tc_prepare(c, xmag, zmag, st);
    CV_CUDA(cudaStreamSynchronize(st));
    cudaFree(xmag);
    cudaFree(zmag);
    return s;
}

static cv_status new_cache(cv_net* net, cv_cache** out) {
    cv_cache* c = new cv_cache();
    memset(c, 0, sizeof(*c));
    c->net = net;
    c->cc_items[0] = CV_CC_ITEMS_1;
    c->cc_items[1] = CV_CC_ITEMS_2;
    c->cc_items[2] = CV_CC_ITEMS_3;
    c->n0 = net->dims[0];
    c->H = net->H;
    *out = c;
    if (dalloc(&c->root_l, net->H) || dalloc(&c->root_u, net->H) || dalloc(&c->root_state, net->H) ||
        dalloc(&c->root_lo, c->n0) || dalloc(&c->root_hi, c->n0))
        return CV_ENOMEM;
    return CV_OK;
}

__global__ void k_gather_unstable(int H, int n0, const int* ids, int U, const float* AL, const float* CL,
                                  const float* AU, const float* CU, float* lA, float* lc, float* uA, float* uc) {
    const int c = blockIdx.x;
    if (c >= U) return;
    const int g = ids[c];
    for (int q = threadIdx.x; q < n0; q += blockDim.x) {
        lA[(size_t)c * n0 + q] = AL[(size_t)g * n0 + q];
        uA[(size_t)c * n0 + q] = AU[(size_t)g * n0 + q];
    }
    if (threadIdx.x == 0) { lc[c] = CL[g]; uc[c] = CU[g]; }
}

extern "C" cv_status cv_cache_build(cv_net* net, const float* root_lo, const float* root_hi,
                                    int alpha_mode, cv_cache** out, void* stream) {
    if (!net || !root_lo || !root_hi || !out || alpha_mode < 0 || alpha_mode > 2) {
        cv_set_error("cv_cache_build: bad arguments");
        return CV_EINVAL;
    }
    cudaStream_t st = (cudaStream_t)stream;
    cv_cache* c = nullptr;
    *out = nullptr;
    cv_status s = new_cache(net, &c);
    if (s) { cache_free(c); return s; }
    const int n0 = c->n0, H = net->H, L = net->L;
    CV_CUDA(cudaMemcpyAsync(c->root_lo, root_lo, n0 * sizeof(float), cudaMemcpyDeviceToDevice, st));
    CV_CUDA(cudaMemcpyAsync(c->root_hi, root_hi, n0 * sizeof(float), cudaMemcpyDeviceToDevice, st));
    // FP64 back-substitution for every hidden layer; planes of all hidden neurons (temporary)
    float *AL = nullptr, *CL = nullptr, *AU = nullptr, *CU = nullptr, *xmag = nullptr, *zmag = nullptr;
    double *l64 = nullptr, *u64 = nullptr;
    int nkmax = 1;
    for (int k = 1; k < L; ++k) nkmax = net->dims[k] > nkmax ? net->dims[k] : nkmax;
    const int R = 2 * nkmax;
    const int ncb = cv_bwd_ncb_max(net);
    double *lamA = nullptr, *lamB = nullptr, *lam0 = nullptr, *lower64 = nullptr;
    double *pb = nullptr, *pp = nullptr, *pf = nullptr, *pm = nullptr, *ab = nullptr, *ap = nullptr, *br = nullptr, *pr = nullptr;
    bool ok = !(dalloc(&AL, (size_t)(H ? H : 1) * n0) || dalloc(&CL, H) || dalloc(&AU, (size_t)(H ? H : 1) * n0) ||
                dalloc(&CU, H) || dalloc(&xmag, n0) || dalloc(&zmag, H) || dalloc(&l64, H) || dalloc(&u64, H) ||
                dalloc(&lamA, (size_t)R * net->wmax) || dalloc(&lamB, (size_t)R * net->wmax) ||
                dalloc(&lam0, (size_t)R * n0) || dalloc(&lower64, R) || dalloc(&pb, (size_t)R * ncb) ||
                dalloc(&pp, (size_t)R * ncb) || dalloc(&pf, (size_t)R * ncb) || dalloc(&pm, (size_t)R * ncb) ||
                dalloc(&ab, R) || dalloc(&ap, R) || dalloc(&br, R) || dalloc(&pr, R));
    for (int i = 1; i <= L && ok; ++i) ok = !dalloc(&c->V[i], net->dims[i]);
    auto cleanup = [&]() {
        cudaFree(AL); cudaFree(CL); cudaFree(AU); cudaFree(CU); cudaFree(xmag); cudaFree(zmag); cudaFree(l64);
        cudaFree(u64); cudaFree(lamA); cudaFree(lamB); cudaFree(lam0); cudaFree(lower64); cudaFree(pb);
        cudaFree(pp); cudaFree(pf); cudaFree(pm); cudaFree(ab); cudaFree(ap); cudaFree(br); cudaFree(pr);
    };
    if (!ok) { cleanup(); cache_free(c); return CV_ENOMEM; }
    k_absmax<<<(n0 + 255) / 256, 256, 0, st>>>(n0, c->root_lo, c->root_hi, xmag);
    {
        dim3 blk(32, 8);
        k_padweights<<<(net->dims[1] + 7) / 8, blk, 0, st>>>(net->dims[1], n0, net->W[1], net->b[1], xmag, c->V[1]);
    }
    for (int k = 1; k < L; ++k) {
        const int nk = net->dims[k], ho = net->hoff[k];
        s = cv_backward_t<double>(net, 2 * nk, 2 * nk, k, 2, 1, nullptr, nullptr, nullptr, l64, u64,
                                  c->root_state, nullptr, nullptr, nullptr, nullptr, 0, nullptr, alpha_mode, c->V,
                                  c->root_lo, c->root_hi, nullptr, nullptr, lower64, nullptr, lam0, nullptr, br, pr,
                                  lamA, lamB, pb, pp, pf, pm, ab, ap, nullptr, st);
        if (s) { cleanup(); cache_free(c); return s; }
        k_root_bounds<<<nk, 256, 0, st>>>(nk, n0, lower64, lam0, br, pr, xmag, l64 + ho, u64 + ho, c->root_l + ho,
                                          c->root_u + ho, c->root_state + ho, zmag + ho, AL + (size_t)ho * n0,
                                          CL + ho, AU + (size_t)ho * n0, CU + ho);
        dim3 blk(32, 8);
        k_padweights<<<(net->dims[k + 1] + 7) / 8, blk, 0, st>>>(net->dims[k + 1], nk, net->W[k + 1],
                                                                  net->b[k + 1], zmag + ho, c->V[k + 1]);
        CV_LAUNCH_CHECK("root layer");
    }
    // cache the root-unstable neurons
    std::vector<int8_t> hst(H > 0 ? H : 1);
    CV_CUDA(cudaMemcpyAsync(hst.data(), c->root_state, H, cudaMemcpyDeviceToHost, st));
    CV_CUDA(cudaStreamSynchronize(st));
    std::vector<int> ids;
    for (int g = 0; g < H; ++g) if (hst[g] == 0) ids.push_back(g);
    c->U = (int)ids.size();
    const int U = c->U;
    ok = !(dalloc(&c->ids, U) || dalloc(&c->lA, (size_t)U * n0) || dalloc(&c->lc, U) ||
           dalloc(&c->uA, (size_t)U * n0) || dalloc(&c->uc, U));
    if (!ok) { cleanup(); cache_free(c); return CV_ENOMEM; }
    if (U > 0) {
        CV_CUDA(cudaMemcpyAsync(c->ids, ids.data(), U * sizeof(int), cudaMemcpyHostToDevice, st));
        k_gather_unstable<<<U, 256, 0, st>>>(H, n0, c->ids, U, AL, CL, AU, CU, c->lA, c->lc, c->uA, c->uc);
        CV_LAUNCH_CHECK("k_gather_unstable");
    }
    s = finish_cache(c, st);
    cleanup();
    if (s) { cache_free(c); return s; }
    *out = c;
    return CV_OK;
}

__global__ void k_states(int H, const float* l, const float* u, int8_t* st) {
    int g = blockIdx.x * blockDim.x + threadIdx.x;
    if (g < H) st[g] = (l[g] >= 0.f) ? 1 : ((u[g] <= 0.f) ? -1 : 0);
}

extern "C" cv_status cv_cache_create(cv_net* net, const float* root_lo, const float* root_hi,
                                     const float* root_l, const float* root_u, int U, const int* ids,
                                     const float* lA, const float* lc, const float* uA, const float* uc,
                                     cv_cache** out) {
    if (!net || !root_lo || !root_hi || !root_l || !root_u || !out || U < 0 ||
        (U > 0 && (!ids || !lA || !lc || !uA || !uc))) {
        cv_set_error("cv_cache_create: bad arguments");
        return CV_EINVAL;
    }
    const int H = net->H;
    for (int c = 0; c < U; ++c) {
        if (ids[c] < 0 || ids[c] >= H || (c > 0 && ids[c] <= ids[c - 1])) {
            cv_set_error("cv_cache_create: ids must be strictly increasing hidden ids");
            return CV_ESHAPE;
        }
    }
    *out = nullptr;
    cv_cache* c = nullptr;
    cv_status s = new_cache(net, &c);
    if (s) { cache_free(c); return s; }
    const int n0 = c->n0;
    c->U = U;
    bool ok = !(dalloc(&c->ids, U) || dalloc(&c->lA, (size_t)U * n0) || dalloc(&c->lc, U) ||
                dalloc(&c->uA, (size_t)U * n0) || dalloc(&c->uc, U));
    if (!ok) { cache_free(c); return CV_ENOMEM; }
    cudaStream_t st = 0;
    CV_CUDA(cudaMemcpy(c->root_lo, root_lo, n0 * sizeof(float), cudaMemcpyHostToDevice));
    CV_CUDA(cudaMemcpy(c->root_hi, root_hi, n0 * sizeof(float), cudaMemcpyHostToDevice));
    if (H > 0) {
        CV_CUDA(cudaMemcpy(c->root_l, root_l, H * sizeof(float), cudaMemcpyHostToDevice));
        CV_CUDA(cudaMemcpy(c->root_u, root_u, H * sizeof(float), cudaMemcpyHostToDevice));
        k_states<<<(H + 255) / 256, 256, 0, st>>>(H, c->root_l, c->root_u, c->root_state);
    }
    if (U > 0) {
        CV_CUDA(cudaMemcpy(c->ids, ids, U * sizeof(int), cudaMemcpyHostToDevice));
        CV_CUDA(cudaMemcpy(c->lA, lA, (size_t)U * n0 * sizeof(float), cudaMemcpyHostToDevice));
        CV_CUDA(cudaMemcpy(c->lc, lc, U * sizeof(float), cudaMemcpyHostToDevice));
        CV_CUDA(cudaMemcpy(c->uA, uA, (size_t)U * n0 * sizeof(float), cudaMemcpyHostToDevice));
        CV_CUDA(cudaMemcpy(c->uc, uc, U * sizeof(float), cudaMemcpyHostToDevice));
    }
    s = finish_cache(c, st);
    if (s) { cache_free(c); return s; }
    *out = c;
    return CV_OK;
}

extern "C" cv_status cv_cache_size(const cv_cache* c, int* U) {
    if (!c || !U) { cv_set_error("cv_cache_size: bad arguments"); return CV_EINVAL; }
    *U = c->U;
    return CV_OK;
}

extern "C" cv_status cv_cache_read(const cv_cache* c, int* ids, float* lA, float* lc, float* uA, float* uc,
                                   float* root_l, float* root_u) {
    if (!c) { cv_set_error("cv_cache_read: null cache"); return CV_EINVAL; }
    CV_CUDA(cudaDeviceSynchronize());
    const size_t U = c->U, n0 = c->n0, H = c->H;
    if (ids && U) CV_CUDA(cudaMemcpy(ids, c->ids, U * sizeof(int), cudaMemcpyDeviceToHost));
    if (lA && U) CV_CUDA(cudaMemcpy(lA, c->lA, U * n0 * sizeof(float), cudaMemcpyDeviceToHost));
    if (lc && U) CV_CUDA(cudaMemcpy(lc, c->lc, U * sizeof(float), cudaMemcpyDeviceToHost));
    if (uA && U) CV_CUDA(cudaMemcpy(uA, c->uA, U * n0 * sizeof(float), cudaMemcpyDeviceToHost));
    if (uc && U) CV_CUDA(cudaMemcpy(uc, c->uc, U * sizeof(float), cudaMemcpyDeviceToHost));
    if (root_l && H) CV_CUDA(cudaMemcpy(root_l, c->root_l, H * sizeof(float), cudaMemcpyDeviceToHost));
    if (root_u && H) CV_CUDA(cudaMemcpy(root_u, c->root_u, H * sizeof(float), cudaMemcpyDeviceToHost));
    return CV_OK;
}

extern "C" void cv_cache_destroy(cv_cache* c) { cache_free(c); }
