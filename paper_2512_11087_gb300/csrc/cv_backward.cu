// CROWN back-substitution (the Omega recursion of the paper's Appendix "Formulating
// bounding hyperplanes", with the ReLU relaxation Lemma) for a batch of rows, and the
// final concretisation over each row's box (Lemma A.1).
//
// One step per affine layer i = k..1:   P = Lam^(i) W^(i)   (rows x n_{i-1})
//   i > 1 : Lam^(i-1)_q = P_q d_q, bias += P_q e_q   (d, e from the relaxation of neuron q
//           of hidden layer i-1, chosen by the sign of P_q), bias += Lam^(i-1) . b^(i-1)
//   i = 1 : f = sum_q min(P_q lo_q, P_q hi_q) + bias
// Two instantiations of the same kernels:
//  T = float  (the per-round spec bound): P is accumulated in FP32 chains of at most 32 FMAs whose
//    results are summed with a compensated (TwoSum) accumulator, so |P~ - P| <= (33 u) sum_j
//    |Lam_j||W_jq| (u = 2^-24).  Every step adds gamma * |Lam^(i)| V^(i) to the pad,
//    V^(i) = |W^(i)| zmag^(i-1) + |b^(i)| with zmag a bound on |z^(i-1)| over the root box;
//    gamma = 48 u covers the product chain, the relaxation products and the FP32 partial sums of
//    the epilogue.
//  T = double (the once-per-property root cache): the same recursion in FP64, gamma = 2^-40.
// Row sums (bias, pad, final concretisation) are FP64 in both.
#include "cv_internal.cuh"

#include <math.h>

namespace {

constexpr int BM = 64, BN = 64, BK = 16, KC_TILES = 2;  // KC = 32 FMAs per FP32 chain

template <typename T> struct Gam;
template <> struct Gam<float> { static constexpr double v = 48.0 * CV_U32; };
template <> struct Gam<double> { static constexpr double v = 9.094947017729282e-13; };  // 2^-40

template <typename T>
struct LayerArgs {
    const T* A;        // Lam^(i) [R x K]
    const float* W;    // W^(i) [K x N]
    int R, K, N, i;    // i: layer index of W
    int rows_per_sub, m;
    int hoff;          // first global id of hidden layer i-1
    int H;
    const T* root_l; const T* root_u; const int8_t* root_state;
    const int* slot_of; const T* l; const T* u; const int8_t* mask; int U;
    const float* alpha; int alpha_mode;
    const float* bnext;   // b^(i-1) [N]
    const float* Vnext;   // V^(i-1) [N]
    T* Aout;              // Lam^(i-1) [R x N]
    const float* lo; const float* hi;  // [nsub x N] (i == 1)
    T* lam0;              // optional [R x N]
    T* keepP;             // optional [R x N]: the product P^(i) (i > 1), kept for the alpha adjoint
    const float* beta;    // optional [nsub x m x H] split multipliers (with bsign [nsub x H])
    const int8_t* bsign;
    double* part_bias; double* part_pad; double* part_f; double* part_fmag; int ncb;
};

__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
    s = a + b;
    float bp = s - a;
    e = (a - (s - bp)) + (b - bp);
}

template <typename T>
__device__ __forceinline__ T tabs(T x) { return x < T(0) ? -x : x; }

// lam - sign beta, rounded away from lam (down for sign +1, up for -1): the multiplier in effect,
// |result - lam|, is then at least beta >= 0, so the bound stays valid
__device__ __forceinline__ float beta_shift(float lam, int sg, float bt) {
    return sg > 0 ? __fsub_rd(lam, bt) : __fadd_ru(lam, bt);
}
__device__ __forceinline__ double beta_shift(double lam, int sg, float bt) {
    return sg > 0 ? __dsub_rd(lam, (double)bt) : __dadd_ru(lam, (double)bt);
}

template <typename T>
__global__ void __launch_bounds__(256) k_bwd_layer(LayerArgs<T> a) {
    __shared__ T As[BK][BM + 4];
    __shared__ T Bs[BK][BN + 4];
    const int tid = threadIdx.x;
    const int tx = tid & 15, ty = tid >> 4;
    const int row0 = blockIdx.y * BM, col0 = blockIdx.x * BN;
    constexpr bool F32 = sizeof(T) == 4;

    T acc[4][4], tot[4][4], cmp[4][4];
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) { acc[i][j] = T(0); tot[i][j] = T(0); cmp[i][j] = T(0); }

    const int ntiles = (a.K + BK - 1) / BK;
    for (int kt = 0; kt < ntiles; ++kt) {
        const int k0 = kt * BK;
#pragma unroll
        for (int e = 0; e < 4; ++e) {
            int idx = tid * 4 + e;
            int r = idx >> 4, kk = idx & 15;
            int gr = row0 + r, gk = k0 + kk;
            As[kk][r] = (gr < a.R && gk < a.K) ? a.A[(size_t)gr * a.K + gk] : T(0);
        }
#pragma unroll
        for (int e = 0; e < 4; ++e) {
            int idx = tid * 4 + e;
            int kk = idx >> 6, c = idx & 63;
            int gk = k0 + kk, gc = col0 + c;
            Bs[kk][c] = (gk < a.K && gc < a.N) ? (T)a.W[(size_t)gk * a.N + gc] : T(0);
        }
        __syncthreads();
#pragma unroll
        for (int kk = 0; kk < BK; ++kk) {
            T av[4], bv[4];
#pragma unroll
            for (int i = 0; i < 4; ++i) av[i] = As[kk][ty * 4 + i];
#pragma unroll
            for (int j = 0; j < 4; ++j) bv[j] = Bs[kk][tx * 4 + j];
#pragma unroll
            for (int i = 0; i < 4; ++i)
#pragma unroll
                for (int j = 0; j < 4; ++j) acc[i][j] = fma(av[i], bv[j], acc[i][j]);
        }
        __syncthreads();
        if (F32 && ((kt % KC_TILES) == KC_TILES - 1 || kt == ntiles - 1)) {
#pragma unroll
            for (int i = 0; i < 4; ++i)
#pragma unroll
                for (int j = 0; j < 4; ++j) {
                    float s, e;
                    two_sum((float)tot[i][j], (float)acc[i][j], s, e);
                    tot[i][j] = s;
                    cmp[i][j] += e;
                    acc[i][j] = T(0);
                }
        }
    }
    if (!F32) {
#pragma unroll
        for (int i = 0; i < 4; ++i)
#pragma unroll
            for (int j = 0; j < 4; ++j) tot[i][j] = acc[i][j];
    }

    double pb[4], pp[4], pf[4], pm[4];
#pragma unroll
    for (int i = 0; i < 4; ++i) { pb[i] = 0.0; pp[i] = 0.0; pf[i] = 0.0; pm[i] = 0.0; }
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        const int r = row0 + ty * 4 + i;
        if (r >= a.R) continue;
        const int sub = r / a.rows_per_sub;
        T bsum = T(0), psum = T(0);
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const int q = col0 + tx * 4 + j;
            if (q >= a.N) continue;
            const T p = tot[i][j] + cmp[i][j];
            if (a.i > 1) {
                const int g = a.hoff + q;
                T l, u; int st;
                int slot = (a.slot_of && a.l) ? a.slot_of[g] : -1;
                if (slot >= 0) {
                    size_t o = (size_t)sub * a.U + slot;
                    l = a.l[o]; u = a.u[o]; st = a.mask[o];
                } else {
                    l = a.root_l[g]; u = a.root_u[g]; st = a.root_state[g];
                }
                T d, e;
                if (st > 0) { d = T(1); e = T(0); }
                else if (st < 0) { d = T(0); e = T(0); }
                else if (p >= T(0)) {
                    if (a.alpha) d = (T)a.alpha[((size_t)sub * a.m + (r % a.m)) * a.H + g];
                    else d = (a.alpha_mode == CV_ALPHA_ONE) ? T(1)
                           : (a.alpha_mode == CV_ALPHA_ZERO) ? T(0) : ((u >= -l) ? T(1) : T(0));
                    e = T(0);
                } else {
                    const T s = u / (u - l);
                    d = s;
                    e = -s * l;
                }
                T lam = p * d;
                if (a.bsign) {  // split multiplier: Lam_g -= sign_g beta_g
                    const int sg = a.bsign[(size_t)sub * a.H + g];
                    if (sg) lam = beta_shift(lam, sg, a.beta[((size_t)sub * a.m + (r % a.m)) * a.H + g]);
                }
                a.Aout[(size_t)r * a.N + q] = lam;
                if (a.keepP) a.keepP[(size_t)r * a.N + q] = p;
                bsum = fma(p, e, bsum);
                bsum = fma(lam, (T)a.bnext[q], bsum);
                psum = fma(tabs(lam), (T)a.Vnext[q], psum);
            } else {
                const size_t o = (size_t)sub * a.N + q;
                const double lo = (double)a.lo[o], hi = (double)a.hi[o];
                const double pd = (double)p;
                pf[i] += fmin(pd * lo, pd * hi);
                pm[i] += fabs(pd) * fmax(fabs(lo), fabs(hi));
                if (a.lam0) a.lam0[(size_t)r * a.N + q] = p;
            }
        }
        pb[i] = (double)bsum;
        pp[i] = (double)psum;
    }
#pragma unroll
    for (int i = 0; i < 4; ++i) {
#pragma unroll
        for (int off = 8; off > 0; off >>= 1) {
            pb[i] += __shfl_xor_sync(0xffffffffu, pb[i], off);
            pp[i] += __shfl_xor_sync(0xffffffffu, pp[i], off);
            pf[i] += __shfl_xor_sync(0xffffffffu, pf[i], off);
            pm[i] += __shfl_xor_sync(0xffffffffu, pm[i], off);
        }
    }
    if (tx == 0) {
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            const int r = row0 + ty * 4 + i;
            if (r >= a.R) continue;
            const size_t o = (size_t)r * a.ncb + blockIdx.x;
            if (a.i > 1) { a.part_bias[o] = pb[i]; a.part_pad[o] = pp[i]; }
            else { a.part_f[o] = pf[i]; a.part_fmag[o] = pm[i]; }
        }
    }
}

// Initial Lam^(k), its bias term and its pad weight.
template <typename T>
__global__ void k_bwd_init(int R, int nk, int mode, int m, const float* lam_init, const float* C,
                           const float* t, const float* bk, const float* Vk, T* A,
                           double* acc_bias, double* acc_pad, double gam) {
    const int r = blockIdx.x * blockDim.y + threadIdx.y;
    if (r >= R) return;
    double bs = 0.0, ps = 0.0;
    for (int q = threadIdx.x; q < nk; q += 32) {
        float v;
        if (mode == 0) v = lam_init[(size_t)r * nk + q];
        else if (mode == 1) v = C[(size_t)(r % m) * nk + q];
        else v = (q == r % nk) ? (((r / nk) & 1) ? -1.f : 1.f) : 0.f;
        A[(size_t)r * nk + q] = (T)v;
        bs += (double)v * (double)bk[q];
        ps += (double)fabsf(v) * (double)Vk[q];
    }
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
        bs += __shfl_xor_sync(0xffffffffu, bs, off);
        ps += __shfl_xor_sync(0xffffffffu, ps, off);
    }
    if (threadIdx.x == 0) {
        double t0 = (mode == 1 && t) ? (double)t[r % m] : 0.0;
        acc_bias[r] = t0 + bs;
        acc_pad[r] = gam * ps;
    }
}

__global__ void k_bwd_reduce(int R, int ncb, double gam, const double* part_bias, const double* part_pad,
                             double* acc_bias, double* acc_pad) {
    const int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= R) return;
    double b = 0.0, p = 0.0;
    for (int c = 0; c < ncb; ++c) { b += part_bias[(size_t)r * ncb + c]; p += part_pad[(size_t)r * ncb + c]; }
    acc_bias[r] += b;
    acc_pad[r] += gam * p;
}

// final: f = sum min(P lo, P hi) + bias - pad  (FP64), rounded down to FP32
__global__ void k_bwd_final(int R, int ncb, int rows_per_sub, const double* part_f,
                            const double* part_fmag, const double* acc_bias, const double* acc_pad,
                            const uint8_t* skip, float* lower, double* lower64, float* err, float* bias_out,
                            double* bias_raw, double* pad_raw, double fm_gamma) {
    const int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= R) return;
    double f = 0.0, fm = 0.0;
    for (int c = 0; c < ncb; ++c) { f += part_f[(size_t)r * ncb + c]; fm += part_fmag[(size_t)r * ncb + c]; }
    // FP64 rounding of the sums above and of the bias accumulation: <= 2^-40 of the magnitudes
    const double b = acc_bias[r];
    const double pad = acc_pad[r] * (1.0 + 1e-6) + fm_gamma * fm + ldexp(fm + fabs(b) + acc_pad[r], -40);
    const double v = f + b - pad;
    const bool sk = skip && skip[r / rows_per_sub];
    if (lower) lower[r] = sk ? INFINITY : __double2float_rd(v);
    if (lower64) lower64[r] = sk ? INFINITY : v;
    if (err) err[r] = sk ? 0.f : __double2float_ru(pad);
    if (bias_out) bias_out[r] = __double2float_rd(b - pad);
    if (bias_raw) bias_raw[r] = b;
    if (pad_raw) pad_raw[r] = pad;
}

// BaBSR weight of hidden layer i-1 (Appendix, neuron selection heuristic): thread per (subdomain,
// neuron) of the layer, the m rows of the subdomain summed in increasing order (coalesced over q)
__global__ void k_babsr_weight(int nsub, int m, int N, int hoff, const int* slot_of, int U, const float* P,
                               const uint8_t* skip, float* w) {
    const size_t x = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (x >= (size_t)nsub * N) return;
    const int sub = (int)(x / N), q = (int)(x % N);
    const int slot = slot_of[hoff + q];
    if (slot < 0 || (skip && skip[sub])) return;  // infeasible subdomains keep the zeros
    float s = 0.f;
    for (int r = 0; r < m; ++r) s = __fadd_rn(s, P[((size_t)sub * m + r) * N + q]);
    w[(size_t)sub * U + slot] = __fdiv_rn(s, (float)m);
}

}  // namespace

cv_status cv_babsr_weight_layer(int nsub, int m, int N, int hoff, const int* slot_of, int U, const float* P,
                                const uint8_t* skip, float* w, cudaStream_t st) {
    const size_t n = (size_t)nsub * N;
    if (n == 0 || m <= 0 || U <= 0) return CV_OK;
    k_babsr_weight<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(nsub, m, N, hoff, slot_of, U, P, skip, w);
    CV_LAUNCH_CHECK("k_babsr_weight");
    return CV_OK;
}

template <typename T>
cv_status cv_backward_t(const cv_net* net, int R, int rows_per_sub, int k, int init_mode, int m,
                        const float* lam_init, const float* C, const float* t,
                        const T* root_l, const T* root_u, const int8_t* root_state,
                        const int* slot_of, const T* l, const T* u, const int8_t* mask,
                        int U, const float* alpha, int alpha_mode, float* const* V,
                        const float* lo, const float* hi, const uint8_t* skip,
                        float* lower, double* lower64, float* err, T* lam0, float* bias_out,
                        double* bias_raw, double* pad_raw,
                        T* lamA, T* lamB, double* part_bias, double* part_pad,
                        double* part_f, double* part_fmag, double* acc_bias, double* acc_pad,
                        T* const* keepP, cudaStream_t st, float* bab_weight, const float* beta,
                        const int8_t* bsign) {
    const int nk = net->dims[k];
    {
        dim3 blk(32, 8);
        dim3 grd((R + 7) / 8);
        k_bwd_init<T><<<grd, blk, 0, st>>>(R, nk, init_mode, m, lam_init, C, t, net->b[k], V[k], lamA,
                                            acc_bias, acc_pad, Gam<T>::v);
        CV_LAUNCH_CHECK("k_bwd_init");
    }
    T* cur = lamA;
    T* nxt = lamB;
    for (int i = k; i >= 1; --i) {
        LayerArgs<T> a;
        a.A = cur; a.W = net->W[i];
        a.R = R; a.K = net->dims[i]; a.N = net->dims[i - 1]; a.i = i;
        a.rows_per_sub = rows_per_sub; a.m = m > 0 ? m : 1;
        a.hoff = (i > 1) ? net->hoff[i - 1] : 0;
        a.H = net->H;
        a.root_l = root_l; a.root_u = root_u; a.root_state = root_state;
        a.slot_of = slot_of; a.l = l; a.u = u; a.mask = mask; a.U = U;
        a.alpha = alpha; a.alpha_mode = alpha_mode;
        a.bnext = (i > 1) ? net->b[i - 1] : nullptr;
        a.Vnext = (i > 1) ? V[i - 1] : nullptr;
        a.Aout = nxt;
        a.lo = lo; a.hi = hi; a.lam0 = lam0;
        a.keepP = (keepP && i > 1) ? keepP[i] : nullptr;
        a.beta = (i > 1) ? beta : nullptr;
        a.bsign = (i > 1 && beta) ? bsign : nullptr;
        a.ncb = (a.N + BN - 1) / BN;
        a.part_bias = part_bias; a.part_pad = part_pad; a.part_f = part_f; a.part_fmag = part_fmag;
        dim3 grd(a.ncb, (R + BM - 1) / BM);
        k_bwd_layer<T><<<grd, 256, 0, st>>>(a);
        CV_LAUNCH_CHECK("k_bwd_layer");
        if (i > 1) {
            k_bwd_reduce<<<(R + 255) / 256, 256, 0, st>>>(R, a.ncb, Gam<T>::v, part_bias, part_pad, acc_bias,
                                                          acc_pad);
            CV_LAUNCH_CHECK("k_bwd_reduce");
            if constexpr (sizeof(T) == sizeof(float)) {
                if (bab_weight && a.keepP && m > 0 && rows_per_sub == m) {
                    cv_status s = cv_babsr_weight_layer(R / m, m, a.N, a.hoff, slot_of, U, (const float*)a.keepP,
                                                        skip, bab_weight, st);
                    if (s) return s;
                }
            }
            T* tmp = cur; cur = nxt; nxt = tmp;
        } else {
            k_bwd_final<<<(R + 255) / 256, 256, 0, st>>>(R, a.ncb, rows_per_sub, part_f, part_fmag,
                                                         acc_bias, acc_pad, skip, lower, lower64, err, bias_out,
                                                         bias_raw, pad_raw, 0.0);
            CV_LAUNCH_CHECK("k_bwd_final");
        }
    }
    return CV_OK;
}

template cv_status cv_backward_t<float>(const cv_net*, int, int, int, int, int, const float*, const float*,
                                        const float*, const float*, const float*, const int8_t*, const int*,
                                        const float*, const float*, const int8_t*, int, const float*, int,
                                        float* const*, const float*, const float*, const uint8_t*, float*,
                                        double*, float*, float*, float*, double*, double*, float*, float*,
                                        double*, double*, double*, double*, double*, double*, float* const*,
                                        cudaStream_t, float*, const float*, const int8_t*);
template cv_status cv_backward_t<double>(const cv_net*, int, int, int, int, int, const float*, const float*,
                                         const float*, const double*, const double*, const int8_t*,
                                         const int*, const double*, const double*, const int8_t*, int,
                                         const float*, int, float* const*, const float*, const float*,
                                         const uint8_t*, float*, double*, float*, double*, float*, double*,
                                         double*, double*, double*, double*, double*, double*, double*,
                                         double*, double*, double* const*, cudaStream_t, float*, const float*,
                                         const int8_t*);

// number of column blocks of the widest layer (sizing of the partial buffers)
int cv_bwd_ncb_max(const cv_net* net) {
    int w = 0;
    for (int i = 0; i < net->L; ++i) w = net->dims[i] > w ? net->dims[i] : w;
    return (w + BN - 1) / BN;
}

// Launchers of the spec-bound steps shared with the tensor-core back-substitution (cv_tc.cu):
// the start from the spec rows, the per-layer reduction of the row partials (gam: the pad per unit
// of sum |Lam| V), and the final concretisation (fm_gamma: extra pad per unit of the
// concretisation's magnitude sum).
cv_status cv_bwd_spec_init(int R, int nk, int m, const float* C, const float* t, const float* bk, const float* Vk,
                           float* A, double* acc_bias, double* acc_pad, double gam, cudaStream_t st) {
    dim3 blk(32, 8);
    dim3 grd((R + 7) / 8);
    k_bwd_init<float><<<grd, blk, 0, st>>>(R, nk, 1, m, nullptr, C, t, bk, Vk, A, acc_bias, acc_pad, gam);
    CV_LAUNCH_CHECK("k_bwd_init");
    return CV_OK;
}

cv_status cv_bwd_reduce(int R, int ncb, const double* part_bias, const double* part_pad, double* acc_bias,
                        double* acc_pad, double gam, cudaStream_t st) {
    k_bwd_reduce<<<(R + 255) / 256, 256, 0, st>>>(R, ncb, gam, part_bias, part_pad, acc_bias, acc_pad);
    CV_LAUNCH_CHECK("k_bwd_reduce");
    return CV_OK;
}

cv_status cv_bwd_final(int R, int ncb, int rows_per_sub, const double* part_f, const double* part_fmag,
                       const double* acc_bias, const double* acc_pad, const uint8_t* skip, float* lower, float* err,
                       float* bias_out, double fm_gamma, cudaStream_t st) {
    k_bwd_final<<<(R + 255) / 256, 256, 0, st>>>(R, ncb, rows_per_sub, part_f, part_fmag, acc_bias, acc_pad, skip,
                                                 lower, nullptr, err, bias_out, nullptr, nullptr, fm_gamma);
    CV_LAUNCH_CHECK("k_bwd_final");
    return CV_OK;
}
