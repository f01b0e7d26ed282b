// Re-concretisation of the cached planes over each subdomain's clipped box (a5; the paper's
// Section 3.3: intermediate bounds are re-concretised over the shrunk box instead of being
// re-propagated), intersected with the inherited bounds, then the split signs and the
// stability mask.
//
// One contraction per round:  out[b, j] = [lo_b | hi_b] . PC_j + PCc_j  (K = 2 n0)
// with PC_j = [A+ | A-] of the lower plane of slot j (j < U) and [A- | A+] of the upper plane
// (j >= U), i.e. min / max of the plane over the box (Lemma A.1) without forming centre and
// radius.  FP32 chains of <= 32 FMAs with a compensated running sum: error <= 33 u of the term
// magnitudes, bounded by pscale_j = |A_j| max(|lo_root|,|hi_root|) + |c_j|; the pad is
// 40 u pscale_j.  When the padded value straddles 0 (the stability decision is uncertain) the
// bound is recomputed in FP64 from the same FP32 operands.
#include "cv_internal.cuh"

#include <math.h>

namespace {

constexpr int BM = 64, BN = 64, BK = 16, KC_TILES = 2;
constexpr double GAMMA_RC = 40.0 * CV_U32;

__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
    s = a + b;
    float bp = s - a;
    e = (a - (s - bp)) + (b - bp);
}

__global__ void __launch_bounds__(256) k_reconc(int B, int U, int n0, const float* lo, const float* hi,
                                                const float* PC, const float* PCc, const float* pscale,
                                                const float* root_l_slot, const float* root_u_slot,
                                                const float* l_in, const float* u_in, const uint8_t* infeasible,
                                                float* l_out, float* u_out) {
    __shared__ float Xs[BK][BM + 4];
    __shared__ float Ps[BK][BN + 4];
    const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
    const int b0 = blockIdx.y * BM, j0 = blockIdx.x * BN;
    const int K = 2 * n0, N = 2 * U;
    float acc[4][4], tot[4][4], cmp[4][4];
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) { acc[i][j] = 0.f; tot[i][j] = 0.f; cmp[i][j] = 0.f; }
    const int ntiles = (K + BK - 1) / BK;
    for (int kt = 0; kt < ntiles; ++kt) {
        const int k0 = kt * BK;
#pragma unroll
        for (int e = 0; e < 4; ++e) {
            const int idx = tid * 4 + e;
            const int r = idx >> 4, kk = idx & 15;
            const int gb = b0 + r, gk = k0 + kk;
            float v = 0.f;
            if (gb < B && gk < K) v = (gk < n0) ? lo[(size_t)gb * n0 + gk] : hi[(size_t)gb * n0 + gk - n0];
            Xs[kk][r] = v;
            const int gj = j0 + r;
            Ps[kk][r] = (gj < N && gk < K) ? PC[(size_t)gj * K + gk] : 0.f;
        }
        __syncthreads();
#pragma unroll
        for (int kk = 0; kk < BK; ++kk) {
            float xv[4], pv[4];
#pragma unroll
            for (int i = 0; i < 4; ++i) xv[i] = Xs[kk][ty * 4 + i];
#pragma unroll
            for (int j = 0; j < 4; ++j) pv[j] = Ps[kk][tx * 4 + j];
#pragma unroll
            for (int i = 0; i < 4; ++i)
#pragma unroll
                for (int j = 0; j < 4; ++j) acc[i][j] = fmaf(xv[i], pv[j], acc[i][j]);
        }
        __syncthreads();
        if ((kt % KC_TILES) == KC_TILES - 1 || kt == ntiles - 1) {
#pragma unroll
            for (int i = 0; i < 4; ++i)
#pragma unroll
                for (int j = 0; j < 4; ++j) {
                    float s, e;
                    two_sum(tot[i][j], acc[i][j], s, e);
                    tot[i][j] = s;
                    cmp[i][j] += e;
                    acc[i][j] = 0.f;
                }
        }
    }
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        const int b = b0 + ty * 4 + i;
        if (b >= B) continue;
        const bool skip = infeasible[b] != 0;
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const int jj = j0 + tx * 4 + j;
            if (jj >= N) continue;
            const bool up = jj >= U;
            const int c = up ? jj - U : jj;
            const size_t o = (size_t)b * U + c;
            const float inh = up ? (u_in ? u_in[o] : root_u_slot[c]) : (l_in ? l_in[o] : root_l_slot[c]);
            float res = inh;
            if (!skip) {
                const float val = (tot[i][j] + cmp[i][j]) + PCc[jj];
                const float pad = __double2float_ru(GAMMA_RC * (double)pscale[jj]);
                float lo_v = __fsub_rd(val, pad), hi_v = __fadd_ru(val, pad);
                // stability decision uncertain: recompute this bound in FP64
                if (lo_v < 0.f && hi_v >= 0.f) {
                    double s = (double)PCc[jj], mag = fabs((double)PCc[jj]);
                    const float* pr = PC + (size_t)jj * K;
                    for (int k = 0; k < n0; ++k) {
                        const double t1 = (double)pr[k] * (double)lo[(size_t)b * n0 + k];
                        const double t2 = (double)pr[n0 + k] * (double)hi[(size_t)b * n0 + k];
                        s += t1 + t2;
                        mag += fabs(t1) + fabs(t2);
                    }
                    const double e64 = ldexp(mag, -40);
                    lo_v = __double2float_rd(s - e64);
                    hi_v = __double2float_ru(s + e64);
                }
                if (up) res = fminf(inh, hi_v);
                else res = fmaxf(inh, lo_v);
            }
            if (up) u_out[o] = res; else l_out[o] = res;
        }
    }
}

// per subdomain: stability mask, split signs, l > u infeasibility
__global__ void k_post_reconc(cv_cache cc, cv_batch_in in, int enforce, float* l, float* u, int8_t* mask,
                              uint8_t* infeasible) {
    const int b = blockIdx.x;
    const int U = cc.U;
    for (int c = threadIdx.x; c < U; c += blockDim.x) {
        const size_t o = (size_t)b * U + c;
        mask[o] = (l[o] >= 0.f) ? 1 : ((u[o] <= 0.f) ? -1 : 0);
    }
    __syncthreads();
    if (threadIdx.x == 0 && enforce && in.split_off && in.split_ids) {
        const int s0 = in.split_off[b], s1 = in.split_off[b + 1];
        for (int s = s0; s < s1 && s1 - s0 <= in.max_splits; ++s) {
            const int code = in.split_ids[s];
            const int g = (code > 0 ? code : -code) - 1;
            if (code == 0 || g >= cc.H) continue;
            const int slot = cc.slot_of[g];
            if (slot < 0) continue;
            const size_t o = (size_t)b * U + slot;
            if (code > 0) { if (l[o] < 0.f) l[o] = 0.f; mask[o] = 1; }
            else { if (u[o] > 0.f) u[o] = 0.f; mask[o] = -1; }
        }
    }
    __syncthreads();
    if (infeasible[b]) return;
    __shared__ int bad;
    if (threadIdx.x == 0) bad = 0;
    __syncthreads();
    for (int c = threadIdx.x; c < U; c += blockDim.x) {
        const size_t o = (size_t)b * U + c;
        if (l[o] > u[o]) bad = 1;
    }
    __syncthreads();
    if (threadIdx.x == 0 && bad) infeasible[b] = 1;
}

__global__ void k_gather_root(int U, const int* ids, const float* rl, const float* ru, float* ls, float* us) {
    int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c < U) { ls[c] = rl[ids[c]]; us[c] = ru[ids[c]]; }
}

}  // namespace

cv_status cv_launch_reconc(const cv_net* net, const cv_cache* cache, const cv_batch_in* in,
                           const cv_options* opt, const cv_ws_layout* lay, char* ws,
                           const float* lo_clip, const float* hi_clip, float* l, float* u,
                           int8_t* mask, uint8_t* infeasible, cudaStream_t st) {
    const int U = cache->U, B = in->B;
    if (U == 0) return CV_OK;
    float* rls = (float*)(ws + lay->rowdesc);
    float* rus = rls + U;
    k_gather_root<<<(U + 255) / 256, 256, 0, st>>>(U, cache->ids, cache->root_l, cache->root_u, rls, rus);
    if (opt->precision == CV_PREC_BF16X8) {
        cv_status s = cv_reconc_tc(cache, B, lo_clip, hi_clip, rls, rus, in->l_in, in->u_in, infeasible, l, u,
                                   (uint16_t*)(ws + lay->tc_box), (int*)(ws + lay->tc_bexp),
                                   (float*)(ws + lay->tc_bsum), net->status, st);
        if (s) return s;
    } else {
        dim3 grd((2 * U + BN - 1) / BN, (B + BM - 1) / BM);
        k_reconc<<<grd, 256, 0, st>>>(B, U, cache->n0, lo_clip, hi_clip, cache->PC, cache->PCc, cache->pscale, rls,
                                      rus, in->l_in, in->u_in, infeasible, l, u);
        CV_LAUNCH_CHECK("k_reconc");
    }
    k_post_reconc<<<B, 256, 0, st>>>(*cache, *in, opt->enforce_splits, l, u, mask, infeasible);
    CV_LAUNCH_CHECK("k_post_reconc");
    return CV_OK;
}
