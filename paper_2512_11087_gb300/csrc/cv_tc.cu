// Tensor-core back-substitution of the spec rows (a7 with precision CV_PREC_BF16X8): every
// contraction P = Lam^(i) W^(i) of the CROWN recursion runs on tcgen05 tensor cores with TMA-fed
// shared-memory tiles, at exactly known error.
//
// Split arithmetic.  A row r of Lam (and a column q of W) is scaled by a power of two 2^e_r
// (2^f_q) not below its largest magnitude and rounded to a 24-bit fixed-point integer N, |N| <=
// 2^23, with |x 2^-e - N 2^-23| <= 2^-24.  N is written in balanced base-256 digits,
// N = X1 2^16 + X2 2^8 + X3 with X1 in [-128, 128] and X2, X3 in [-128, 127]; every digit is exact
// in BF16.  The digit products X_i Y_j (|.| <= 2^14) are grouped by level s = i + j:
//     P_rq = 2^(e_r + f_q - 46) sum_s L_s 2^(8 (6 - s)),  L_s = sum_k sum_{i+j=s} X_i(r,k) Y_j(k,q).
// Levels 2..5 are kept (eight BF16 MMAs per K step: (1,1) (1,2) (2,1) (1,3) (2,2) (3,1) (2,3)
// (3,2)); level 6 (X3 Y3 <= 2^14 per term) is dropped.  For K <= 256 every partial sum of every
// level is an integer below 2^24 (level 4: 3 K 2^14 <= 1.5 2^23), so the FP32 accumulation in
// tensor memory is exact in any order; longer K runs in chunks of 256 with an accumulator set
// per chunk, two sets at a time (a pass of 512 K): the chunk sums are added in FP32 in chunk
// order, those of every pass but the last through running sums in shared memory while the
// tensor memory is refilled.  The error of P against the exact product of the FP32 operands is
//     |dP_rq| <= c 2^-24 (2^f_q S_r + 2^e_r T_q) + 2^(e_r + f_q) K 2^-31,
//     S_r = sum_k |Lam_rk|,  T_q = sum_k |W_kq|,  c = 1 + 2^-6
// (quantisation of both operands, the dropped level, and the part of the FP32 level sum that
// exceeds 3 u sum_k |Lam_rk||W_kq|, which the gamma |Lam| V pad covers: 24 u, plus one u for
// every chunk beyond two).  Its
// effect on the bound, sum_q |dP_rq| zmag_q, is charged to the row's pad by the splitting
// kernel: 2^-24 c (S_r F1 + 2^e_r F2) + 2^e_r K 2^-31 F1, F1 = sum_q 2^f_q zmag_q,
// F2 = sum_q T_q zmag_q (per layer, computed with the split weights).
//
// Tiles.  One CTA computes 128 rows x 64 columns of P over all of K: TMA loads the three digit
// slices of the row tile and of the column tile (128-byte swizzle) into a two-stage ring; one
// thread issues the tcgen05.mma instructions (M = 128, N = 64, K = 16) into four (or eight)
// FP32 accumulators in tensor memory and commits each stage back to its producer; the four warps
// then read their 32 rows of every accumulator with tcgen05.ld, form P in FP32 and run the
// relaxation epilogue of the FP32 path (cv_backward.cu).  Every wait on an mbarrier is bounded;
// a wait that runs out sets a status bit and the CTA skips the rest of its work.
#include "cv_internal.cuh"

#include <math.h>
#include <string.h>

#include <mutex>
#include <vector>

namespace {

constexpr int TBM = 128, TBN = 64, TBK = 64;  // CTA tile and K step of the TMA boxes
constexpr int KCH = 256;                       // K rows per exact accumulator set
constexpr int KMAX = 1 << 16;                  // longest K the path takes (passes of two sets)
constexpr int NLEV = 4;                        // kept levels 2..5
constexpr double PAD_C = 1.0 + 1.0 / 64.0;
// Pad per unit of sum_k |Lam_k| V_k for each contraction (V = |W| zmag + |b|): the FP32 sum of
// the levels (three roundings per chunk, then one per chunk added: at most nch + 2, budgeted as
// max(7, nch + 5)) and the FP32 relaxation epilogue (15 u, as in the CUDA-core path), 2 u spare;
// the operand splitting is charged separately.  nch: the most chunks of any layer.
inline double tc_gamma(int nch) { return (24.0 + (nch > 2 ? nch - 2 : 0)) * CV_U32; }
constexpr int TC_RUN_SMEM = TBM * (TBN + 1) * 4;  // running sums of a tile over the passes

// balanced base-256 digits of |n| <= 2^23
__device__ __forceinline__ void digits3(int n, int& x1, int& x2, int& x3) {
    x3 = ((n + 128) & 255) - 128;
    n = (n - x3) >> 8;
    x2 = ((n + 128) & 255) - 128;
    x1 = (n - x2) >> 8;
}

__device__ __forceinline__ uint16_t bf16_of_int(int v) {
    // small integers (|v| <= 128) are exact in BF16: the top half of the FP32 pattern
    return (uint16_t)(__float_as_uint((float)v) >> 16);
}

// exponent e with max_abs <= 2^e (0 for an all-zero vector)
__device__ __forceinline__ int pow2_ceil_exp(float max_abs) {
    if (!(max_abs > 0.f)) return 0;
    int e;
    frexpf(max_abs, &e);  // max_abs = m 2^e, m in [0.5, 1)
    return e;
}

// Split the columns of W^(i) [K x N] into the digit slices of W^T [3][Np][Kp]; fexp, the column
// sums T_q and the pad constants F1, F2 (accumulated in FP64 atomics).  One warp per column.
__global__ void k_tc_wsplit(int K, int N, int Kp, int Np, const float* W, const float* zmag, uint16_t* S,
                            int* fexp, double* F) {
    const int q = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    const int lane = threadIdx.x & 31;
    if (q >= Np) return;
    const size_t plane = (size_t)Np * Kp;
    if (q >= N) {
        for (int k = lane; k < Kp; k += 32) {
            S[(size_t)q * Kp + k] = 0; S[plane + (size_t)q * Kp + k] = 0; S[2 * plane + (size_t)q * Kp + k] = 0;
        }
        return;
    }
    float mx = 0.f;
    double tsum = 0.0;
    int nz = 0;
    for (int k = lane; k < K; k += 32) {
        const float w = fabsf(W[(size_t)k * N + q]);
        mx = fmaxf(mx, w);
        tsum += (double)w;
        nz += w != 0.f;
    }
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
        mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, off));
        tsum += __shfl_xor_sync(0xffffffffu, tsum, off);
        nz += __shfl_xor_sync(0xffffffffu, nz, off);
    }
    const int e = pow2_ceil_exp(mx);
    for (int k = lane; k < Kp; k += 32) {
        int x1 = 0, x2 = 0, x3 = 0;
        if (k < K) digits3(__float2int_rn(ldexpf(W[(size_t)k * N + q], 23 - e)), x1, x2, x3);
        S[(size_t)q * Kp + k] = bf16_of_int(x1);
        S[plane + (size_t)q * Kp + k] = bf16_of_int(x2);
        S[2 * plane + (size_t)q * Kp + k] = bf16_of_int(x3);
    }
    if (lane == 0) {
        fexp[q] = e;
        const double z = (double)zmag[q];
        atomicAdd(&F[0], ldexp(1.0, e) * z);
        atomicAdd(&F[1], tsum * z);
        atomicAdd(&F[2], (double)nz * ldexp(1.0, e) * z);
    }
}

typedef CUresult (*EncodeTiled)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeTiled encoder() {
    static std::once_flag once;
    static EncodeTiled fn = nullptr;
    std::call_once(once, [] {
        cudaDriverEntryPointQueryResult q;
        void* p = nullptr;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess && q == cudaDriverEntryPointSuccess)
            fn = (EncodeTiled)p;
    });
    return fn;
}

// 3-D map over digit slices [3][rows][Kp] (BF16), box {64, box_rows, 1}, 128-byte swizzle; rows
// beyond `rows` read as zero.
cv_status encode_slices(CUtensorMap* m, const void* base, int rows, int Kp, int box_rows) {
    EncodeTiled enc = encoder();
    if (!enc) { cv_set_error("cuTensorMapEncodeTiled is not available from the driver"); return CV_EUNSUPPORTED; }
    cuuint64_t dims[3] = {(cuuint64_t)Kp, (cuuint64_t)rows, 3};
    cuuint64_t strides[2] = {(cuuint64_t)Kp * 2, (cuuint64_t)Kp * 2 * (cuuint64_t)rows};
    cuuint32_t box[3] = {(cuuint32_t)TBK, (cuuint32_t)box_rows, 1};
    cuuint32_t es[3] = {1, 1, 1};
    CUresult r = enc(m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 3, const_cast<void*>(base), dims, strides, box, es,
                     CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
                     CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) {
        cv_set_error("cuTensorMapEncodeTiled failed (" + std::to_string((int)r) + ")");
        return CV_ECUDA;
    }
    return CV_OK;
}

int round_up(int x, int a) { return (x + a - 1) / a * a; }

}  // namespace


namespace {

// Row loaders of the splitting kernel: rows of a row-major matrix, or the box rows [lo_b | hi_b].
struct RowLd {
    const float* A;
    int K;
    __device__ float operator()(int r, int k) const { return A[(size_t)r * K + k]; }
};
struct BoxLd {
    const float* lo;
    const float* hi;
    int n0;
    __device__ float operator()(int r, int k) const {
        return k < n0 ? lo[(size_t)r * n0 + k] : hi[(size_t)r * n0 + (k - n0)];
    }
};

// Split R rows of length K into digit slices [3][R][Kp] and the row exponent; optionally the row's
// absolute sum (rounded up) and the contraction's error term added to the row's pad (see the file
// header).  One warp per row, eight consecutive elements per lane (one 16-byte store per slice).
template <class Ld>
__global__ void k_tc_split(int R, int plane_rows, int K, int Kp, Ld ld, uint16_t* S, int* rexp, float* rsum,
                           int* rnnz, double* acc_pad, double F1, double F2, double F3) {
    const int r = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    const int lane = threadIdx.x & 31;
    if (r >= R) return;
    float mx = 0.f, ssum = 0.f;  // ssum: sum of |row| rounded up
    int nz = 0;
    for (int k = lane; k < K; k += 32) {
        const float v = fabsf(ld(r, k));
        mx = fmaxf(mx, v);
        ssum = __fadd_ru(ssum, v);
        nz += v != 0.f;
    }
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
        mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, off));
        ssum = __fadd_ru(ssum, __shfl_xor_sync(0xffffffffu, ssum, off));
        nz += __shfl_xor_sync(0xffffffffu, nz, off);
    }
    const int e = pow2_ceil_exp(mx);
    const size_t plane = (size_t)plane_rows * Kp;  // slice stride (rows of the tensor map)
    uint16_t* s0 = S + (size_t)r * Kp;
    for (int k0 = lane * 8; k0 < Kp; k0 += 256) {
        unsigned w1[4], w2[4], w3[4];
#pragma unroll
        for (int h = 0; h < 4; ++h) {
            int d1[2], d2[2], d3[2];
#pragma unroll
            for (int t = 0; t < 2; ++t) {
                const int k = k0 + 2 * h + t;
                d1[t] = d2[t] = d3[t] = 0;
                if (k < K) digits3(__float2int_rn(ldexpf(ld(r, k), 23 - e)), d1[t], d2[t], d3[t]);
            }
            w1[h] = (unsigned)bf16_of_int(d1[0]) | ((unsigned)bf16_of_int(d1[1]) << 16);
            w2[h] = (unsigned)bf16_of_int(d2[0]) | ((unsigned)bf16_of_int(d2[1]) << 16);
            w3[h] = (unsigned)bf16_of_int(d3[0]) | ((unsigned)bf16_of_int(d3[1]) << 16);
        }
        *(uint4*)(s0 + k0) = make_uint4(w1[0], w1[1], w1[2], w1[3]);
        *(uint4*)(s0 + plane + k0) = make_uint4(w2[0], w2[1], w2[2], w2[3]);
        *(uint4*)(s0 + 2 * plane + k0) = make_uint4(w3[0], w3[1], w3[2], w3[3]);
    }
    if (lane == 0) {
        rexp[r] = e;
        if (rsum) rsum[r] = ssum;
        if (rnnz) rnnz[r] = nz;
        if (acc_pad) {
            // W's quantisation meets Lam_rk only where W_kq != 0: sum_q min(S_r, nnz_q 2^e) 2^f_q zmag_q
            // <= min(S_r F1, 2^e F3); the dropped level likewise has nnz_q terms per column
            const double pe = ldexp(1.0, e);
            acc_pad[r] += (PAD_C * ldexp(fmin((double)ssum * F1, pe * F3) + pe * F2, -24) + pe * ldexp(F3, -31)) *
                          (1.0 + 1e-12);
        }
    }
}

__device__ __forceinline__ unsigned su32(const void* p) { return (unsigned)__cvta_generic_to_shared(p); }

__device__ __forceinline__ bool bar_wait(uint64_t* bar, unsigned phase) {
    for (int i = 0; i < (1 << 22); ++i) {
        unsigned ok;
        asm volatile(
            "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
            : "=r"(ok)
            : "r"(su32(bar)), "r"(phase)
            : "memory");
        if (ok) return true;
    }
    return false;
}

// shared-memory matrix descriptor: K-major, 128-byte swizzle, 8-row groups 1024 bytes apart
__device__ __forceinline__ uint64_t sdesc(const void* p) {
    uint64_t d = (uint64_t)((su32(p) >> 4) & 0x3fffu);
    d |= (uint64_t)1 << 16;            // leading byte offset (unused for swizzled K-major)
    d |= (uint64_t)(1024 >> 4) << 32;  // stride byte offset
    d |= (uint64_t)1 << 46;            // descriptor version
    d |= (uint64_t)2 << 61;            // 128-byte swizzle
    return d;
}

__device__ __forceinline__ void tma3(void* dst, const CUtensorMap* m, int x, int y, int z, uint64_t* bar) {
    asm volatile(
        "cp.async.bulk.tensor.3d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4}], [%5];" ::"r"(
            su32(dst)),
        "l"(m), "r"(x), "r"(y), "r"(z), "r"(su32(bar))
        : "memory");
}

__device__ __forceinline__ void tmem_ld8(unsigned taddr, float* v) {
    unsigned r[8];
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7])
                 : "r"(taddr)
                 : "memory");
#pragma unroll
    for (int j = 0; j < 8; ++j) v[j] = __uint_as_float(r[j]);
}

struct TcArgs {
    int R, K, N, i, Kp, nch;
    int rows_per_sub, m, hoff, H;
    const int* rexp; const int* fexp;
    const float* root_l; const float* root_u; const int8_t* root_state;
    const int* slot_of; const float* l; const float* u; const int8_t* mask; int U;
    const float* alpha; int alpha_mode;
    const float* bnext; const float* Vnext;
    const float* T0; const float* T1; const float* T2;  // relaxation table of layer i-1 [B x N]
    float* Aout;
    float* keepP;        // optional [R x N]: the product P^(i) (i > 1), for the BaBSR weight or the adjoint
    // slope adjoint (adj = 1): P is dLam^(h) = dP^(h) W^(h)^T with W^(h)'s rows as the B operand;
    // the epilogue applies the fixed relaxation of the forward (its products Pfwd = P^(h+1))
    int adj, last;
    const float* bvec;   // b^(h) [N]
    const float* Pfwd;   // P^(h+1) [R x N]
    const float* grad_f; // [R] or NULL
    float* grad_alpha;   // [B x m x H]
    const float* beta;   // split multipliers [B x m x H] with their signs bsign [B x H], or NULL
    const int8_t* bsign;
    float* grad_beta;    // adjoint: [B x m x H]
    const float* lo; const float* hi;
    float* lam0;
    double* part_bias; double* part_pad; double* part_f; double* part_fmag; int ncb;
    int* status;
};

constexpr int STAGE_A = 3 * TBM * TBK * 2;  // bytes of the three A slices of one K step
constexpr int STAGE_B = 3 * TBN * TBK * 2;
constexpr int STAGE = STAGE_A + STAGE_B;
constexpr int NSTAGE = 1;  // one stage: two CTAs share an SM and overlap each other's phases
constexpr int TC_SMEM = NSTAGE * STAGE + 1024;

__global__ void __launch_bounds__(256, 2) k_tc_layer(const __grid_constant__ CUtensorMap tA,
                                                     const __grid_constant__ CUtensorMap tB, TcArgs a) {
    extern __shared__ __align__(1024) unsigned char tc_raw[];
    unsigned char* sm = (unsigned char*)(((uintptr_t)tc_raw + 1023) & ~(uintptr_t)1023);
    __shared__ __align__(8) uint64_t full[2], empty[2], done;
    __shared__ unsigned tmem_base;
    __shared__ int s_fail;
    const int warp = threadIdx.x >> 5;
    const int row0 = blockIdx.y * TBM, col0 = blockIdx.x * TBN;
    const int KT = a.Kp / TBK;
    // K runs in passes of two chunks (two exact accumulator sets); the sums of every pass but the
    // last are drained into FP32 running sums in shared memory, in chunk order
    const int nset = a.nch < 2 ? a.nch : 2;
    const unsigned ncols = (unsigned)(nset * NLEV * TBN);  // 256 or 512
    const int npass = (a.nch + 1) / 2;
    constexpr int KTP = 2 * KCH / TBK;                      // K tiles per pass
    float* s_run = (float*)(sm + NSTAGE * STAGE);           // [TBM][TBN + 1] when npass > 1
    if (threadIdx.x == 0) {
        s_fail = 0;
        for (int s = 0; s < 2; ++s) {
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(su32(&full[s])) : "memory");
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(su32(&empty[s])) : "memory");
        }
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(su32(&done)) : "memory");
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(su32(&tmem_base)),
                     "r"(ncols)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const unsigned tmem = tmem_base;

    bool fine = true;
    for (int pass = 0; pass < npass; ++pass) {
    const int kt0 = pass * KTP, kt1 = min(KT, kt0 + KTP);
    if (threadIdx.x == 0) {
        // producer: TMA ring of NSTAGE stages (its phases run on over the passes)
        for (int kt = kt0; kt < kt1; ++kt) {
            const int s = kt % NSTAGE;
            if (kt >= NSTAGE && !bar_wait(&empty[s], ((kt - NSTAGE) / NSTAGE) & 1)) { s_fail = 1; break; }
            unsigned char* st = sm + s * STAGE;
            asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(su32(&full[s])), "r"(STAGE)
                         : "memory");
            for (int z = 0; z < 3; ++z) {
                tma3(st + z * (TBM * TBK * 2), &tA, kt * TBK, row0, z, &full[s]);
                tma3(st + STAGE_A + z * (TBN * TBK * 2), &tB, kt * TBK, col0, z, &full[s]);
            }
        }
    } else if (threadIdx.x == 32) {
        // MMA issuer: eight digit products per 16-wide K step into the level accumulators
        const unsigned idesc = (1u << 4) | (1u << 7) | (1u << 10) | ((unsigned)(TBN >> 3) << 17) |
                               ((unsigned)(TBM >> 4) << 24);
        const int pi[8] = {0, 0, 1, 0, 1, 2, 1, 2};  // digit of A (slice)
        const int pj[8] = {0, 1, 0, 2, 1, 0, 2, 1};  // digit of B
        bool ok = true;
        for (int kt = kt0; kt < kt1 && ok; ++kt) {
            const int s = kt % NSTAGE;
            if (!bar_wait(&full[s], (kt / NSTAGE) & 1)) { s_fail = 1; ok = false; break; }
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            const unsigned char* st = sm + s * STAGE;
            const int ch = (kt * TBK) / KCH - 2 * pass;  // accumulator set of the pass
            const bool first_tile = (kt * TBK) % KCH == 0;
            for (int kk = 0; kk < TBK / 16; ++kk) {
#pragma unroll
                for (int p = 0; p < 8; ++p) {
                    const int lev = pi[p] + pj[p];  // level - 2
                    const unsigned d = tmem + (unsigned)((ch * NLEV + lev) * TBN);
                    const uint64_t da = sdesc(st + pi[p] * (TBM * TBK * 2)) + (uint64_t)(kk * 2);
                    const uint64_t db = sdesc(st + STAGE_A + pj[p] * (TBN * TBK * 2)) + (uint64_t)(kk * 2);
                    // the first product of each level in the first K step of a chunk starts the sum
                    const bool first_of_level = (p == 0) || (p == 1) || (p == 3) || (p == 6);
                    const unsigned acc = (first_tile && kk == 0 && first_of_level) ? 0u : 1u;
                    asm volatile(
                        "{\n .reg .pred p;\n setp.ne.u32 p, %4, 0;\n tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(
                            d),
                        "l"(da), "l"(db), "r"(idesc), "r"(acc)
                        : "memory");
                }
            }
            asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                             su32(&empty[s]))
                         : "memory");
        }
        if (ok)
            asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                             su32(&done))
                         : "memory");
    }
    __syncthreads();
    fine = __syncthreads_and(fine && !s_fail && bar_wait(&done, pass & 1)) != 0;
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    if (!fine || pass == npass - 1) break;
    {
        // drain both sets of this pass into the running sums, then hand tensor memory back
        const int dw = warp & 3, dh = warp >> 2;
        const int dr = dw * 32 + (threadIdx.x & 31);
        const unsigned dbase = tmem + ((unsigned)(dw * 32) << 16);
        for (int cc = 0; cc < 32; cc += 8) {
            const int c0 = dh * 32 + cc;
            for (int ch = 0; ch < 2; ++ch) {
                float lv[NLEV][8];
#pragma unroll
                for (int v = 0; v < NLEV; ++v) tmem_ld8(dbase + (unsigned)((ch * NLEV + v) * TBN + c0), lv[v]);
                asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
                float* run = s_run + (size_t)dr * (TBN + 1) + c0;
#pragma unroll
                for (int j = 0; j < 8; ++j) {
                    const float lev = fmaf(lv[0][j], 16777216.f, fmaf(lv[1][j], 65536.f, fmaf(lv[2][j], 256.f, lv[3][j])));
                    run[j] = (pass == 0 && ch == 0) ? 0.f + lev : run[j] + lev;
                }
            }
        }
        asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
        __syncthreads();
    }
    }
    if (!fine && threadIdx.x == 0) atomicOr(a.status, CV_DEV_TIMEOUT);
    if (a.adj) {
        // Slope adjoint: dLam^(h)_q = (dP W^T)_q + g_f b_q; with the forward's relaxation choice
        // (P^(h+1) >= 0 selects the lower line): d alpha = dLam P^(h+1) for unstable neurons on
        // the lower line; dP^(h+1)_q = dLam d_q + g_f e_q (unless h is the last hidden layer).
        const int wq = warp & 3, half = warp >> 2;
        const int tr = wq * 32 + (threadIdx.x & 31);
        const int r = row0 + tr;
        const bool rok = fine && r < a.R;
        const int er = rok ? a.rexp[r] : 0;
        const int sub = rok ? r / a.m : 0;
        const float gf = (rok && a.grad_f) ? a.grad_f[r] : 1.f;
        const unsigned lane_base = tmem + ((unsigned)(wq * 32) << 16);
        for (int cc = 0; cc < 32 && fine; cc += 8) {
            const int c0 = half * 32 + cc;
            float acc[8];
            const float* run = s_run + (size_t)tr * (TBN + 1) + c0;
#pragma unroll
            for (int j = 0; j < 8; ++j) acc[j] = npass > 1 ? run[j] : 0.f;
            for (int ch = 0; ch < a.nch - 2 * (npass - 1); ++ch) {
                float lv[NLEV][8];
#pragma unroll
                for (int v = 0; v < NLEV; ++v) tmem_ld8(lane_base + (unsigned)((ch * NLEV + v) * TBN + c0), lv[v]);
                asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
                for (int j = 0; j < 8; ++j)
                    acc[j] += fmaf(lv[0][j], 16777216.f, fmaf(lv[1][j], 65536.f, fmaf(lv[2][j], 256.f, lv[3][j])));
            }
            if (!rok) continue;
            // the eight columns' independent loads are issued together (one round trip each stage
            // instead of one per column): slot, exponent, bias, kept product, slope; then the bounds
            int slotv[8], fev[8];
            float bvv[8], pfv[8], alv[8], lbv[8], ubv[8];
            int stv[8];
            const size_t gar = ((size_t)sub * a.m + (r % a.m)) * a.H + a.hoff;
            // all eight columns inside the layer and 16-byte aligned: kept products in and the next
            // dP out as 16-byte accesses
            const bool vq = (a.N & 3) == 0 && col0 + c0 + 8 <= a.N;
            float aov[8], gav[8], gbv[8];
            int sgv[8];
            if (vq) {
                const float4* pf4 = (const float4*)(a.Pfwd + (size_t)r * a.N + col0 + c0);
                const float4 x0 = pf4[0], x1 = pf4[1];
                pfv[0] = x0.x; pfv[1] = x0.y; pfv[2] = x0.z; pfv[3] = x0.w;
                pfv[4] = x1.x; pfv[5] = x1.y; pfv[6] = x1.z; pfv[7] = x1.w;
            }
            // the slopes and their gradient (and the multipliers' gradient) as 16-byte accesses when
            // their addresses allow; every entry of the eight is then written (0 where nothing enters:
            // the buffers were cleared before the sweep)
            const bool vg = vq && ((uintptr_t)(a.alpha + gar + col0 + c0) & 15) == 0 &&
                            ((uintptr_t)(a.grad_alpha + gar + col0 + c0) & 15) == 0 &&
                            (!a.bsign || ((uintptr_t)(a.grad_beta + gar + col0 + c0) & 15) == 0);
            if (vg) {
                const float4* al4 = (const float4*)(a.alpha + gar + col0 + c0);
                const float4 x0 = al4[0], x1 = al4[1];
                alv[0] = x0.x; alv[1] = x0.y; alv[2] = x0.z; alv[3] = x0.w;
                alv[4] = x1.x; alv[5] = x1.y; alv[6] = x1.z; alv[7] = x1.w;
            }
#pragma unroll
            for (int j = 0; j < 8; ++j) {
                gav[j] = 0.f;
                gbv[j] = 0.f;
                sgv[j] = (a.bsign && col0 + c0 + j < a.N) ? (int)a.bsign[(size_t)sub * a.H + a.hoff + col0 + c0 + j] : 0;
            }
#pragma unroll
            for (int j = 0; j < 8; ++j) {
                const int q = col0 + c0 + j;
                const bool qv = q < a.N;
                slotv[j] = qv ? a.slot_of[a.hoff + q] : -1;
                fev[j] = qv ? a.fexp[q] : 0;
                bvv[j] = qv ? a.bvec[q] : 0.f;
                if (!vq) pfv[j] = qv ? a.Pfwd[(size_t)r * a.N + q] : 0.f;
                if (!vg) alv[j] = qv ? a.alpha[gar + q] : 0.f;
            }
#pragma unroll
            for (int j = 0; j < 8; ++j) {
                const int g = a.hoff + col0 + c0 + j;
                if (col0 + c0 + j >= a.N) { lbv[j] = 0.f; ubv[j] = 0.f; stv[j] = 0; continue; }
                if (slotv[j] >= 0) {
                    const size_t o = (size_t)sub * a.U + slotv[j];
                    lbv[j] = a.l[o]; ubv[j] = a.u[o]; stv[j] = a.mask[o];
                } else {
                    lbv[j] = a.root_l[g]; ubv[j] = a.root_u[g]; stv[j] = a.root_state[g];
                }
            }
#pragma unroll
            for (int j = 0; j < 8; ++j) {
                const int q = col0 + c0 + j;
                if (q >= a.N) continue;
                const float dl = ldexpf(acc[j], er + fev[j] - 38) + gf * bvv[j];
                const float lb = lbv[j], ub = ubv[j];
                const int st = stv[j];
                const float pf = pfv[j];
                float d, e;
                const size_t ga = gar + q;
                if (st > 0) { d = 1.f; e = 0.f; }
                else if (st < 0) { d = 0.f; e = 0.f; }
                else if (pf >= 0.f) {
                    d = alv[j];
                    e = 0.f;
                    if (vg) gav[j] = dl * pf;
                    else a.grad_alpha[ga] = dl * pf;
                } else {
                    const float s = ub / (ub - lb);
                    d = s;
                    e = -s * lb;
                }
                if (a.bsign) {
                    const int sg = sgv[j];
                    if (sg) {
                        if (vg) gbv[j] = (float)(-sg) * dl;
                        else a.grad_beta[ga] = (float)(-sg) * dl;
                    }
                }
                if (!a.last) {
                    if (vq) aov[j] = dl * d + gf * e;
                    else a.Aout[(size_t)r * a.N + q] = dl * d + gf * e;
                }
            }
            if (vq && !a.last) {
                float4* ao = (float4*)(a.Aout + (size_t)r * a.N + col0 + c0);
                ao[0] = make_float4(aov[0], aov[1], aov[2], aov[3]);
                ao[1] = make_float4(aov[4], aov[5], aov[6], aov[7]);
            }
            if (vg) {
                float4* go = (float4*)(a.grad_alpha + gar + col0 + c0);
                go[0] = make_float4(gav[0], gav[1], gav[2], gav[3]);
                go[1] = make_float4(gav[4], gav[5], gav[6], gav[7]);
                if (a.bsign) {
                    float4* bo = (float4*)(a.grad_beta + gar + col0 + c0);
                    bo[0] = make_float4(gbv[0], gbv[1], gbv[2], gbv[3]);
                    bo[1] = make_float4(gbv[4], gbv[5], gbv[6], gbv[7]);
                }
            }
        }
        asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
        __syncthreads();
        if (warp == 0) {
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(ncols) : "memory");
        }
        return;
    }
    // Epilogue.  Stage what the tile's elements need in the (now idle) stage buffers: per column
    // its exponent, b^(i-1) and V^(i-1); per (subdomain, column) the relaxation table of layer
    // i-1 (i > 1) or the box (i = 1).  Warp w reads tensor-memory lanes 32 (w % 4) .. + 31 (its
    // rows) and takes columns 32 (w / 4) .. + 31.
    const int m = a.rows_per_sub;
    const int sub0 = row0 / m;
    const int sub1 = min(row0 + TBM - 1, a.R - 1) / m;
    const int nsub = sub1 - sub0 + 1;
    // staged when the tile's subdomains fit the stage buffer, else read from global memory
    const bool staged = (size_t)nsub * TBN * 3 * sizeof(float) <= (size_t)NSTAGE * STAGE;
    const int tstride = staged ? TBN : a.N;
    const float* g_t0 = (a.i > 1) ? a.T0 : a.lo;
    const float* g_t1 = (a.i > 1) ? a.T1 : a.hi;
    const float* tb0 = staged ? (const float*)sm : g_t0 + (size_t)sub0 * a.N + col0;
    const float* tb1 = staged ? (const float*)sm + (size_t)nsub * TBN : g_t1 + (size_t)sub0 * a.N + col0;
    const float* tb2 = staged ? (const float*)sm + (size_t)2 * nsub * TBN
                              : (a.i > 1 ? a.T2 + (size_t)sub0 * a.N + col0 : nullptr);
    __shared__ int s_fexp[TBN];
    __shared__ float s_bn[TBN], s_vn[TBN];
    __shared__ double s_red[2][TBM];
    if (fine) {
        for (int c = threadIdx.x; c < TBN; c += blockDim.x) {
            const int q = col0 + c;
            const bool ok = q < a.N;
            s_fexp[c] = ok ? a.fexp[q] : 0;
            s_bn[c] = (ok && a.i > 1) ? a.bnext[q] : 0.f;
            s_vn[c] = (ok && a.i > 1) ? a.Vnext[q] : 0.f;
        }
        if (staged) {
            float* s_t = (float*)sm;
            for (int x = threadIdx.x; x < nsub * TBN; x += blockDim.x) {
                const int sb = sub0 + x / TBN, c = x % TBN, q = col0 + c;
                float t0 = 0.f, t1 = 0.f, t2 = 0.f;
                if (q < a.N) {
                    const size_t o = (size_t)sb * a.N + q;
                    t0 = g_t0[o]; t1 = g_t1[o];
                    if (a.i > 1) t2 = a.T2[o];
                }
                s_t[x] = t0; s_t[nsub * TBN + x] = t1; s_t[2 * nsub * TBN + x] = t2;
            }
        }
    }
    __syncthreads();
    const int wq = warp & 3, half = warp >> 2;
    const int tr = wq * 32 + (threadIdx.x & 31);  // row within the tile (tensor-memory lane)
    const int r = row0 + tr;
    const bool rok = fine && r < a.R;
    const int sb = rok ? r / m - sub0 : 0;
    const int er = rok ? a.rexp[r] : 0;
    double pb = 0.0, pp = 0.0;
    const unsigned lane_base = tmem + ((unsigned)(wq * 32) << 16);
    const float* t0 = tb0 + (size_t)sb * tstride;
    const float* t1 = tb1 + (size_t)sb * tstride;
    const float* t2 = (a.i > 1) ? tb2 + (size_t)sb * tstride : nullptr;
    for (int cc = 0; cc < 32 && fine; cc += 8) {
        const int c0 = half * 32 + cc;
        float acc[8];
        const float* run = s_run + (size_t)tr * (TBN + 1) + c0;
#pragma unroll
        for (int j = 0; j < 8; ++j) acc[j] = npass > 1 ? run[j] : 0.f;
        for (int ch = 0; ch < a.nch - 2 * (npass - 1); ++ch) {
            float lv[NLEV][8];
#pragma unroll
            for (int v = 0; v < NLEV; ++v) tmem_ld8(lane_base + (unsigned)((ch * NLEV + v) * TBN + c0), lv[v]);
            asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
            // sum of the levels, L2 2^24 + L3 2^16 + L4 2^8 + L5 (FP32, three roundings)
#pragma unroll
            for (int j = 0; j < 8; ++j)
                acc[j] += fmaf(lv[0][j], 16777216.f, fmaf(lv[1][j], 65536.f, fmaf(lv[2][j], 256.f, lv[3][j])));
        }
        if (!rok) continue;
        float s1 = 0.f, s2 = 0.f;
        // products and relaxation of the eight columns first, so that their global loads (slopes
        // given per row, split signs and multipliers) are issued together, not one column at a time
        float pv[8], dv[8], ev[8], btv[8], lamv[8];
        int sgv[8];
        // all eight columns inside the layer and 16-byte aligned: the outputs leave as two 16-byte
        // stores per lane (a quarter of the sector writes of eight 4-byte ones)
        const bool vec8 = a.i > 1 && (a.N & 3) == 0 && col0 + c0 + 8 <= a.N;
        if (a.i > 1) {
            const size_t arow = ((size_t)(sub0 + sb) * a.m + (r % a.m)) * a.H + a.hoff;
            const size_t srow = (size_t)(sub0 + sb) * a.H + a.hoff;
#pragma unroll
            for (int j = 0; j < 8; ++j) {
                const int c = c0 + j;
                const bool qv = col0 + c < a.N;
                pv[j] = ldexpf(acc[j], er + s_fexp[c] - 38);  // 2^(e + f - 46) times the 2^8 level unit
                // relaxation of neuron q by the sign of p (table of layer i-1; NaN: slope from alpha)
                if (pv[j] >= 0.f) { dv[j] = qv ? t0[c] : 0.f; ev[j] = 0.f; }
                else { dv[j] = qv ? t1[c] : 0.f; ev[j] = qv ? t2[c] : 0.f; }
                sgv[j] = (qv && a.bsign) ? (int)a.bsign[srow + col0 + c] : 0;
                btv[j] = (qv && a.bsign) ? a.beta[arow + col0 + c] : 0.f;
            }
            bool need = false;  // the table says NaN only when slopes are given per row (alpha set)
#pragma unroll
            for (int j = 0; j < 8; ++j) need |= dv[j] != dv[j];
            if (need && vec8 && a.alpha && ((uintptr_t)(a.alpha + arow + col0 + c0) & 15) == 0) {
                // slopes given per row: all eight as two 16-byte loads, used where the table says NaN
                const float4* al4 = (const float4*)(a.alpha + arow + col0 + c0);
                const float4 x0 = al4[0], x1 = al4[1];
                const float xs[8] = {x0.x, x0.y, x0.z, x0.w, x1.x, x1.y, x1.z, x1.w};
#pragma unroll
                for (int j = 0; j < 8; ++j)
                    if (dv[j] != dv[j]) dv[j] = xs[j];
            } else if (need) {
#pragma unroll
                for (int j = 0; j < 8; ++j)
                    if (col0 + c0 + j < a.N && dv[j] != dv[j]) dv[j] = a.alpha[arow + col0 + c0 + j];
            }
        }
#pragma unroll
        for (int j = 0; j < 8; ++j) {
            const int c = c0 + j, q = col0 + c;
            if (q >= a.N) continue;
            if (a.i > 1) {
                const float p = pv[j], d = dv[j], e = ev[j];
                float lam = p * d;
                if (a.bsign) {  // split multiplier: Lam_g -= sign_g beta_g, rounded away from lam
                    const int sg = sgv[j];
                    if (sg) {
                        const float bt = btv[j];
                        lam = sg > 0 ? __fsub_rd(lam, bt) : __fadd_ru(lam, bt);
                    }
                }
                if (vec8) lamv[j] = lam;
                else {
                    a.Aout[(size_t)r * a.N + q] = lam;
                    if (a.keepP) a.keepP[(size_t)r * a.N + q] = p;
                }
                s1 = fmaf(p, e, s1);
                s1 = fmaf(lam, s_bn[c], s1);
                s2 = fmaf(fabsf(lam), s_vn[c], s2);
            } else {
                // FP32 terms in chains of four (charged 8 u of the magnitude sum in the final pad);
                // the magnitude sum itself is rounded up
                const float p = ldexpf(acc[j], er + s_fexp[c] - 38);
                const float lo = t0[c], hi = t1[c];
                s1 += fminf(p * lo, p * hi);
                s2 = __fadd_ru(s2, __fmul_ru(fabsf(p), fmaxf(fabsf(lo), fabsf(hi))));
                if (a.lam0) a.lam0[(size_t)r * a.N + q] = p;
            }
            if ((j & 3) == 3) { pb += (double)s1; pp += (double)s2; s1 = 0.f; s2 = 0.f; }
        }
        if (vec8) {
            float4* ao = (float4*)(a.Aout + (size_t)r * a.N + col0 + c0);
            ao[0] = make_float4(lamv[0], lamv[1], lamv[2], lamv[3]);
            ao[1] = make_float4(lamv[4], lamv[5], lamv[6], lamv[7]);
            if (a.keepP) {
                float4* ko = (float4*)(a.keepP + (size_t)r * a.N + col0 + c0);
                ko[0] = make_float4(pv[0], pv[1], pv[2], pv[3]);
                ko[1] = make_float4(pv[4], pv[5], pv[6], pv[7]);
            }
        }
        pb += (double)s1;
        pp += (double)s2;
    }
    // the two column halves of a row meet in shared memory
    if (half == 1) { s_red[0][tr] = pb; s_red[1][tr] = pp; }
    __syncthreads();
    if (half == 0 && rok) {
        pb += s_red[0][tr];
        pp += s_red[1][tr];
        const size_t o = (size_t)r * a.ncb + blockIdx.x;
        if (a.i > 1) { a.part_bias[o] = pb; a.part_pad[o] = pp; }
        else { a.part_f[o] = pb; a.part_fmag[o] = pp; }
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (warp == 0) {
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(ncols) : "memory");
    }
}

// Relaxation table of hidden layer i-1 for every subdomain: the slope for p >= 0 (1 / 0 for
// stable neurons, the alpha rule otherwise, NaN when per-row slopes are given), and the slope
// and intercept for p < 0 (u / (u - l), -s l for unstable neurons).
__global__ void k_tc_relax(int B, int N, int hoff, const float* root_l, const float* root_u,
                           const int8_t* root_state, const int* slot_of, const float* l, const float* u,
                           const int8_t* mask, int U, int alpha_given, int alpha_mode, float* T0, float* T1,
                           float* T2) {
    const size_t x = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (x >= (size_t)B * N) return;
    const int sub = (int)(x / N), q = (int)(x % N);
    const int g = hoff + q;
    float lb, ub;
    int st;
    const int slot = (slot_of && l) ? slot_of[g] : -1;
    if (slot >= 0) {
        const size_t o = (size_t)sub * U + slot;
        lb = l[o]; ub = u[o]; st = mask[o];
    } else {
        lb = root_l[g]; ub = root_u[g]; st = root_state[g];
    }
    float t0, t1, t2 = 0.f;
    if (st > 0) { t0 = 1.f; t1 = 1.f; }
    else if (st < 0) { t0 = 0.f; t1 = 0.f; }
    else {
        if (alpha_given) t0 = __int_as_float(0x7fc00000);
        else t0 = (alpha_mode == CV_ALPHA_ONE) ? 1.f : (alpha_mode == CV_ALPHA_ZERO) ? 0.f : ((ub >= -lb) ? 1.f : 0.f);
        const float s = ub / (ub - lb);
        t1 = s;
        t2 = -s * lb;
    }
    T0[x] = t0; T1[x] = t1; T2[x] = t2;
}

}  // namespace

cv_status cv_backward_tc(const cv_net* net, const cv_cache* cache, int R, int m, const float* C, const float* t,
                         const float* l, const float* u, const int8_t* mask, int U, const float* alpha,
                         int alpha_mode, const float* lo, const float* hi, const uint8_t* skip, float* lower,
                         float* err, float* lam0, float* bias_out, float* lamA, float* lamB, uint16_t* slices,
                         int* rexp, float* tab, double* part_bias, double* part_pad, double* part_f,
                         double* part_fmag, double* acc_bias, double* acc_pad, int* launches, cudaStream_t st,
                         float* pbuf, float* bab_weight, float* const* keepP_layers, const float* beta,
                         const int8_t* bsign) {
    if (!cv_tc_supported(cache)) {
        cv_set_error("tensor-core back-substitution: a layer's weights were not prepared");
        return CV_EUNSUPPORTED;
    }
    if (R == 0) return CV_OK;
    const int L = net->L;
    int nch_max = 1;
    for (int i = 1; i <= L; ++i) nch_max = std::max(nch_max, (cache->tcw[i]->Kp + KCH - 1) / KCH);
    const double gam = tc_gamma(nch_max);
    cv_status s =
        cv_bwd_spec_init(R, net->dims[L], m, C, t, net->b[L], cache->V[L], lamA, acc_bias, acc_pad, gam, st);
    if (s) return s;
    ++*launches;
    CV_CUDA(cudaFuncSetAttribute(k_tc_layer, cudaFuncAttributeMaxDynamicSharedMemorySize, TC_SMEM + TC_RUN_SMEM));
    float* cur = lamA;
    float* nxt = lamB;
    for (int i = L; i >= 1; --i) {
        const cv_tc_w* w = cache->tcw[i];
        const int nsub = R / (m > 0 ? m : 1);
        const size_t tsz = (size_t)nsub * net->wmax;
        if (i > 1) {
            const size_t n = (size_t)nsub * w->N;
            k_tc_relax<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(
                nsub, w->N, net->hoff[i - 1], cache->root_l, cache->root_u, cache->root_state, cache->slot_of, l, u,
                mask, U, alpha != nullptr, alpha_mode, tab, tab + tsz, tab + 2 * tsz);
            CV_LAUNCH_CHECK("k_tc_relax");
            ++*launches;
        }
        k_tc_split<RowLd><<<(R + 7) / 8, 256, 0, st>>>(R, R, w->K, w->Kp, RowLd{cur, w->K}, slices, rexp, nullptr,
                                                        nullptr, acc_pad, w->F1, w->F2, w->F3);
        CV_LAUNCH_CHECK("k_tc_split");
        CUtensorMap tA;
        if ((s = encode_slices(&tA, slices, R, w->Kp, TBM))) return s;
        TcArgs a;
        memset(&a, 0, sizeof(a));
        a.R = R; a.K = w->K; a.N = w->N; a.i = i; a.Kp = w->Kp; a.nch = (w->Kp + KCH - 1) / KCH;
        a.rows_per_sub = m; a.m = m > 0 ? m : 1;
        a.hoff = (i > 1) ? net->hoff[i - 1] : 0;
        a.H = net->H;
        a.rexp = rexp; a.fexp = w->fexp;
        a.root_l = cache->root_l; a.root_u = cache->root_u; a.root_state = cache->root_state;
        a.slot_of = cache->slot_of; a.l = l; a.u = u; a.mask = mask; a.U = U;
        a.alpha = alpha; a.alpha_mode = alpha_mode;
        a.bnext = (i > 1) ? net->b[i - 1] : nullptr;
        a.Vnext = (i > 1) ? cache->V[i - 1] : nullptr;
        a.T0 = tab; a.T1 = tab + tsz; a.T2 = tab + 2 * tsz;
        a.Aout = nxt;
        a.keepP = (i > 1 && keepP_layers) ? keepP_layers[i] : ((i > 1 && bab_weight && m > 0) ? pbuf : nullptr);
        a.beta = (i > 1) ? beta : nullptr;
        a.bsign = (i > 1 && beta) ? bsign : nullptr;
        a.lo = lo; a.hi = hi; a.lam0 = lam0;
        a.part_bias = part_bias; a.part_pad = part_pad; a.part_f = part_f; a.part_fmag = part_fmag;
        a.ncb = (w->N + TBN - 1) / TBN;
        a.status = net->status;
        dim3 grd(a.ncb, (R + TBM - 1) / TBM);
        k_tc_layer<<<grd, 256, TC_SMEM + (a.nch > 2 ? TC_RUN_SMEM : 0), st>>>(tA, w->tmap, a);
        CV_LAUNCH_CHECK("k_tc_layer");
        *launches += 2;
        if (i > 1) {
            if ((s = cv_bwd_reduce(R, a.ncb, part_bias, part_pad, acc_bias, acc_pad, gam, st))) return s;
            ++*launches;
            if (a.keepP && bab_weight && !keepP_layers) {
                if ((s = cv_babsr_weight_layer(nsub, m, w->N, a.hoff, cache->slot_of, U, pbuf, skip, bab_weight, st)))
                    return s;
                ++*launches;
            }
            float* tmp = cur; cur = nxt; nxt = tmp;
        } else {
            // the concretisation's FP32 products and chains of four: 8 u of its magnitude sum
            if ((s = cv_bwd_final(R, a.ncb, m, part_f, part_fmag, acc_bias, acc_pad, skip, lower, err, bias_out,
                                  8.0 * CV_U32, st)))
                return s;
            ++*launches;
        }
    }
    return CV_OK;
}

cv_status cv_alpha_reverse_tc(const cv_net* net, const cv_cache* cache, int R, int m, const float* l, const float* u,
                              const int8_t* mask, const float* alpha, const float* grad_f, float* const* keepP,
                              float* gA, float* gB, uint16_t* slices, int* rexp, float* grad_alpha, int* launches,
                              cudaStream_t st, const int8_t* bsign, float* grad_beta) {
    const int L = net->L;
    for (int h = 1; h < L; ++h)
        if (!cache->tcwT[h]) {
            cv_set_error("tensor-core slope adjoint: a layer's weights were not prepared");
            return CV_EUNSUPPORTED;
        }
    if (R == 0) return CV_OK;
    CV_CUDA(cudaFuncSetAttribute(k_tc_layer, cudaFuncAttributeMaxDynamicSharedMemorySize, TC_SMEM + TC_RUN_SMEM));
    for (int h = 1; h < L; ++h) {
        const cv_tc_w* w = cache->tcwT[h];
        // dP^(h) rows to digit slices (no pad: the gradient is not a bound)
        k_tc_split<RowLd><<<(R + 7) / 8, 256, 0, st>>>(R, R, w->K, w->Kp, RowLd{gA, w->K}, slices, rexp, nullptr,
                                                        nullptr, nullptr, 0.0, 0.0, 0.0);
        CV_LAUNCH_CHECK("k_tc_split");
        CUtensorMap tA;
        cv_status s = encode_slices(&tA, slices, R, w->Kp, TBM);
        if (s) return s;
        TcArgs a;
        memset(&a, 0, sizeof(a));
        a.adj = 1;
        a.last = (h == L - 1);
        a.R = R; a.K = w->K; a.N = w->N; a.i = h; a.Kp = w->Kp; a.nch = (w->Kp + KCH - 1) / KCH;
        a.rows_per_sub = m; a.m = m;
        a.hoff = net->hoff[h];
        a.H = net->H;
        a.rexp = rexp; a.fexp = w->fexp;
        a.root_l = cache->root_l; a.root_u = cache->root_u; a.root_state = cache->root_state;
        a.slot_of = cache->slot_of; a.l = l; a.u = u; a.mask = mask; a.U = cache->U;
        a.alpha = alpha;
        a.bvec = net->b[h];
        a.Pfwd = keepP[h + 1];
        a.grad_f = grad_f;
        a.grad_alpha = grad_alpha;
        a.bsign = bsign;
        a.grad_beta = grad_beta;
        a.Aout = gB;
        a.ncb = (w->N + TBN - 1) / TBN;
        a.status = net->status;
        dim3 grd(a.ncb, (R + TBM - 1) / TBM);
        k_tc_layer<<<grd, 256, TC_SMEM + (a.nch > 2 ? TC_RUN_SMEM : 0), st>>>(tA, w->tmap, a);
        CV_LAUNCH_CHECK("k_tc_layer");
        *launches += 2;
        float* t = gA; gA = gB; gB = t;
    }
    return CV_OK;
}

// ---------------------------------------------------------------- re-concretisation (a5)
// out[b, j] = [lo_b | hi_b] . PC_j + PCc_j over K = 2 n0, on tensor cores.  Each chunk of 256 K
// rows accumulates its four levels exactly in one of two tensor-memory sets; eight epilogue warps
// drain a finished chunk into FP32 running sums (level sum: three roundings; sum over chunks: one
// rounding per chunk) while the MMA warp fills the other set.  Pad: max(12, nch + 5) u pscale_j
// (the FP32 sums: three roundings per chunk's levels, one per chunk added, one for the intercept,
// against |value| <= pscale_j over the root box) plus the splitting term of the file header with
// S_b = sum |box row| (at most nnz_j 2^e_b on PC_j's support), T_j = sum |PC_j|, and the dropped
// level over PC_j's nnz_j nonzeros.  A padded value that straddles 0 is
// recomputed in FP64 from the FP32 operands, as in the CUDA-core kernel.
namespace {

constexpr int RC_CHUNK_TILES = KCH / TBK;  // K tiles per exact chunk
constexpr int RC_NSTAGE = 2;
constexpr int RC_SMEM = RC_NSTAGE * STAGE + 1024;
constexpr int RC_THREADS = 320;            // warps 0-7 epilogue, 8 TMA producer, 9 MMA issuer

struct RcArgs {
    int B, U, N, n0, K, Kp;
    const int* bexp; const float* bsum;   // box rows: exponent, sum |.| (rounded up)
    const int* fexp; const float* tsum;   // PC rows
    const int* nnz;                       // PC rows' nonzeros
    float gamma;                          // the FP32 sums' pad per unit of pscale
    const float* PCc; const float* pscale;
    const float* PC; const float* lo; const float* hi;
    const float* rls; const float* rus; const float* l_in; const float* u_in; const uint8_t* infeasible;
    float* l_out; float* u_out;
    int* status;
};

__device__ __forceinline__ void bar_arrive(uint64_t* bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(su32(bar)) : "memory");
}

__global__ void __launch_bounds__(RC_THREADS, 1) k_tc_reconc(const __grid_constant__ CUtensorMap tX,
                                                            const __grid_constant__ CUtensorMap tP, RcArgs a) {
    extern __shared__ __align__(1024) unsigned char rc_raw[];
    unsigned char* sm = (unsigned char*)(((uintptr_t)rc_raw + 1023) & ~(uintptr_t)1023);
    __shared__ __align__(8) uint64_t full[RC_NSTAGE], empty[RC_NSTAGE], tfull[2], tempty[2];
    __shared__ unsigned tmem_base;
    __shared__ int s_fail;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int row0 = blockIdx.y * TBM, col0 = blockIdx.x * TBN;
    const int KT = a.Kp / TBK;
    const int nch = (KT + RC_CHUNK_TILES - 1) / RC_CHUNK_TILES;
    const unsigned ncols = 2u * NLEV * TBN;  // two accumulator sets
    if (threadIdx.x == 0) {
        s_fail = 0;
        for (int s = 0; s < RC_NSTAGE; ++s) {
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(su32(&full[s])) : "memory");
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(su32(&empty[s])) : "memory");
        }
        for (int s = 0; s < 2; ++s) {
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(su32(&tfull[s])) : "memory");
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 8;" ::"r"(su32(&tempty[s])) : "memory");
        }
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 9) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(su32(&tmem_base)),
                     "r"(ncols)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const unsigned tmem = tmem_base;

    if (warp == 8) {
        if (lane == 0) {
            for (int kt = 0; kt < KT; ++kt) {
                const int s = kt % RC_NSTAGE;
                if (kt >= RC_NSTAGE && !bar_wait(&empty[s], ((kt - RC_NSTAGE) / RC_NSTAGE) & 1)) { s_fail = 1; break; }
                unsigned char* st = sm + s * STAGE;
                asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(su32(&full[s])),
                             "r"(STAGE)
                             : "memory");
                for (int z = 0; z < 3; ++z) {
                    tma3(st + z * (TBM * TBK * 2), &tX, kt * TBK, row0, z, &full[s]);
                    tma3(st + STAGE_A + z * (TBN * TBK * 2), &tP, kt * TBK, col0, z, &full[s]);
                }
            }
        }
    } else if (warp == 9) {
        if (lane == 0) {
            const unsigned idesc = (1u << 4) | (1u << 7) | (1u << 10) | ((unsigned)(TBN >> 3) << 17) |
                                   ((unsigned)(TBM >> 4) << 24);
            const int pi[8] = {0, 0, 1, 0, 1, 2, 1, 2};
            const int pj[8] = {0, 1, 0, 2, 1, 0, 2, 1};
            for (int kt = 0; kt < KT; ++kt) {
                const int c = kt / RC_CHUNK_TILES, set = c & 1;
                const bool chunk_start = (kt % RC_CHUNK_TILES) == 0;
                const bool chunk_end = (kt % RC_CHUNK_TILES) == RC_CHUNK_TILES - 1 || kt == KT - 1;
                if (chunk_start && c >= 2 && !bar_wait(&tempty[set], ((c - 2) >> 1) & 1)) { s_fail = 1; break; }
                const int s = kt % RC_NSTAGE;
                if (!bar_wait(&full[s], (kt / RC_NSTAGE) & 1)) { s_fail = 1; break; }
                asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
                const unsigned char* st = sm + s * STAGE;
                for (int kk = 0; kk < TBK / 16; ++kk) {
#pragma unroll
                    for (int p = 0; p < 8; ++p) {
                        const int lev = pi[p] + pj[p];
                        const unsigned d = tmem + (unsigned)((set * NLEV + lev) * TBN);
                        const uint64_t da = sdesc(st + pi[p] * (TBM * TBK * 2)) + (uint64_t)(kk * 2);
                        const uint64_t db = sdesc(st + STAGE_A + pj[p] * (TBN * TBK * 2)) + (uint64_t)(kk * 2);
                        const bool first_of_level = (p == 0) || (p == 1) || (p == 3) || (p == 6);
                        const unsigned acc = (chunk_start && kk == 0 && first_of_level) ? 0u : 1u;
                        asm volatile(
                            "{\n .reg .pred p;\n setp.ne.u32 p, %4, 0;\n tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(
                                d),
                            "l"(da), "l"(db), "r"(idesc), "r"(acc)
                            : "memory");
                    }
                }
                asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                                 su32(&empty[s]))
                             : "memory");
                if (chunk_end)
                    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                                     su32(&tfull[set]))
                                 : "memory");
            }
        }
    } else {
        // epilogue warps: drain every chunk into FP32 running sums
        const int wq = warp & 3, half = warp >> 2;
        const unsigned lane_base = tmem + ((unsigned)(wq * 32) << 16);
        float acc[32];
#pragma unroll
        for (int j = 0; j < 32; ++j) acc[j] = 0.f;
        bool ok = true;
        for (int c = 0; c < nch; ++c) {
            const int set = c & 1;
            ok = __all_sync(0xffffffffu, bar_wait(&tfull[set], (c >> 1) & 1));
            if (!ok) break;
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
#pragma unroll
            for (int cc = 0; cc < 32; cc += 8) {
                float lv[NLEV][8];
#pragma unroll
                for (int v = 0; v < NLEV; ++v)
                    tmem_ld8(lane_base + (unsigned)((set * NLEV + v) * TBN + half * 32 + cc), lv[v]);
                asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
                for (int j = 0; j < 8; ++j)
                    acc[cc + j] += fmaf(lv[0][j], 16777216.f, fmaf(lv[1][j], 65536.f, fmaf(lv[2][j], 256.f, lv[3][j])));
            }
            asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
            __syncwarp();
            if (lane == 0) bar_arrive(&tempty[set]);
        }
        if (!ok && lane == 0) atomicOr(a.status, CV_DEV_TIMEOUT);
        const int b = row0 + wq * 32 + lane;
        if (ok && b < a.B) {
            const bool skip = a.infeasible[b] != 0;
            const int eb = a.bexp[b];
            const float sb = a.bsum[b];
            const float c24 = 1.016f * 5.9604645e-08f;  // (1 + 2^-6) 2^-24, rounded up
            unsigned straddle = 0u;                      // bit j: value straddles 0 after padding
#pragma unroll
            for (int j = 0; j < 32; ++j) {
                const int jj = col0 + half * 32 + j;
                if (jj >= a.N) continue;
                const bool up = jj >= a.U;
                const int slot = up ? jj - a.U : jj;
                const size_t o = (size_t)b * a.U + slot;
                const float inh = up ? (a.u_in ? a.u_in[o] : a.rus[slot]) : (a.l_in ? a.l_in[o] : a.rls[slot]);
                float res = inh;
                if (!skip) {
                    const int fj = a.fexp[jj];
                    const float val = ldexpf(acc[j], eb + fj - 38) + a.PCc[jj];
                    // pad, every operation rounded up; PC's quantisation and the dropped level meet
                    // the box row only on PC_j's support: min(S_b, nnz_j 2^eb) in place of S_b
                    const float nzj = (float)a.nnz[jj];
                    const float sbj = fminf(sb, ldexpf(nzj, eb));
                    float pad = __fmul_ru(a.gamma, a.pscale[jj]);
                    pad = __fadd_ru(pad, __fmul_ru(c24, __fadd_ru(__fmul_ru(sbj, ldexpf(1.f, fj)),
                                                                  __fmul_ru(ldexpf(1.f, eb), a.tsum[jj]))));
                    pad = __fadd_ru(pad, ldexpf(nzj, eb + fj - 31));
                    const float lo_v = __fsub_rd(val, pad), hi_v = __fadd_ru(val, pad);
                    if (lo_v < 0.f && hi_v >= 0.f) straddle |= 1u << j;
                    res = up ? fminf(inh, hi_v) : fmaxf(inh, lo_v);
                }
                if (up) a.u_out[o] = res; else a.l_out[o] = res;
            }
            // rare: the stability decision is uncertain in FP32; recompute those bounds in FP64
            while (straddle) {
                const int j = __ffs(straddle) - 1;
                straddle &= straddle - 1u;
                const int jj = col0 + half * 32 + j;
                const bool up = jj >= a.U;
                const int slot = up ? jj - a.U : jj;
                const size_t o = (size_t)b * a.U + slot;
                const float inh = up ? (a.u_in ? a.u_in[o] : a.rus[slot]) : (a.l_in ? a.l_in[o] : a.rls[slot]);
                double sacc = (double)a.PCc[jj], mag = fabs((double)a.PCc[jj]);
                const float* pr = a.PC + (size_t)jj * a.K;
                for (int k = 0; k < a.n0; ++k) {
                    const double t1 = (double)pr[k] * (double)a.lo[(size_t)b * a.n0 + k];
                    const double t2 = (double)pr[a.n0 + k] * (double)a.hi[(size_t)b * a.n0 + k];
                    sacc += t1 + t2;
                    mag += fabs(t1) + fabs(t2);
                }
                const double e64 = ldexp(mag, -40);
                if (up) a.u_out[o] = fminf(inh, __double2float_ru(sacc + e64));
                else a.l_out[o] = fmaxf(inh, __double2float_rd(sacc - e64));
            }
        }
    }
    if (threadIdx.x == 0 && s_fail) atomicOr(a.status, CV_DEV_TIMEOUT);
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (warp == 9) {
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(ncols) : "memory");
    }
}

}  // namespace

size_t cv_tc_box_bytes(const cv_cache* c, int B) {
    if (!c->tcpc) return 0;
    return (size_t)3 * B * c->tcpc->Kp * sizeof(uint16_t);
}

cv_status cv_reconc_tc(const cv_cache* cache, int B, const float* lo, const float* hi, const float* rls,
                       const float* rus, const float* l_in, const float* u_in, const uint8_t* infeasible, float* l,
                       float* u, uint16_t* xslices, int* bexp, float* bsum, int* status, cudaStream_t st) {
    const cv_tc_pc* pc = cache->tcpc;
    if (!pc) { cv_set_error("tensor-core re-concretisation: no split operand"); return CV_EUNSUPPORTED; }
    if (B == 0) return CV_OK;
    const int n0 = cache->n0;
    k_tc_split<BoxLd><<<(B + 7) / 8, 256, 0, st>>>(B, B, pc->K, pc->Kp, BoxLd{lo, hi, n0}, xslices, bexp, bsum,
                                                    nullptr, nullptr, 0.0, 0.0, 0.0);
    CV_LAUNCH_CHECK("k_tc_split");
    CUtensorMap tX;
    cv_status s = encode_slices(&tX, xslices, B, pc->Kp, TBM);
    if (s) return s;
    RcArgs a;
    memset(&a, 0, sizeof(a));
    a.B = B; a.U = cache->U; a.N = pc->N; a.n0 = n0; a.K = pc->K; a.Kp = pc->Kp;
    a.bexp = bexp; a.bsum = bsum; a.fexp = pc->fexp; a.tsum = pc->tsum; a.nnz = pc->nnz;
    a.gamma = (float)(std::max(12, (pc->Kp + KCH - 1) / KCH + 5) * CV_U32 * (1.0 + 1e-6));
    a.PCc = cache->PCc; a.pscale = cache->pscale; a.PC = cache->PC; a.lo = lo; a.hi = hi;
    a.rls = rls; a.rus = rus; a.l_in = l_in; a.u_in = u_in; a.infeasible = infeasible;
    a.l_out = l; a.u_out = u; a.status = status;
    CV_CUDA(cudaFuncSetAttribute(k_tc_reconc, cudaFuncAttributeMaxDynamicSharedMemorySize, RC_SMEM));
    dim3 grd(pc->Np / TBN, (B + TBM - 1) / TBM);
    k_tc_reconc<<<grd, RC_THREADS, RC_SMEM, st>>>(tX, pc->tmap, a);
    CV_LAUNCH_CHECK("k_tc_reconc");
    return CV_OK;
}

void cv_tc_release(cv_cache* c) {
    if (!c) return;
    for (int i = 0; i <= CV_MAX_LAYERS; ++i) {
        for (cv_tc_w** slot : {&c->tcw[i], &c->tcwT[i]}) {
            cv_tc_w* w = *slot;
            if (!w) continue;
            cudaFree(w->slices);
            cudaFree(w->fexp);
            delete w;
            *slot = nullptr;
        }
    }
    if (c->tcpc) {
        cudaFree(c->tcpc->slices);
        cudaFree(c->tcpc->fexp);
        cudaFree(c->tcpc->tsum);
        cudaFree(c->tcpc->nnz);
        delete c->tcpc;
        c->tcpc = nullptr;
    }
}

bool cv_tc_supported(const cv_cache* c) {
    for (int i = 1; i <= c->net->L; ++i)
        if (!c->tcw[i]) return false;
    return true;
}

cv_status cv_tc_prepare(cv_cache* c, const float* xmag, const float* zmag, cudaStream_t st) {
    const cv_net* n = c->net;
    for (int i = 1; i <= n->L; ++i) {
        const int K = n->dims[i], N = n->dims[i - 1];
        const int Kp = round_up(K, TBK), Np = round_up(N, TBN);
        if (Kp > KMAX) continue;  // beyond the path's 32-bit slice indexing
        cv_tc_w* w = new cv_tc_w();
        memset(w, 0, sizeof(*w));
        c->tcw[i] = w;
        w->K = K; w->N = N; w->Kp = Kp; w->Np = Np;
        double* F = nullptr;
        CV_CUDA(cudaMalloc(&w->slices, (size_t)3 * Np * Kp * sizeof(uint16_t)));
        CV_CUDA(cudaMalloc(&w->fexp, (size_t)N * sizeof(int)));
        CV_CUDA(cudaMalloc(&F, 3 * sizeof(double)));
        CV_CUDA(cudaMemsetAsync(F, 0, 3 * sizeof(double), st));
        const float* zm = (i == 1) ? xmag : zmag + n->hoff[i - 1];
        k_tc_wsplit<<<(Np + 7) / 8, 256, 0, st>>>(K, N, Kp, Np, n->W[i], zm, w->slices, w->fexp, F);
        CV_LAUNCH_CHECK("k_tc_wsplit");
        double hF[3];
        CV_CUDA(cudaMemcpyAsync(hF, F, sizeof(hF), cudaMemcpyDeviceToHost, st));
        CV_CUDA(cudaStreamSynchronize(st));
        cudaFree(F);
        w->F1 = hF[0] * (1.0 + 1e-12);
        w->F2 = hF[1] * (1.0 + 1e-12);
        w->F3 = hF[2] * (1.0 + 1e-12);
        cv_status s = encode_slices(&w->tmap, w->slices, Np, Kp, TBN);
        if (s) return s;
    }
    // the rows of W^(h), h < L, for the slope adjoint's contraction dP^(h) W^(h)^T (K = n_{h-1})
    for (int h = 1; h < n->L; ++h) {
        const int K = n->dims[h - 1], N = n->dims[h];
        const int Kp = round_up(K, TBK), Np = round_up(N, TBN);
        if (Kp > KMAX) continue;
        cv_tc_w* w = new cv_tc_w();
        memset(w, 0, sizeof(*w));
        c->tcwT[h] = w;
        w->K = K; w->N = N; w->Kp = Kp; w->Np = Np;
        CV_CUDA(cudaMalloc(&w->slices, (size_t)3 * Np * Kp * sizeof(uint16_t)));
        CV_CUDA(cudaMemsetAsync(w->slices, 0, (size_t)3 * Np * Kp * sizeof(uint16_t), st));
        CV_CUDA(cudaMalloc(&w->fexp, (size_t)N * sizeof(int)));
        k_tc_split<RowLd><<<(N + 7) / 8, 256, 0, st>>>(N, Np, K, Kp, RowLd{n->W[h], K}, w->slices, w->fexp, nullptr,
                                                        nullptr, nullptr, 0.0, 0.0, 0.0);
        CV_LAUNCH_CHECK("k_tc_split");
        cv_status s = encode_slices(&w->tmap, w->slices, Np, Kp, TBN);
        if (s) return s;
    }
    if (c->U > 0) {
        cv_tc_pc* pc = new cv_tc_pc();
        memset(pc, 0, sizeof(*pc));
        c->tcpc = pc;
        pc->K = 2 * c->n0; pc->N = 2 * c->U;
        pc->Kp = round_up(pc->K, TBK); pc->Np = round_up(pc->N, TBN);
        CV_CUDA(cudaMalloc(&pc->slices, (size_t)3 * pc->Np * pc->Kp * sizeof(uint16_t)));
        CV_CUDA(cudaMemsetAsync(pc->slices, 0, (size_t)3 * pc->Np * pc->Kp * sizeof(uint16_t), st));
        CV_CUDA(cudaMalloc(&pc->fexp, (size_t)pc->N * sizeof(int)));
        CV_CUDA(cudaMalloc(&pc->tsum, (size_t)pc->N * sizeof(float)));
        CV_CUDA(cudaMalloc(&pc->nnz, (size_t)pc->N * sizeof(int)));
        // rows of PC, written into the first N of the Np slice rows (the rest stay zero)
        k_tc_split<RowLd><<<(pc->N + 7) / 8, 256, 0, st>>>(pc->N, pc->Np, pc->K, pc->Kp, RowLd{c->PC, pc->K},
                                                            pc->slices, pc->fexp, pc->tsum, pc->nnz, nullptr, 0.0,
                                                            0.0, 0.0);
        CV_LAUNCH_CHECK("k_tc_split");
        cv_status s = encode_slices(&pc->tmap, pc->slices, pc->Np, pc->Kp, TBN);
        if (s) return s;
    }
    return CV_OK;
}

size_t cv_tc_slices_bytes(const cv_net* net, int R) {
    int kp = 0;
    for (int i = 1; i <= net->L; ++i) kp = std::max(kp, round_up(net->dims[i], TBK));
    return (size_t)3 * R * kp * sizeof(uint16_t);
}
