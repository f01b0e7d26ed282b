// Internal declarations of the Clip-and-Verify GB300 library (not part of the C-ABI).
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>
#include <stdint.h>
#include <string>

#include "../../include/clipverify.h"

// ---------------------------------------------------------------- error plumbing
void cv_set_error(const std::string& msg);
cv_status cv_cuda_fail(cudaError_t e, const char* what);

#define CV_SEQ_SMEM_MAX (220 * 1024)  // dynamic shared memory of sequential relaxed clipping

#define CV_CUDA(call)                                                   \
    do {                                                                \
        cudaError_t e_ = (call);                                        \
        if (e_ != cudaSuccess) return cv_cuda_fail(e_, #call);          \
    } while (0)

#define CV_LAUNCH_CHECK(what)                                           \
    do {                                                                \
        cudaError_t e_ = cudaGetLastError();                            \
        if (e_ != cudaSuccess) return cv_cuda_fail(e_, what);           \
    } while (0)

// device status bits (cv_device_status)
#define CV_DEV_CSR_COUNT   1
#define CV_DEV_SPLIT_RANGE 2
#define CV_DEV_NONFINITE   4
#define CV_DEV_TARGET      8
#define CV_DEV_TIMEOUT     16

// unit roundoff of FP32 round-to-nearest (with a small safety factor)
#define CV_U32 (5.9604644775390625e-08 * 1.0001)

// ---------------------------------------------------------------- objects
struct cv_net {
    int L;                       // affine layers
    int dims[CV_MAX_LAYERS + 1]; // flattened widths
    int hoff[CV_MAX_LAYERS + 1]; // first global hidden id of hidden layer i (1..L-1)
    int H;                       // hidden neurons
    int wmax;                    // max width
    float* W[CV_MAX_LAYERS + 1]; // device, W[i]: dims[i] x dims[i-1] row-major (i = 1..L)
    float* b[CV_MAX_LAYERS + 1]; // device, b[i]: dims[i]
    int* status;                 // device status word; status[1]: cv_batch_check's result
    int device;
};

// Split-BF16 copy of one layer's weights for the tensor-core back-substitution (cv_tc.cu).
// W^(i) [K x N] is stored transposed (K-major) as three BF16 digit slices of the column-scaled
// 24-bit fixed-point values, zero padded to Np x Kp (multiples of 64).
struct cv_tc_w {
    uint16_t* slices;   // [3][Np][Kp] BF16 bit patterns
    int* fexp;          // [N] column exponents: |W_kq| <= 2^fexp[q]
    double F1, F2;      // sum_q 2^fexp[q] zmag_q and sum_q (sum_k |W_kq|) zmag_q (pad constants)
    double F3;          // sum_q nnz_q 2^fexp[q] zmag_q, nnz_q the nonzeros of column q (sparse layers)
    int K, N, Kp, Np;
    CUtensorMap tmap;   // 3-D map {Kp, Np, 3}, box {64, 64, 1}, 128-byte swizzle
};

// Split-BF16 copy of the re-concretisation operand PC [2U x 2n0] for the tensor cores (cv_tc.cu).
struct cv_tc_pc {
    uint16_t* slices;   // [3][Np][Kp] BF16 digits of the rows of PC (row-scaled), zero padded
    int* fexp;          // [2U] row exponents
    float* tsum;        // [2U] sum_k |PC_jk|, rounded up
    int* nnz;           // [2U] nonzeros of PC_j (its support bounds the quantisation and dropped-level terms)
    int K, N, Kp, Np;
    CUtensorMap tmap;   // 3-D map {Kp, Np, 3}, box {64, 64, 1}, 128-byte swizzle
};

struct cv_cache {
    const cv_net* net;
    int U, n0, H;
    int* ids;          // [U] global hidden ids
    int* slot_of;      // [H] cache slot or -1
    float* lA;         // [U x n0]
    float* lc;         // [U]
    float* uA;         // [U x n0]
    float* uc;         // [U]
    float* PC;         // [2U x 2n0]: row c < U: [A̲⁺_c | A̲⁻_c]; row U+c: [Ā⁻_c | Ā⁺_c]
    float* PCc;        // [2U]: lc, uc
    float* pscale;     // [2U]: |A|.xmag_root + |c| of the lower / upper plane
    float* amax;       // [2U]: max_q |A_q| of the lower / upper plane (complete clipping's error bounds)
    float* root_l;     // [H]
    float* root_u;     // [H]
    int8_t* root_state;// [H] +1 / -1 / 0
    float* V[CV_MAX_LAYERS + 1]; // V[i] [dims[i]]: |W^(i)| zmag^(i-1) + |b^(i)| (pad weights)
    float* root_lo;    // [n0]
    float* root_hi;    // [n0]
    cv_tc_w* tcw[CV_MAX_LAYERS + 1]; // tensor-core weights per layer (host objects), or null
    cv_tc_w* tcwT[CV_MAX_LAYERS + 1];// rows of W^(i) split for the slope adjoint's W^T contraction, or null
    cv_tc_pc* tcpc;                  // tensor-core re-concretisation operand, or null
    int cc_items[3];   // complete clipping: tasks per work item for 1, 2 and more active rows
};

#define CV_TIMER_COUNTERS 6
struct cv_timer {
    cudaEvent_t ev[CV_N_PHASES + 1];
    unsigned long long* d_steps;  // device counters: complete-clipping row steps, then cv_timer_read_cc's five
    int launches;
    bool used;
};

// ---------------------------------------------------------------- helpers shared by kernels
__host__ __device__ inline size_t cv_align256(size_t x) { return (x + 255) & ~(size_t)255; }

// workspace carving: returns the offset of the next 256-aligned block
struct cv_ws_layout {
    size_t rowflag, vmin, lam0, lam1, part_bias, part_pad, part_f, part_fmag, acc_bias, acc_pad, rowdesc, cc, total;
    size_t tc_slices, tc_exp, tc_tab;  // split-BF16 back-substitution scratch (CV_PREC_BF16X8 only)
    size_t tc_box, tc_bexp, tc_bsum;   // split-BF16 re-concretisation scratch (CV_PREC_BF16X8 only)
    size_t pbuf;                       // layer product P^(i) [R x wmax] for the BaBSR weight (or 0)
    int R, Rmax, ncb;  // rows of the spec backward, max constraint rows, column blocks
};
size_t cv_cc_workspace(int B, int Rmax, int n0);  // complete-clipping region (cv_complete.cu)
// complete clipping of the spec rows' final planes (cv_complete.cu); sscale: [2 x B x m] floats of scratch;
// step_counter: optional device counters as in cv_launch_complete (six)
cv_status cv_launch_spec_clip(const cv_net* net, const cv_cache* cache, const cv_batch_in* in, cv_batch_out* out,
                              const cv_options* opt, const cv_ws_layout* lay, char* ws, float* sscale,
                              unsigned long long* step_counter, int* launches, cudaStream_t st);
cv_status cv_ws_plan(const cv_net* net, const cv_cache* cache, int B, int m, int max_splits,
                     int max_rows, int precision, cv_ws_layout* lay, int babsr_weight = 0);

// Tensor-core back-substitution (cv_tc.cu).  cv_tc_prepare builds the split weights of every
// layer once per cache (called by the cache constructors; layers whose shape the path does not
// take keep a null entry); cv_tc_release frees them.  cv_tc_slices_bytes: digit-slice scratch of R rows.
cv_status cv_tc_prepare(cv_cache* c, const float* xmag, const float* zmag, cudaStream_t st);
void cv_tc_release(cv_cache* c);
bool cv_tc_supported(const cv_cache* c);
size_t cv_tc_slices_bytes(const cv_net* net, int R);
size_t cv_tc_box_bytes(const cv_cache* c, int B);
cv_status cv_reconc_tc(const cv_cache* cache, int B, const float* lo, const float* hi, const float* rls,
                       const float* rus, const float* l_in, const float* u_in, const uint8_t* infeasible, float* l,
                       float* u, uint16_t* xslices, int* bexp, float* bsum, int* status, cudaStream_t st);
cv_status cv_backward_tc(const cv_net* net, const cv_cache* cache, int R, int m, const float* C, const float* t,
                         const float* l, const float* u, const int8_t* mask, int U, const float* alpha,
                         int alpha_mode, const float* lo, const float* hi, const uint8_t* skip, float* lower,
                         float* err, float* lam0, float* bias_out, float* lamA, float* lamB, uint16_t* slices,
                         int* rexp, float* tab, double* part_bias, double* part_pad, double* part_f,
                         double* part_fmag, double* acc_bias, double* acc_pad, int* launches, cudaStream_t st,
                         float* pbuf = nullptr, float* bab_weight = nullptr, float* const* keepP_layers = nullptr,
                         const float* beta = nullptr, const int8_t* bsign = nullptr);
// Reverse sweep of the slope adjoint on tensor cores (cv_tc.cu): g0 = dLam_0 [R x n0] in, the
// layer products P^(h+1) of the forward in keepP[h + 1]; gA / gB [R x wmax] scratch (gA holds g0);
// slices / rexp as for cv_backward_tc.  Writes grad_alpha (zeroed by the caller).
cv_status cv_alpha_reverse_tc(const cv_net* net, const cv_cache* cache, int R, int m, const float* l, const float* u,
                              const int8_t* mask, const float* alpha, const float* grad_f, float* const* keepP,
                              float* gA, float* gB, uint16_t* slices, int* rexp, float* grad_alpha, int* launches,
                              cudaStream_t st, const int8_t* bsign = nullptr, float* grad_beta = nullptr);

// kernels (launch wrappers); each returns CV_OK or a launch error
cv_status cv_launch_rows(const cv_net* net, const cv_cache* cache, const cv_batch_in* in,
                         const cv_ws_layout* lay, char* ws, uint8_t* infeasible, cudaStream_t st);
cv_status cv_launch_relaxed(const cv_net* net, const cv_cache* cache, const cv_batch_in* in,
                            const cv_options* opt, const cv_ws_layout* lay, char* ws,
                            float* lo_clip, float* hi_clip, uint8_t* infeasible, cudaStream_t st);
cv_status cv_launch_reconc(const cv_net* net, const cv_cache* cache, const cv_batch_in* in,
                           const cv_options* opt, const cv_ws_layout* lay, char* ws,
                           const float* lo_clip, const float* hi_clip, float* l, float* u,
                           int8_t* mask, uint8_t* infeasible, cudaStream_t st);
cv_status cv_launch_complete(const cv_net* net, const cv_cache* cache, const cv_batch_in* in,
                             const cv_options* opt, const cv_ws_layout* lay, char* ws,
                             const float* lo_clip, const float* hi_clip, float* l, float* u,
                             int8_t* mask, uint8_t* infeasible, unsigned long long* step_counter,
                             int* launches, cudaStream_t st);
cv_status cv_launch_spec_backward(const cv_net* net, const cv_cache* cache, const cv_batch_in* in,
                                  const cv_options* opt, const cv_ws_layout* lay, char* ws,
                                  const float* lo_clip, const float* hi_clip, const float* l,
                                  const float* u, const int8_t* mask, const uint8_t* infeasible,
                                  cv_batch_out* out, cudaStream_t st);

// Back-substitution of R rows (cv_backward.cu), T = float (per-round spec bound) or double (root
// cache).  Row r belongs to subdomain r / rows_per_sub.  Start layer k with Lam^(k): init_mode 0
// explicit lam_init [R x n_k], 1 spec rows C[r % m] (bias t[r % m]), 2 stacked +/- identity
// (row r -> +e_{r % n_k} for r < n_k, else -e).  Relaxation of hidden neuron g: per-subdomain
// (l, u, mask)[sub * U + slot_of[g]] when slot_of and l are given and the neuron is cached, else
// the root arrays.  Outputs (all optional): lower (rounded down), lower64, err (pad), lam0
// [R x n0], bias_out (bias - pad, rounded down), bias_raw / pad_raw (FP64), keepP[i] [R x n_{i-1}]
// (the products P^(i), i = 2..k, for the alpha adjoint).  lamA/lamB [R x wmax] and the partial
// buffers are scratch.  bab_weight [nsub x U] (T = float, needs keepP): the BaBSR weight of every
// cached neuron (cv_babsr_weight_layer after each layer i > 1 on keepP[i]).
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
                        T* const* keepP, cudaStream_t st, float* bab_weight = nullptr,
                        const float* beta = nullptr, const int8_t* bsign = nullptr);
// BaBSR weight of the cached neurons of hidden layer i-1 from the layer product P^(i) [R x N]
// (R = nsub m rows): w[sub, slot_of[hoff + q]] = (sum_{r < m} P[sub m + r, q]) / m, the sum in
// FP32 in increasing r (cv_backward.cu); subdomains with skip[sub] set are left untouched.
cv_status cv_babsr_weight_layer(int nsub, int m, int N, int hoff, const int* slot_of, int U, const float* P,
                                const uint8_t* skip, float* w, cudaStream_t st);
int cv_bwd_ncb_max(const cv_net* net);
cv_status cv_bwd_spec_init(int R, int nk, int m, const float* C, const float* t, const float* bk, const float* Vk,
                           float* A, double* acc_bias, double* acc_pad, double gam, cudaStream_t st);
cv_status cv_bwd_reduce(int R, int ncb, const double* part_bias, const double* part_pad, double* acc_bias,
                        double* acc_pad, double gam, cudaStream_t st);
cv_status cv_bwd_final(int R, int ncb, int rows_per_sub, const double* part_f, const double* part_fmag,
                       const double* acc_bias, const double* acc_pad, const uint8_t* skip, float* lower, float* err,
                       float* bias_out, double fm_gamma, cudaStream_t st);

