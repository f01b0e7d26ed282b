// Input branch and bound: the split step of Algorithm 4 (Domain_Filter, then Batch_Split with the
// parent's final-layer hyperplane shared by both children; Section 3.3, final-layer bounds as
// clipping constraints).  The rules, in the order the header states them:
//  - a verified or infeasible parent is dropped; kept parents give children 2k and 2k + 1 in order;
//  - the split axis maximises (hi_i - lo_i) * sum_{unproven r} |A_r,i| (FP32, rows in increasing r,
//    the first maximum), the widest axis when no score is positive;
//  - the split point is fl(fl(lo + hi) * 0.5);
//  - with exactly one unproven spec row r, both children get the row A_r . x + c_r <= 0.
// The axis and the split point are FP32 decisions taken with explicitly rounded operations in the
// oracle's order, so they match it bit for bit.
//
// GB300 mapping: three launches.  k_split_mark (one block per parent) reads the parent's planes
// once to score the axes; a one-block scan places the children and their rows; k_split_write (one
// block per parent) streams the children's boxes and rows out.  The step is HBM-bound: per parent
// it reads the box and the m planes and writes two boxes and at most two rows.
#include "cv_internal.cuh"

#include <string>

namespace {

struct SplitWs {
    int* keep;    // [B] 1 for a kept parent
    int* axis;    // [B]
    int* row1;    // [B] the single unproven row, or -1 (none or several)
    int* cpos;    // [B] index of the parent's first child / 2 (exclusive prefix of keep)
    int* rpos;    // [B] index of the parent's first row (exclusive prefix of 2 * [row1 >= 0])
};

__device__ __forceinline__ bool better(float s, int i, float bs, int bi) {
    return s > bs || (s == bs && i < bi);
}

// one block per parent: keep flag, single unproven row, split axis.  The unproven rows are listed
// in shared memory (dynamic, m ints) first; each thread then scores four consecutive axes with one
// 16-byte load per row when n0 is a multiple of 4 and the planes are 16-byte aligned (independent loads; the sum of every axis still
// runs over the rows in increasing order), else one axis at a time.
__global__ void k_split_mark(int B, int n0, int m, const float* lo, const float* hi, const float* A,
                             const float* lower, const uint8_t* verified, const uint8_t* infeasible, SplitWs w) {
    extern __shared__ int s_rows[];
    const int b = blockIdx.x;
    __shared__ float rs[32];
    __shared__ int ri[32];
    __shared__ int s_nun;
    const bool keep = !verified[b] && !infeasible[b];
    if (!keep) {
        if (threadIdx.x == 0) { w.keep[b] = 0; w.axis[b] = 0; w.row1[b] = -1; }
        return;
    }
    const float* lb = lower + (size_t)b * m;
    for (int r = threadIdx.x; r < m; r += blockDim.x) s_rows[r] = !(lb[r] > 0.f);
    __syncthreads();
    if (threadIdx.x == 0) {
        int nun = 0;
        for (int r = 0; r < m; ++r)
            if (s_rows[r]) s_rows[nun++] = r;  // in place: nun <= r
        s_nun = nun;
    }
    __syncthreads();
    const int nun = s_nun;
    const float* l = lo + (size_t)b * n0;
    const float* u = hi + (size_t)b * n0;
    const float* Ab = A + (size_t)b * m * n0;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    const bool vec = (n0 & 3) == 0 && ((uintptr_t)A & 15) == 0;  // 16-byte aligned rows
    for (int pass = 0; pass < 2; ++pass) {
        // pass 0: plane extents; pass 1 (only when no extent is positive): widths
        float bs = -1.f;
        int bi = 0x7fffffff;
        if (vec) {
            for (int i4 = threadIdx.x; 4 * i4 < n0; i4 += blockDim.x) {
                const int i = 4 * i4;
                float acc[4] = {0.f, 0.f, 0.f, 0.f};
                if (pass == 0) {
#pragma unroll 4
                    for (int q = 0; q < nun; ++q) {
                        const float4 v = __ldg((const float4*)(Ab + (size_t)s_rows[q] * n0 + i));
                        acc[0] = __fadd_rn(acc[0], fabsf(v.x));
                        acc[1] = __fadd_rn(acc[1], fabsf(v.y));
                        acc[2] = __fadd_rn(acc[2], fabsf(v.z));
                        acc[3] = __fadd_rn(acc[3], fabsf(v.w));
                    }
                }
#pragma unroll
                for (int e = 0; e < 4; ++e) {
                    const float wd = __fsub_rn(u[i + e], l[i + e]);
                    const float sc = (pass == 0) ? __fmul_rn(wd, acc[e]) : wd;
                    if (sc > bs) { bs = sc; bi = i + e; }  // increasing axis: the first maximum
                }
            }
        } else {
            for (int i = threadIdx.x; i < n0; i += blockDim.x) {
                const float wd = __fsub_rn(u[i], l[i]);
                float sc = wd;
                if (pass == 0) {
                    float acc = 0.f;
                    for (int q = 0; q < nun; ++q) acc = __fadd_rn(acc, fabsf(Ab[(size_t)s_rows[q] * n0 + i]));
                    sc = __fmul_rn(wd, acc);
                }
                if (sc > bs) { bs = sc; bi = i; }
            }
        }
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) {
            const float os = __shfl_xor_sync(0xffffffffu, bs, off);
            const int oi = __shfl_xor_sync(0xffffffffu, bi, off);
            if (better(os, oi, bs, bi)) { bs = os; bi = oi; }
        }
        if (lane == 0) { rs[warp] = bs; ri[warp] = bi; }
        __syncthreads();
        float fs = -1.f;
        int fi = 0x7fffffff;
        for (int q = 0; q < nw; ++q)
            if (better(rs[q], ri[q], fs, fi)) { fs = rs[q]; fi = ri[q]; }
        __syncthreads();
        if (pass == 0 && fs > 0.f) {
            if (threadIdx.x == 0) { w.keep[b] = 1; w.axis[b] = fi; w.row1[b] = (nun == 1) ? s_rows[0] : -1; }
            return;
        }
        if (pass == 1 && threadIdx.x == 0) {
            w.keep[b] = 1;
            w.axis[b] = (fi == 0x7fffffff) ? 0 : fi;
            w.row1[b] = (nun == 1) ? s_rows[0] : -1;
        }
    }
}

// one block: exclusive prefixes of the kept parents and of their rows; totals
__global__ void __launch_bounds__(1024) k_split_scan(int B, SplitWs w, int* row_off, int* n_children) {
    __shared__ int sc[1024], sr[1024];
    const int tid = threadIdx.x, nt = blockDim.x;
    const int per = (B + nt - 1) / nt;
    int c = 0, r = 0;
    for (int i = 0; i < per; ++i) {
        const int b = tid * per + i;
        if (b < B && w.keep[b]) { ++c; r += (w.row1[b] >= 0) ? 2 : 0; }
    }
    sc[tid] = c;
    sr[tid] = r;
    __syncthreads();
    for (int off = 1; off < nt; off <<= 1) {
        const int tc = tid >= off ? sc[tid - off] : 0;
        const int tr = tid >= off ? sr[tid - off] : 0;
        __syncthreads();
        sc[tid] += tc;
        sr[tid] += tr;
        __syncthreads();
    }
    int pc = sc[tid] - c, pr = sr[tid] - r;
    for (int i = 0; i < per; ++i) {
        const int b = tid * per + i;
        if (b < B) {
            w.cpos[b] = pc;
            w.rpos[b] = pr;
            if (w.keep[b]) { ++pc; pr += (w.row1[b] >= 0) ? 2 : 0; }
        }
    }
    if (tid == 0) {
        *n_children = 2 * sc[nt - 1];
        row_off[0] = 0;
    }
}

// one block per parent: the two children's boxes, rows, row offsets and parent index
__global__ void k_split_write(int B, int n0, int m, const float* lo, const float* hi, const float* A, const float* c,
                              SplitWs w, float* lo_out, float* hi_out, int* row_off, float* G, float* h,
                              int* parent) {
    const int b = blockIdx.x;
    if (!w.keep[b]) return;
    const int ax = w.axis[b], r1 = w.row1[b];
    const int ch0 = 2 * w.cpos[b];
    const int rp = w.rpos[b];
    const float* l = lo + (size_t)b * n0;
    const float* u = hi + (size_t)b * n0;
    const float mid = __fmul_rn(__fadd_rn(l[ax], u[ax]), 0.5f);
    for (int k = 0; k < 2; ++k) {
        float* lo2 = lo_out + (size_t)(ch0 + k) * n0;
        float* hi2 = hi_out + (size_t)(ch0 + k) * n0;
        for (int i = threadIdx.x; i < n0; i += blockDim.x) {
            float a = l[i], z = u[i];
            if (i == ax) {
                if (k == 0) z = mid; else a = mid;
            }
            lo2[i] = a;
            hi2[i] = z;
        }
        if (r1 >= 0) {
            const float* Ar = A + ((size_t)b * m + r1) * n0;
            float* Gr = G + (size_t)(rp + k) * n0;
            for (int i = threadIdx.x; i < n0; i += blockDim.x) Gr[i] = Ar[i];
        }
        if (threadIdx.x == 0) {
            if (r1 >= 0) h[rp + k] = c[(size_t)b * m + r1];
            row_off[ch0 + k + 1] = rp + ((r1 >= 0) ? k + 1 : 0);
            parent[ch0 + k] = b;
        }
    }
}

size_t split_ws_bytes(int B) { return 5 * cv_align256((size_t)(B > 0 ? B : 1) * sizeof(int)); }

}  // namespace

extern "C" cv_status cv_input_split_workspace(int B, size_t* bytes) {
    if (B < 0 || !bytes) { cv_set_error("cv_input_split_workspace: negative B or null bytes"); return CV_EINVAL; }
    *bytes = split_ws_bytes(B);
    return CV_OK;
}

extern "C" cv_status cv_input_split(int B, int n0, int m, const float* lo, const float* hi, const float* final_A,
                                    const float* final_c, const float* lower, const uint8_t* verified,
                                    const uint8_t* infeasible, float* lo_out, float* hi_out, int* row_off, float* G,
                                    float* h, int* parent, int* n_children, void* workspace,
                                    size_t workspace_bytes, void* stream) {
    if (B < 0 || n0 < 1 || m < 1) { cv_set_error("cv_input_split: B < 0, n0 < 1 or m < 1"); return CV_EINVAL; }
    if (!row_off || !n_children) { cv_set_error("cv_input_split: null row_off or n_children"); return CV_EINVAL; }
    cudaStream_t st = (cudaStream_t)stream;
    if (B == 0) {
        CV_CUDA(cudaMemsetAsync(row_off, 0, sizeof(int), st));
        CV_CUDA(cudaMemsetAsync(n_children, 0, sizeof(int), st));
        return CV_OK;
    }
    if (!lo || !hi || !final_A || !final_c || !lower || !verified || !infeasible || !lo_out || !hi_out || !G ||
        !h || !parent || !workspace) {
        cv_set_error("cv_input_split: null argument");
        return CV_EINVAL;
    }
    if (workspace_bytes < split_ws_bytes(B)) {
        cv_set_error("cv_input_split: workspace smaller than cv_input_split_workspace()");
        return CV_EWORKSPACE;
    }
    SplitWs w;
    char* p = (char*)workspace;
    const size_t step = cv_align256((size_t)B * sizeof(int));
    w.keep = (int*)p; p += step;
    w.axis = (int*)p; p += step;
    w.row1 = (int*)p; p += step;
    w.cpos = (int*)p; p += step;
    w.rpos = (int*)p;
    const size_t mark_smem = (size_t)m * sizeof(int);
    if (mark_smem > 48 * 1024) {
        cv_set_error("cv_input_split: more than 12288 spec rows");
        return CV_EINVAL;
    }
    k_split_mark<<<B, 256, mark_smem, st>>>(B, n0, m, lo, hi, final_A, lower, verified, infeasible, w);
    CV_LAUNCH_CHECK("k_split_mark");
    k_split_scan<<<1, 1024, 0, st>>>(B, w, row_off, n_children);
    CV_LAUNCH_CHECK("k_split_scan");
    k_split_write<<<B, 256, 0, st>>>(B, n0, m, lo, hi, final_A, final_c, w, lo_out, hi_out, row_off, G, h, parent);
    CV_LAUNCH_CHECK("k_split_write");
    return CV_OK;
}
