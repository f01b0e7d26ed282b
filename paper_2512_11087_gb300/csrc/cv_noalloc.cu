// Allocation-free entry point: constraint rows, pre-check and relaxed clipping with their scratch
// in a fixed device array of this library instead of a caller workspace.
//
// Some callers cannot allocate device memory at the point where they bound subdomains: a host
// framework whose caching allocator or memory pool must own every device byte, or a latency-bound
// loop where cudaMalloc / cudaFree (which can synchronise the device) are not allowed once the run
// has started.  cv_relaxed_clip_static serves them: it calls no cudaMalloc, cudaFree or allocating
// library routine.  Its scratch (a row-status byte and an FP64 row minimum per (subdomain, row)
// slot) lives in cv_static_scratch, a file-scope __device__ array of CV_STATIC_SCRATCH_BYTES that
// every GPU which loads the library holds until the process exits.
//
// Host code cannot pass the array's name to a kernel (on the host it is only a stand-in symbol),
// so the first call on each device, with that device current, looks up its device address with
// cudaGetSymbolAddress and remembers it; make that first call before any stream capture.  All
// calls share the array and it keeps the last call's contents: the row kernel writes every slot it
// later reads, so nothing needs clearing, and calls whose kernels overlap on the GPU race on it.
#include "cv_internal.cuh"

#include <climits>
#include <string.h>

#include <mutex>

namespace {

constexpr int kMaxDevices = 64;

static __device__ __align__(256) unsigned char cv_static_scratch[CV_STATIC_SCRATCH_BYTES];

std::mutex g_lock;
void* g_addr[kMaxDevices] = {nullptr};

cv_status scratch_address(void** out) {
    int dev = 0;
    CV_CUDA(cudaGetDevice(&dev));
    if (dev < 0 || dev >= kMaxDevices) {
        cv_set_error("cv_relaxed_clip_static: device index above the supported maximum");
        return CV_EUNSUPPORTED;
    }
    std::lock_guard<std::mutex> guard(g_lock);
    if (!g_addr[dev]) {
        void* p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, cv_static_scratch);
        if (e != cudaSuccess || !p) return cv_cuda_fail(e, "cudaGetSymbolAddress(cv_static_scratch)");
        g_addr[dev] = p;
    }
    *out = g_addr[dev];
    return CV_OK;
}

}  // namespace

extern "C" cv_status cv_relaxed_clip_static(cv_net* net, const cv_cache* cache, const cv_batch_in* in,
                                            float* lo_clip, float* hi_clip, uint8_t* infeasible, int relaxed,
                                            void* stream) {
    if (!net || !cache || !in || !lo_clip || !hi_clip || !infeasible) {
        cv_set_error("cv_relaxed_clip_static: null argument");
        return CV_EINVAL;
    }
    if (cache->net != net) { cv_set_error("cv_relaxed_clip_static: cache was built for another network"); return CV_EINVAL; }
    if (in->B < 0 || in->max_splits < 0 || in->max_rows < 0) {
        cv_set_error("cv_relaxed_clip_static: negative B, max_splits or max_rows");
        return CV_EINVAL;
    }
    if (in->B > 0 && (!in->lo || !in->hi)) { cv_set_error("cv_relaxed_clip_static: lo/hi required"); return CV_EINVAL; }
    if (!in->split_off && in->split_ids) { cv_set_error("cv_relaxed_clip_static: split_ids without split_off"); return CV_EINVAL; }
    if (in->split_off && !in->split_ids && in->max_splits > 0) {
        cv_set_error("cv_relaxed_clip_static: split_ids required when max_splits > 0");
        return CV_EINVAL;
    }
    if ((!in->split_off && in->max_splits > 0) || (!in->row_off && in->max_rows > 0) ||
        (in->row_off && (!in->G || !in->h) && in->max_rows > 0)) {
        cv_set_error("cv_relaxed_clip_static: inconsistent split / row arguments");
        return CV_EINVAL;
    }
    if ((long long)in->max_splits + in->max_rows > INT_MAX ||
        (long long)in->B * ((long long)in->max_splits + in->max_rows) > INT_MAX) {
        cv_set_error("cv_relaxed_clip_static: B x (max_splits + max_rows) must fit in int");
        return CV_EINVAL;
    }
    if (in->B == 0) return CV_OK;
    // scratch: row status [B x Rmax] bytes, then row minima [B x Rmax] doubles (256-aligned)
    cv_ws_layout lay;
    memset(&lay, 0, sizeof(lay));
    lay.Rmax = in->max_splits + in->max_rows;
    const size_t slots = (size_t)in->B * (size_t)lay.Rmax;
    lay.rowflag = 0;
    lay.vmin = cv_align256(slots ? slots : 1);
    const size_t need = lay.vmin + slots * sizeof(double);
    if (need > (size_t)CV_STATIC_SCRATCH_BYTES) {
        cv_set_error("cv_relaxed_clip_static: B x (max_splits + max_rows) = " + std::to_string(slots) +
                     " row slots need " + std::to_string(need) + " scratch bytes; the static array holds " +
                     std::to_string((size_t)CV_STATIC_SCRATCH_BYTES));
        return CV_EWORKSPACE;
    }
    void* scratch = nullptr;
    cv_status s = scratch_address(&scratch);
    if (s) return s;
    cudaStream_t st = (cudaStream_t)stream;
    cv_options opt;
    cv_options_default(&opt);
    opt.relaxed = relaxed ? 1 : 0;
    CV_CUDA(cudaMemsetAsync(infeasible, 0, in->B, st));
    if ((s = cv_launch_rows(net, cache, in, &lay, (char*)scratch, infeasible, st))) return s;
    return cv_launch_relaxed(net, cache, in, &opt, &lay, (char*)scratch, lo_clip, hi_clip, infeasible, st);
}
