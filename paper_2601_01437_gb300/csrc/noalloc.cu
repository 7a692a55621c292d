// lm_apply_pencil_noalloc: the FP64 pencil product for callers that cannot
// allocate device memory.
//
// Some callers of this library cannot call cudaMalloc at the point where they
// need a pencil product: a framework whose caching allocator has reserved the
// device memory and forbids allocations behind its back, an embedded solver
// that was given a fixed memory budget at start-up, or a time-critical loop
// that cannot afford the device-wide synchronisation an allocation or a free
// may cause. lm_apply_pencil needs a pencil handle whose buffers the library
// allocated; this entry point instead takes the caller's O_c, G'_c, weights, v
// and outputs, and keeps its own scratch (the per-CTA partial products, the
// zero-padded copy of v and a status word) in one file-scope device array of
// fixed size. Every GPU that loads the library holds that array until the
// process exits.
#include <algorithm>
#include <mutex>

#include "internal.cuh"

// Scratch: LM_NOALLOC_SCRATCH_DOUBLES doubles (4 MiB), 256-byte aligned.
// Layout per call: [0, 32) status words, [32, 32 + ld) padded v,
// [32 + ld_pad, ...) grid x 2 ld partial products.
#define LM_NOALLOC_SCRATCH_DOUBLES (1u << 19)  // 4 MiB
static __device__ __align__(256) double g_noalloc_scratch[LM_NOALLOC_SCRATCH_DOUBLES];

namespace {

struct NoallocDevice {
    bool ready;
    double *scratch;  // device address of g_noalloc_scratch on this device
    int sms;
    int smem_optin;
};

std::mutex g_noalloc_mu;
NoallocDevice g_noalloc_dev[256];

// Once per device, with that device current: resolve the array's device
// address (host code cannot use the symbol itself) and cache the attributes.
int noalloc_setup(int dev, NoallocDevice **out) {
    if (dev < 0 || dev >= 256) return LM_ERR_ARG;
    std::lock_guard<std::mutex> lock(g_noalloc_mu);
    NoallocDevice &d = g_noalloc_dev[dev];
    if (!d.ready) {
        void *ptr = nullptr;
        if (cudaGetSymbolAddress(&ptr, g_noalloc_scratch) != cudaSuccess) {
            cudaGetLastError();
            return LM_ERR_CUDA;
        }
        if (cudaDeviceGetAttribute(&d.sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
            cudaDeviceGetAttribute(&d.smem_optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) !=
                cudaSuccess)
            return LM_ERR_CUDA;
        d.scratch = static_cast<double *>(ptr);
        d.ready = true;
    }
    *out = &d;
    return LM_OK;
}

// Clear the status words and stage v (p1 entries) zero-padded to ld.
__global__ void k_noalloc_prep(double *scratch, const double *v, int p1, int ld) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < 32) scratch[i] = 0.0;
    if (i < ld) scratch[32 + i] = i < p1 ? v[i] : 0.0;
}

// A device array of the current device `dev` (or managed memory). Memory of
// another GPU is refused: the kernel would read it over the peer path, which
// faults when peer access is not enabled.
bool on_device(const void *p, int dev) {
    if (!p) return false;
    cudaPointerAttributes at;
    if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    if (at.type == cudaMemoryTypeManaged) return true;
    return at.type == cudaMemoryTypeDevice && at.device == dev;
}

}  // namespace

extern "C" int lm_apply_pencil_noalloc(const double *O_c, const double *G_c, const double *w,
                                       int64_t n_rows, int ld, int p1, const double *v,
                                       double *Hv, double *Sv, int sym, void *stream) {
    if (!O_c || !G_c || !w || !v || (!Hv && !Sv)) return LM_ERR_ARG;
    if (n_rows < 1 || p1 < 1 || ld < p1 || ld % 8 != 0) return LM_ERR_SIZE;
    if (ld > LM_NOALLOC_MAX_LD) return LM_ERR_SIZE;
    if (sym != LM_SYM_NONE && sym != LM_SYM_HALF) return LM_ERR_ARG;
    // the kernel copies whole rows with the bulk-copy engine: 16-byte aligned starts
    if ((reinterpret_cast<uintptr_t>(O_c) | reinterpret_cast<uintptr_t>(G_c)) % 16 != 0)
        return LM_ERR_ARG;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return LM_ERR_CUDA;
    if (!on_device(O_c, dev) || !on_device(G_c, dev) || !on_device(w, dev) ||
        !on_device(v, dev) || (Hv && !on_device(Hv, dev)) || (Sv && !on_device(Sv, dev)))
        return LM_ERR_ARG;
    NoallocDevice *d = nullptr;
    if (int rc = noalloc_setup(dev, &d)) return rc;
    // partial products of at most as many CTAs as fit beside v in the array
    const int64_t ld_pad = (ld + 31) / 32 * 32;
    const int64_t room = (int64_t)LM_NOALLOC_SCRATCH_DOUBLES - 32 - ld_pad;
    const int grid = (int)std::min<int64_t>(d->sms, room / (2 * (int64_t)ld));
    if (grid < 1) return LM_ERR_SIZE;
    cudaStream_t s = (cudaStream_t)stream;
    double *scratch = d->scratch;
    int *flags = reinterpret_cast<int *>(scratch);
    double *vpad = scratch + 32;
    double *part = scratch + 32 + ld_pad;
    k_noalloc_prep<<<(std::max(ld, 32) + 255) / 256, 256, 0, s>>>(scratch, v, p1, ld);
    if (cudaGetLastError() != cudaSuccess) return LM_ERR_CUDA;
    return lm_pencil_fp64_on_scratch(O_c, G_c, w, n_rows, ld, p1, vpad, part, grid,
                                     sym == LM_SYM_HALF, Hv, Sv, d->smem_optin, flags, s);
}
