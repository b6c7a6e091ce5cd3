// tm_field_norm2_noalloc: the squared-norm reduction of tm_field_norm2 for
// callers that cannot allocate device memory when they need a norm.
//
// Who cannot allocate, and why:
// - a host framework that has reserved the whole device memory budget for its
//   own pool allocator: a side cudaMalloc from a library either fails outright
//   or takes memory the pool has already promised elsewhere;
// - a latency-critical loop (a solver driven from an outer integrator, a serving
//   step) that must never reach the device allocator, because cudaMalloc and
//   cudaFree can synchronise the whole device.
// The existing tm_field_norm2 keeps its block partials in reduction scratch that
// tm_create allocated; this variant keeps them instead in a fixed array in the
// library's own device memory (below), so a call allocates nothing.
//
// The array is NOALLOC_MAX_BLOCKS partial sums plus the last-block counter
// (about 512 KB). Every GPU that loads the library holds it until the process
// exits. Fields are limited to NOALLOC_MAX_BLOCKS * BLAS_BS = 16,777,216 sites
// per parity; larger fields are rejected with TM_ERR_ARG. The field and the
// result must be device memory: other pointers are rejected with TM_ERR_ARG
// before anything is launched.
#include <mutex>

#include "tm_host.h"

using namespace tmk;

namespace tmk {
tm_status tmk_fail_msg(tm_status s, const char* msg);   // records tm_last_error (api.cu)
}

constexpr int NOALLOC_MAX_BLOCKS = 65536;

// [0, NOALLOC_MAX_BLOCKS): per-block partial sums; the next 8 bytes: counter
static __device__ __align__(256) double tm_noalloc_scratch[NOALLOC_MAX_BLOCKS + 32];

static std::mutex g_noalloc_mu;

// device (or managed) memory, as the kernel needs; cudaPointerGetAttributes
// allocates nothing
static bool noalloc_device_ptr(const void* p) {
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}
static double* g_noalloc_addr[256] = {};   // device address of the array, per device ordinal

// Device address of the scratch array on the current device (looked up once per
// device; host code may not use the symbol itself as a device address).
static tm_status noalloc_scratch(int device, double** out) {
    if (device < 0 || device >= 256) return tmk_fail_msg(TM_ERR_ARG, "tm_field_norm2_noalloc: device ordinal out of range");
    std::lock_guard<std::mutex> lock(g_noalloc_mu);
    if (!g_noalloc_addr[device]) {
        void* p = nullptr;
        const cudaError_t e = cudaGetSymbolAddress(&p, tm_noalloc_scratch);
        if (e != cudaSuccess) return tmk_fail_msg(TM_ERR_CUDA, cudaGetErrorString(e));
        g_noalloc_addr[device] = reinterpret_cast<double*>(p);
    }
    *out = g_noalloc_addr[device];
    return TM_OK;
}

template <int P>
static cudaError_t noalloc_launch(const tm_ctx* c, int nf, const void* f, double* res, double* partial,
                                  unsigned int* counter, cudaStream_t st) {
    VecBatch<1> b{};
    b.n = 1;
    b.fin = FIN_STORE;
    const int nb = (int)((c->vh + BLAS_BS - 1) / BLAS_BS);
    b.blk_start[0] = 0;
    b.blk_start[1] = nb;
    b.p[0].vh = c->vh;
    b.p[0].nblk = nb;
    b.p[0].v[0] = const_cast<void*>(f);
    b.p[0].partial = partial;
    b.p[0].counter = counter;
    b.p[0].dst = res;
    return nf == 1 ? launch_norm2<P, 12, 1>(b, nb, st) : launch_norm2<P, 24, 1>(b, nb, st);
}

extern "C" tm_status tm_field_norm2_noalloc(const tm_ctx* c, tm_prec prec, int nf, const void* field, double* result,
                                            void* stream) {
    if (!c || !field || !result || (nf != 1 && nf != 2))
        return tmk_fail_msg(TM_ERR_ARG, "tm_field_norm2_noalloc: bad argument");
    if (((uintptr_t)field & 15) || ((uintptr_t)result & 7))
        return tmk_fail_msg(TM_ERR_ARG, "tm_field_norm2_noalloc: misaligned pointer");
    if (prec < TM_F64 || prec > TM_F16) return tmk_fail_msg(TM_ERR_ARG, "tm_field_norm2_noalloc: unknown precision");
    if (c->vh > (long)NOALLOC_MAX_BLOCKS * BLAS_BS)
        return tmk_fail_msg(TM_ERR_ARG,
                            "tm_field_norm2_noalloc: field too large (at most 16777216 sites per parity); "
                            "use tm_field_norm2");
    cudaError_t e = cudaSetDevice(c->device);
    if (e != cudaSuccess) return tmk_fail_msg(TM_ERR_CUDA, cudaGetErrorString(e));
    if (!noalloc_device_ptr(field) || !noalloc_device_ptr(result))
        return tmk_fail_msg(TM_ERR_ARG, "tm_field_norm2_noalloc: field and result must be device pointers");
    double* scratch = nullptr;
    const tm_status s = noalloc_scratch(c->device, &scratch);
    if (s != TM_OK) return s;
    unsigned int* counter = reinterpret_cast<unsigned int*>(scratch + NOALLOC_MAX_BLOCKS);
    const cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    // the last-block counter must start at zero (the kernel leaves it at zero, but
    // an earlier call that failed mid-way might not have)
    e = cudaMemsetAsync(counter, 0, sizeof(unsigned int), st);
    if (e == cudaSuccess) {
        switch (prec) {
            case TM_F64: e = noalloc_launch<P64>(c, nf, field, result, scratch, counter, st); break;
            case TM_F32: e = noalloc_launch<P32>(c, nf, field, result, scratch, counter, st); break;
            case TM_BF16: e = noalloc_launch<PB16>(c, nf, field, result, scratch, counter, st); break;
            default: e = noalloc_launch<PF16>(c, nf, field, result, scratch, counter, st); break;
        }
    }
    if (e != cudaSuccess) return tmk_fail_msg(TM_ERR_CUDA, cudaGetErrorString(e));
    return TM_OK;
}
