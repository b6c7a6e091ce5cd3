// Device geometry and launchers of the parallel-transport network kernels (ptc.cu).
#pragma once

#include "tm_internal.h"

namespace tmk {

constexpr int PTC_MAXC = 8;                // channels per layer

struct PtcGeom {
    int X, Y, Z, T;
    long V, vh;
    float bc_t;
    const void* gauge[2];   // FP16 native links per parity
    const uint32_t* lp;     // transport links of paths 1..8, FP16 (re, im) pairs [8][9][V]
                            // (U^dagger for backward paths, time boundary phase included)
};

// one layer on the tensor cores; *err is set to 1 if a wait on the tensor cores ran
// out of its bound (the layer's output is then incomplete).  Layers with one
// output channel and cin > 1 mix first into zbuf (9 x 3 x 16 bytes per site)
// and transport it afterwards; other layers ignore zbuf.
cudaError_t launch_ptc_layer(int cin, int cout, const PtcGeom& g, const void* in, void* out, const void* wemb,
                             int nsm, int* err, void* zbuf, cudaStream_t st);
// weight gradient of one layer into grad (scaled, accumulated); partial holds
// 9 * 4096 floats per block, min(nsm, sites / 32) blocks
// lp[(p - 1) * 9 + 3 c + d][x] from the FP16 even-odd links of g
cudaError_t launch_ptc_links(const PtcGeom& g, uint32_t* lp, cudaStream_t st);
cudaError_t launch_ptc_wgrad(int cin, int cout, const PtcGeom& g, const void* in, const void* delta, float* partial,
                             int nsm, float2* grad, float scale, int* err, cudaStream_t st);
cudaError_t launch_ptc_embed_weights(const float2* W, int cin, int cout, void* fwd, void* adj, cudaStream_t st);
cudaError_t launch_ptc_adam(float2* W, float2* m, float2* v, float2* grad, int n, float lr, float b1, float b2,
                            float eps, int step, cudaStream_t st);
cudaError_t launch_ptc_embed_odd(int prec, const void* r, void* a0, const PtcGeom& g, cudaStream_t st);
cudaError_t launch_ptc_extract_odd(int prec, const void* a, void* z, const PtcGeom& g, cudaStream_t st);
// loss sum ||z - e||^2 -> *out, delta = (z - e) / *ee on odd sites (0 elsewhere)
cudaError_t launch_ptc_loss_delta(const void* aL, const void* e, void* delta, const PtcGeom& g, const double* ee,
                                  double* partial, double* out, cudaStream_t st);
// one thread waits (bounded by bound_ns) on an mbarrier nobody arrives on; *out = 1 if the bound ran out
cudaError_t launch_ptc_wait_selftest(long long bound_ns, int* out, cudaStream_t st);
cudaError_t launch_ptc_gauss_odd(void* e, long vh, unsigned long long seed, unsigned long long stream,
                                 cudaStream_t st);

// complex BLAS-1 used by flexible CG (single problem, FP32 fields)
cudaError_t launch_cdot32(const void* a, const void* b, long vh, double* partial, unsigned int* counter,
                          double* dst2, cudaStream_t st);
cudaError_t launch_caxpy32(void* y, const void* x, double ar, double ai, long vh, cudaStream_t st);
cudaError_t launch_cxpay32(void* y, const void* x, double br, double bi, long vh, cudaStream_t st);

}  // namespace tmk
