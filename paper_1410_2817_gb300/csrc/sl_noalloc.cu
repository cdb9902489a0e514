// sl_noalloc.cu -- discrete moments of one field plane for callers that cannot allocate device
// memory.  The reduction's scratch (per-block partial sums and the final sums) lives in a
// fixed-size file-scope device array instead of a caller-supplied workspace.
#include <mutex>
#include <string.h>

#include "sl_internal.h"

// Scratch of sl_moments_noalloc: SL_MOMENT_BLOCKS rows of 8 partial sums, then the 8 final sums
// (about 33 KB).  Every GPU that loads libsl.so holds this array until the process exits, and
// every call on that GPU shares it.
static __device__ __align__(256) double g_noalloc_scratch[SL_MOMENT_BLOCKS * 8 + 8];

// Device address of the scratch array on the current device.  The host-side name of a
// __device__ variable is only a stand-in, so the address is looked up with that device current.
// Outside stream capture it is looked up on every call (a cheap table lookup once the module is
// loaded), so that a reset of the device's primary context between calls, which moves the array,
// is picked up; the last address seen on each device is kept for calls made while `s` is being
// captured, where no lookup is made.  A first call on a device inside a capture therefore fails
// with cudaErrorStreamCaptureUnsupported.
static cudaError_t scratch_address(int device, cudaStream_t s, double **out)
{
    static std::mutex mu;
    static double *addr[64];
    static bool ready[64];
    if (device < 0 || device >= 64) return cudaErrorInvalidDevice;
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    cudaError_t e = cudaStreamIsCapturing(s, &cs);
    if (e != cudaSuccess) return e;
    std::lock_guard<std::mutex> lock(mu);
    if (cs == cudaStreamCaptureStatusNone) {
        double *p = nullptr;
        e = cudaGetSymbolAddress((void **)&p, g_noalloc_scratch);
        if (e != cudaSuccess) return e;
        addr[device] = p;
        ready[device] = true;
    } else if (!ready[device]) {
        return cudaErrorStreamCaptureUnsupported;
    }
    *out = addr[device];
    return cudaSuccess;
}

// record the reason where sl_last_error() finds it, as every other entry point does
static sl_status noalloc_fail(sl_status st, const char *why)
{
    sl_record_error(st == SL_ERR_ARG ? "sl_moments_noalloc: invalid argument" : "sl_moments_noalloc", why);
    return st;
}

extern "C" sl_status sl_moments_noalloc(int dim, const int64_t n[3], const double lo[3], const double hi[3], int dtype,
                                        const void *field, int pmax, double *host_out, void *stream)
{
    if (dim != 2 && dim != 3) return noalloc_fail(SL_ERR_ARG, "dim must be 2 or 3");
    if (!n || !lo || !hi || !field || !host_out) return noalloc_fail(SL_ERR_ARG, "NULL argument");
    if (dtype != SL_F64 && dtype != SL_F32) return noalloc_fail(SL_ERR_ARG, "dtype must be SL_F64 or SL_F32");
    if (pmax < 0 || pmax > 7)
        return noalloc_fail(SL_ERR_ARG, "pmax must be in [0, 7]: the static scratch holds 8 moments per block");
    long long N = 1;
    for (int a = 0; a < dim; ++a) {
        if (n[a] < 1 || n[a] > (1 << 20)) return noalloc_fail(SL_ERR_ARG, "each n[a] must be in [1, 2^20]");
        if (!(hi[a] > lo[a])) return noalloc_fail(SL_ERR_ARG, "hi must exceed lo on every axis");
        N *= n[a];
    }
    if (N > (1LL << 31) - 1) return noalloc_fail(SL_ERR_ARG, "too many nodes (limit 2^31 - 1)");
    const size_t tsize = dtype == SL_F64 ? 8 : 4;
    if (((uintptr_t)field % tsize) != 0) return noalloc_fail(SL_ERR_ARG, "field is not aligned to its dtype");

    int device = 0;
    cudaError_t e = cudaGetDevice(&device);
    double *scratch = nullptr;
    if (e == cudaSuccess) e = scratch_address(device, (cudaStream_t)stream, &scratch);
    if (e != cudaSuccess) return noalloc_fail(SL_ERR_CUDA, cudaGetErrorString(e));

    // a host-side grid object that carries only what the moments launcher reads
    sl_grid g;
    memset(&g, 0, sizeof(g));
    g.dim = dim;
    g.dtype = dtype;
    g.nfields = 1;
    g.N = 1;
    for (int a = 0; a < 3; ++a) {
        g.n[a] = a < dim ? n[a] : 1;
        g.N *= g.n[a];
        g.desc.lo[a] = a < dim ? lo[a] : 0.0;
        g.desc.hi[a] = a < dim ? hi[a] : 1.0;
        g.dx[a] = a < dim ? (hi[a] - lo[a]) / (double)n[a] : 1.0;
    }
    g.device = device;
    g.partials = scratch;
    g.moment_out = scratch + SL_MOMENT_BLOCKS * 8;

    cudaStream_t s = (cudaStream_t)stream;
    e = dtype == SL_F64 ? Launch<double>::moments(&g, field, pmax, s) : Launch<float>::moments(&g, field, pmax, s);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(host_out, g.moment_out, sizeof(double) * (pmax + 1), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return noalloc_fail(SL_ERR_CUDA, cudaGetErrorString(e));
    return SL_OK;
}
