// sl_remap2d.cu -- launchers of the persistent 2-D FP32 remap with TMA-staged windows
// (sl_remap2d.cuh): tensor maps of the field planes and the displacement, one CTA (or two) per SM;
// the tensor-map encoder shared with the staged 3-D kernel.
#include <mutex>
#include <string.h>

#include "sl_remap2d.cuh"

typedef CUresult (*EncodeTiledFn)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *, const cuuint64_t *,
                                  const cuuint64_t *, const cuuint32_t *, const cuuint32_t *, CUtensorMapInterleave,
                                  CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

// cuTensorMapEncodeTiled from the driver, found through the runtime (no link against libcuda)
static EncodeTiledFn encode_fn()
{
    static EncodeTiledFn fn = nullptr;
    static std::once_flag once;
    std::call_once(once, [] {
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = (EncodeTiledFn)p;
    });
    return fn;
}

bool encode_tensor_f32(CUtensorMap *m, const void *base, int rank, const unsigned long long *dims,
                       const unsigned long long *strides, const unsigned *box)
{
    EncodeTiledFn fn = encode_fn();
    if (!fn || rank < 2 || rank > 3 || ((uintptr_t)base & 15u) != 0 || (box[0] * 4u) % 16u != 0) return false;
    cuuint64_t d[3], st[2];
    cuuint32_t b[3], es[3];
    for (int k = 0; k < rank; ++k) {
        d[k] = dims[k];
        b[k] = box[k];
        es[k] = 1;
        if (k + 1 < rank) {
            if (strides[k] % 16 != 0) return false;
            st[k] = strides[k];
        }
    }
    return fn(m, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, (cuuint32_t)rank, const_cast<void *>(base), d, st, b, es,
              CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
              CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

// a FP32 matrix of `w` x `h` values, rows `w` values apart, copied in boxes of bw x bh
static bool encode_f32(CUtensorMap *m, const void *base, unsigned long long w, unsigned long long h, unsigned bw,
                       unsigned bh)
{
    const unsigned long long dims[2] = {w, h}, strides[1] = {w * 4};
    const unsigned box[2] = {bw, bh};
    return encode_tensor_f32(m, base, 2, dims, strides, box);
}

template <class Cfg, int NF, bool FUSED>
static cudaError_t launch_r2_nf(const sl_grid *g, const R2Args &A, const R2Maps &maps, const VelArgs<float> &vn,
                                cudaStream_t s)
{
    static bool configured[64] = {};
    cudaError_t e = allow_smem(remap2d_tma_kernel<Cfg, NF, FUSED>, g->device, Cfg::SMEM, configured);
    if (e != cudaSuccess) return e;
    const int ctas = (int)std::min<long long>(A.ntiles, (long long)g->num_sms * Cfg::MINB);
    remap2d_tma_kernel<Cfg, NF, FUSED><<<ctas, Cfg::NT, Cfg::SMEM, s>>>(A, maps, vn);
    return cudaGetLastError();
}

template <class Cfg>
static cudaError_t launch_r2(const sl_grid *g, const void *D, void *D_next, double t_next, double dt, bool fused,
                             const void *const *in, void *const *out, cudaStream_t s)
{
    R2Args A;
    memset(&A, 0, sizeof(A));
    A.t = make_tile_args(g, D, D_next, in, out);
    const long long n0 = g->n[0], n1 = g->n[1];
    A.tiles_x = (int)((n0 + Cfg::TX - 1) / Cfg::TX);
    A.ntiles = A.tiles_x * (int)((n1 + Cfg::TY - 1) / Cfg::TY);
    A.timeouts = &g->counters->timeouts;
    R2Maps maps;
    memset(&maps, 0, sizeof(maps));
    bool tma = true;
    for (int f = 0; f < g->nfields; ++f) tma = tma && encode_f32(&maps.f[f], in[f], n0, n1, Cfg::WX, Cfg::WY);
    tma = tma && encode_f32(&maps.D, D, 2 * n0, n1, 2 * Cfg::WX, Cfg::WY);
    A.use_tma = tma ? 1 : 0;
    VelArgs<float> vn;
    memset(&vn, 0, sizeof(vn));
    if (fused) vn = make_vel_args<float>(g, t_next, dt);
    switch (g->nfields) {
    case 1: return fused ? launch_r2_nf<Cfg, 1, true>(g, A, maps, vn, s) : launch_r2_nf<Cfg, 1, false>(g, A, maps, vn, s);
    case 2: return fused ? launch_r2_nf<Cfg, 2, true>(g, A, maps, vn, s) : launch_r2_nf<Cfg, 2, false>(g, A, maps, vn, s);
    default: return fused ? launch_r2_nf<Cfg, 3, true>(g, A, maps, vn, s) : launch_r2_nf<Cfg, 3, false>(g, A, maps, vn, s);
    }
}

// The TMA-staged kernel serves 2-D FP32 grids with at most 3 fields, cubic or linear Z-splines and
// an analytic velocity (a carried one writes the next displacement from the remapped fields,
// which this kernel does not do), an even row length and 16-byte aligned planes (the pair stores
// and the displacement loads are 8 and 16 bytes wide).
bool remap2d_tma_supported(const sl_grid *g, const void *const *in, void *const *out)
{
    if (g->dim != 2 || g->dtype != SL_F32 || g->desc.max_order > 1 || g->nfields > 3 || g->carried || g->nlsw)
        return false;
    if (g->n[0] % 2 != 0 || g->desc.walk_start != SL_START_BACKWARD) return false;
    for (int f = 0; f < g->nfields; ++f)
        if (((uintptr_t)in[f] & 15u) != 0 || ((uintptr_t)out[f] & 7u) != 0) return false;
    return true;
}

cudaError_t launch_remap2d_tma(const sl_grid *g, int config, const void *D, void *D_next, double t_next, double dt,
                               bool fused, const void *const *in, void *const *out, cudaStream_t s)
{
    if (config == 7) return launch_r2<R2Square>(g, D, D_next, t_next, dt, fused, in, out, s);
    return launch_r2<R2Wide>(g, D, D_next, t_next, dt, fused, in, out, s);
}
