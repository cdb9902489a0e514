// sl_tiled.cu -- dispatch of the FP32 production kernels: 2-D grids go to the persistent kernel with
// TMA-staged windows (sl_remap2d.cuh; tile configurations 0, 6, 7, up to 3 fields, analytic
// velocities) or to the shared-memory tiled kernels (sl_tile2d.cuh, one translation unit per tile
// configuration; the quintic Z-spline to sl_tiled_z2.cu), 3-D grids to the staged or blocked
// kernels (sl_blocked3d.cu, cubic and linear only).
#include <string.h>

#include "sl_internal.h"

// 2-D: one tiled launch; 3-D: flags with the x-OR, the y/z-OR, one staged or blocked launch
int tiled_kernels_per_call(const sl_grid *g) { return g->dim == 2 ? 1 : 3; }

template <typename T>
bool Launch<T>::tiled_supported(const sl_grid *g)
{
    if (sizeof(T) != 4 || g->desc.walk_start != SL_START_BACKWARD) return false;
    // the 2-D tile bodies invert in FP32 (FP64 re-solves only for failed or degenerate targets):
    // an FP64 inversion of every target runs on the plain kernels
    if (g->dim == 2 && g->desc.newton_mode == SL_NEWTON_F64) return false;
    if (g->desc.max_order > 1) return g->dim == 2 && tiled2d_smem_bytes_z2(g->nfields) <= 200 * 1024;
    // the 3-D kernels form 32-bit node offsets; their blocks are at least 4 rows and planes deep
    if (g->dim == 3) return g->N < (1LL << 31) && (g->n[1] + 3) / 4 <= 65535 && (g->n[2] + 3) / 4 <= 65535;
    const int c = g->desc.tile_config;
    const size_t smem = c == 2   ? tiled2d_smem_bytes_cfgb(g->nfields)
                        : c == 3 ? tiled2d_smem_bytes_cfgc(g->nfields)
                        : c == 4 ? tiled2d_smem_bytes_cfgd(g->nfields)
                                 : tiled2d_smem_bytes_cfga(g->nfields);  // 5 falls back to 1 above 4 fields
    return smem <= 200 * 1024;
}

static cudaError_t launch_tiled2d(const sl_grid *g, const void *D, void *D_next, double t_next, double dt, bool fused,
                                  const void *const *in, void *const *out, cudaStream_t s)
{
    if (g->desc.max_order > 1) return launch_tiled2d_z2(g, D, D_next, t_next, dt, fused, in, out, s);
    const int c = g->desc.tile_config;
    if ((c == 0 || c == 6 || c == 7) && remap2d_tma_supported(g, in, out))
        return launch_remap2d_tma(g, c == 6 ? 6 : 7, D, D_next, t_next, dt, fused, in, out, s);
    switch (c) {
    case 5:
        if (g->nfields <= 4) return launch_tiled2d_cfgp(g, D, D_next, t_next, dt, fused, in, out, s);
        return launch_tiled2d_cfga(g, D, D_next, t_next, dt, fused, in, out, s);
    case 2: return launch_tiled2d_cfgb(g, D, D_next, t_next, dt, fused, in, out, s);
    case 3: return launch_tiled2d_cfgc(g, D, D_next, t_next, dt, fused, in, out, s);
    case 4: return launch_tiled2d_cfgd(g, D, D_next, t_next, dt, fused, in, out, s);
    default: return launch_tiled2d_cfga(g, D, D_next, t_next, dt, fused, in, out, s);
    }
}

template <typename T>
cudaError_t Launch<T>::remap_tiled(const sl_grid *g, const void *D, const void *const *in, void *const *out,
                                   cudaStream_t s)
{
    if (!tiled_supported(g)) return cudaErrorNotSupported;
    if (g->dim == 3) {
        cudaError_t e = launch_box_flags3d(g, in, g->flags, g->flags2, s);
        if (e != cudaSuccess) return e;
        return launch_blocked3d(g, D, nullptr, g->flags2, 0.0, 0.0, false, in, out, s);
    }
    return launch_tiled2d(g, D, nullptr, 0.0, 0.0, false, in, out, s);
}

template <typename T>
cudaError_t Launch<T>::step_fused(const sl_grid *g, const void *D, void *D_next, double t_next, double dt,
                                  const void *const *in, void *const *out, cudaStream_t s)
{
    if (!tiled_supported(g)) return cudaErrorNotSupported;
    if (g->dim == 3) {
        cudaError_t e = launch_box_flags3d(g, in, g->flags, g->flags2, s);
        if (e != cudaSuccess) return e;
        return launch_blocked3d(g, D, D_next, g->flags2, t_next, dt, true, in, out, s);
    }
    return launch_tiled2d(g, D, D_next, t_next, dt, true, in, out, s);
}

template bool Launch<double>::tiled_supported(const sl_grid *);
template bool Launch<float>::tiled_supported(const sl_grid *);
template cudaError_t Launch<double>::remap_tiled(const sl_grid *, const void *, const void *const *, void *const *,
                                                 cudaStream_t);
template cudaError_t Launch<float>::remap_tiled(const sl_grid *, const void *, const void *const *, void *const *,
                                                cudaStream_t);
template cudaError_t Launch<double>::step_fused(const sl_grid *, const void *, void *, double, double,
                                                const void *const *, void *const *, cudaStream_t);
template cudaError_t Launch<float>::step_fused(const sl_grid *, const void *, void *, double, double,
                                               const void *const *, void *const *, cudaStream_t);
