// sl_tiled_cfg_d.cu -- the 2-D FP32 tiled kernels instantiated for tile configuration CfgD
// (one translation unit per configuration so that they compile in parallel).
#include "sl_tile2d.cuh"

cudaError_t launch_tiled2d_cfgd(const sl_grid *g, const void *D, void *D_next, double t_next, double dt, bool fused,
                                   const void *const *in, void *const *out, cudaStream_t s)
{
    return launch_tiled_cfg<CfgD>(g, D, D_next, t_next, dt, fused, in, out, s);
}

size_t tiled2d_smem_bytes_cfgd(int nfields) { return tile_smem_bytes<CfgD>(nfields); }
