// sl_tiled_cfg_p.cu -- the pipelined persistent 2-D FP32 kernels (tile configuration CfgP,
// at most 4 fields).
#include "sl_tile2d.cuh"

cudaError_t launch_tiled2d_cfgp(const sl_grid *g, const void *D, void *D_next, double t_next, double dt, bool fused,
                                const void *const *in, void *const *out, cudaStream_t s)
{
    return launch_pipe_cfg<CfgP>(g, D, D_next, t_next, dt, fused, in, out, s);
}

size_t tiled2d_smem_bytes_cfgp(int nfields) { return nfields <= 4 ? pipe_smem_bytes<CfgP>(nfields) : (size_t)-1; }
