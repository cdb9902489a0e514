// sl_tiled_z2.cu -- the 2-D FP32 tiled kernels for the quintic Z-spline (one CTA per 32 x 32
// tile; the tile body is in sl_tile2d_z2.cuh).
#include "sl_tile2d_z2.cuh"

namespace {

template <int NF, bool FUSED>
__global__ void __launch_bounds__(CfgZ::NT, CfgZ::MINB)
    remap_tiled2d_z2_kernel(const __grid_constant__ TileArgs a, const VelArgs<float> vn)
{
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ int sBox[4];
    const TileSmemZ2<NF> sm(smem);
    LocalCounters cnt;
    cnt.clear();
    process_tile_z2<NF, FUSED>(a, vn, blockIdx.x * CfgZ::TX, blockIdx.y * CfgZ::TY, sm, sBox, cnt);
    flush_counters_sm(cnt, a);
}

template <int NF, bool FUSED>
cudaError_t launch_z2_nf(const sl_grid *g, const TileArgs &a, const VelArgs<float> &vn, cudaStream_t s)
{
    const size_t smem = z2_smem_bytes(NF);
    static bool configured[64] = {};
    cudaError_t e = allow_smem(remap_tiled2d_z2_kernel<NF, FUSED>, g->device, smem, configured);
    if (e != cudaSuccess) return e;
    dim3 grid((unsigned)((g->n[0] + CfgZ::TX - 1) / CfgZ::TX), (unsigned)((g->n[1] + CfgZ::TY - 1) / CfgZ::TY));
    remap_tiled2d_z2_kernel<NF, FUSED><<<grid, CfgZ::NT, smem, s>>>(a, vn);
    return cudaGetLastError();
}

template <bool FUSED>
cudaError_t launch_z2(const sl_grid *g, const TileArgs &a, const VelArgs<float> &vn, cudaStream_t s)
{
    switch (g->nfields) {
    case 1: return launch_z2_nf<1, FUSED>(g, a, vn, s);
    case 2: return launch_z2_nf<2, FUSED>(g, a, vn, s);
    case 3: return launch_z2_nf<3, FUSED>(g, a, vn, s);
    case 4: return launch_z2_nf<4, FUSED>(g, a, vn, s);
    case 5: return launch_z2_nf<5, FUSED>(g, a, vn, s);
    case 6: return launch_z2_nf<6, FUSED>(g, a, vn, s);
    case 7: return launch_z2_nf<7, FUSED>(g, a, vn, s);
    default: return launch_z2_nf<8, FUSED>(g, a, vn, s);
    }
}

}  // namespace

cudaError_t launch_tiled2d_z2(const sl_grid *g, const void *D, void *D_next, double t_next, double dt, bool fused,
                              const void *const *in, void *const *out, cudaStream_t s)
{
    TileArgs a = make_tile_args(g, D, D_next, in, out);
    VelArgs<float> vn;
    memset(&vn, 0, sizeof(vn));
    if (fused) {
        set_carried(g, dt, a);
        vn = make_vel_args<float>(g, t_next, dt);
        return launch_z2<true>(g, a, vn, s);
    }
    return launch_z2<false>(g, a, vn, s);
}

size_t tiled2d_smem_bytes_z2(int nfields) { return z2_smem_bytes(nfields); }
