// sl_internal.h -- host-side grid object and kernel launchers of libsl.so.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "sl_device.cuh"

struct sl_grid {
    sl_grid_desc desc;          // copy of the descriptor (velocity_params points at vel_params)
    double vel_params[SL_MAX_VEL_PARAMS];
    int dim, nfields, dtype, ds; // ds: values per node in a displacement buffer (2 in 2-D, 4 in 3-D)
    int64_t n[3], N;
    double dx[3];
    size_t tsize;                // bytes per scalar
    // carved from the caller's workspace
    char *ws;
    size_t ws_bytes;
    DevCounters *counters;
    DevCounters *stripes;
    // sin(pi x), cos(pi x) at the node coordinates of each axis (pairs; axis a at trig_off[a] in
    // units of the dtype), for the trajectory launch of the swirl and the deformation flow
    void *trig;
    int64_t trig_off[3];        // SL_COUNTER_STRIPES more copies, one per SM (kernels with many small
                                 // CTAs add into their SM's copy); read together with counters
    double *partials;            // moments: SL_MOMENT_BLOCKS x 8
    double *moment_out;          // 8 doubles
    uint8_t *flags;              // N
    uint8_t *flags2;             // N (second byte buffer: separable OR of flags over stencils)
    void *D[2];                  // two displacement buffers (ping-pong for the pipelined step)
    int dcur;                    // index of the current displacement
    int device, num_sms;
    unsigned long long launches;  // kernels launched by this grid's calls (host-side count)
    // A steady velocity moves every node by the same displacement each step: D(dt) is integrated
    // once and reused while d_cached says D[dcur] holds it for step d_cached_dt.
    int steady;
    int d_cached;
    double d_cached_dt;
    // The fused FP32 path integrates, inside a call's last remap, the displacement of the step
    // that follows the call: next_valid says D[dcur] holds it for the velocity arguments next_vel,
    // so a call that starts there skips its own integration.
    int next_valid;
    VelArgs<float> next_vel;
    // A carried velocity (SL_VEL_CARRIED) lives in field planes vel_field[a] of the fields.
    int carried;
    int vel_field[3];
    // Shallow water (SL_VEL_NLSW): two sets of RK3 registers of h, u1, u2 and of the displacement,
    // and the viscous stress (thirteen planes in the workspace).
    int nlsw;
    void *rk;
};

#define SL_MOMENT_BLOCKS 512
#define SL_COUNTER_STRIPES 256

// precision-dispatched launchers (sl_kernels.cu)
template <typename T>
struct Launch {
    static cudaError_t advect(const sl_grid *g, void *D, double t, double dt, cudaStream_t s);
    static cudaError_t advect_carried(const sl_grid *g, const void *const *fields, void *D, double dt, cudaStream_t s);
    // shallow water (sl_nlsw.cu): the three RK3 stages of one step on the nodes -- node values
    // from `fields` into `nodes` (`fields` is overwritten), displacement (cells) into D, Dalt as
    // scratch; nlsw_kernels_per_step launches
    static cudaError_t nlsw_stages(const sl_grid *g, const void *const *fields, void *const *nodes, void *D, void *Dalt,
                                   double dt, cudaStream_t s);
    static cudaError_t flags(const sl_grid *g, const void *const *in, uint8_t *flags, cudaStream_t s);
    static cudaError_t remap_generic(const sl_grid *g, const void *D, const uint8_t *flags, const void *const *in,
                                     void *const *out, const sl_remap_debug *dbg, cudaStream_t s);
    static cudaError_t moments(const sl_grid *g, const void *field, int pmax, cudaStream_t s);
    static cudaError_t copy_planes(const sl_grid *g, const void *const *src, void *const *dst, cudaStream_t s);
    static cudaError_t copy_disp(const sl_grid *g, const void *src, int64_t src_stride, void *dst,
                                 int64_t dst_stride, cudaStream_t s);
    // tiled / fused kernels (sl_tiled.cu)
    static bool tiled_supported(const sl_grid *g);
    static cudaError_t remap_tiled(const sl_grid *g, const void *D, const void *const *in, void *const *out,
                                   cudaStream_t s);
    static cudaError_t step_fused(const sl_grid *g, const void *D, void *D_next, double t_next, double dt,
                                  const void *const *in, void *const *out, cudaStream_t s);
};

// 3-D FP32 kernels (sl_blocked3d.cu): box flags end up in `tmp`; launch_blocked3d runs a plain
// remap on the staged kernel where it applies, a fused step (and the rest) on the blocked one
cudaError_t launch_trig_tables(const sl_grid *g, cudaStream_t s);
cudaError_t launch_box_flags3d(const sl_grid *g, const void *const *in, uint8_t *flags, uint8_t *tmp, cudaStream_t s);
cudaError_t launch_blocked3d(const sl_grid *g, const void *D, void *D_next, const uint8_t *box, double t_next,
                             double dt, bool fused, const void *const *in, void *const *out, cudaStream_t s);
// kernels one tiled remap / fused step call launches
int tiled_kernels_per_call(const sl_grid *g);
// 2-D FP32 tiled kernels per tile configuration (sl_tiled_cfg_*.cu): a 32x32, b 32x16, c 64x16,
// d 32x16 at 4 CTAs per SM
cudaError_t launch_tiled2d_cfga(const sl_grid *g, const void *D, void *D_next, double t_next, double dt, bool fused,
                                const void *const *in, void *const *out, cudaStream_t s);
cudaError_t launch_tiled2d_cfgb(const sl_grid *g, const void *D, void *D_next, double t_next, double dt, bool fused,
                                const void *const *in, void *const *out, cudaStream_t s);
cudaError_t launch_tiled2d_cfgc(const sl_grid *g, const void *D, void *D_next, double t_next, double dt, bool fused,
                                const void *const *in, void *const *out, cudaStream_t s);
cudaError_t launch_tiled2d_cfgp(const sl_grid *g, const void *D, void *D_next, double t_next, double dt, bool fused,
                                const void *const *in, void *const *out, cudaStream_t s);
size_t tiled2d_smem_bytes_cfga(int nfields);
size_t tiled2d_smem_bytes_cfgp(int nfields);
size_t tiled2d_smem_bytes_cfgb(int nfields);
size_t tiled2d_smem_bytes_cfgc(int nfields);
cudaError_t launch_tiled2d_cfgd(const sl_grid *g, const void *D, void *D_next, double t_next, double dt, bool fused,
                                const void *const *in, void *const *out, cudaStream_t s);
size_t tiled2d_smem_bytes_cfgd(int nfields);
// shallow water (sl_nlsw.cu): the viscosity nu of a grid and the launches of one step's stages
double nlsw_viscosity(const sl_grid *g);
int nlsw_kernels_per_step(const sl_grid *g);
// 2-D FP32 persistent remap with TMA-staged windows (sl_remap2d.cu): configuration 6 (64x32 tiles,
// one CTA per SM) or 7 (32x32 tiles, two CTAs per SM)
bool remap2d_tma_supported(const sl_grid *g, const void *const *in, void *const *out);
cudaError_t launch_remap2d_tma(const sl_grid *g, int config, const void *D, void *D_next, double t_next, double dt,
                               bool fused, const void *const *in, void *const *out, cudaStream_t s);
// 2-D FP32 tiled kernels of the quintic Z-spline (max_order 2; sl_tiled_z2.cu)
cudaError_t launch_tiled2d_z2(const sl_grid *g, const void *D, void *D_next, double t_next, double dt, bool fused,
                              const void *const *in, void *const *out, cudaStream_t s);
size_t tiled2d_smem_bytes_z2(int nfields);

// the text sl_last_error() returns for this thread's last failed call (sl_api.cu)
void sl_record_error(const char *what, const char *why);

// shared argument builders (sl_kernels.cu)
template <typename T>
GridArgs<T> make_grid_args(const sl_grid *g);
template <typename T>
VelArgs<T> make_vel_args(const sl_grid *g, double t, double dt);
int grid_stride_blocks(const sl_grid *g, long long work, int threads);
