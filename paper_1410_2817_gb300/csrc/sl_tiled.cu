// sl_tiled.cu -- shared-memory tiled kernels (filled in below).
#include "sl_internal.h"

template <typename T>
bool Launch<T>::tiled_supported(const sl_grid *)
{
    return false;
}

template <typename T>
cudaError_t Launch<T>::remap_tiled(const sl_grid *, const void *, const void *const *, void *const *, cudaStream_t)
{
    return cudaErrorNotSupported;
}

template <typename T>
cudaError_t Launch<T>::step_fused(const sl_grid *, const void *, void *, double, double, const void *const *,
                                  void *const *, cudaStream_t)
{
    return cudaErrorNotSupported;
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
