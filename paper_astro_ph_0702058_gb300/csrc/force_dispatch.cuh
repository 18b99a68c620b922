// Launch and dispatch of the force kernels over the compiled launch shapes.
// The plain, compensated and summation-check modes run the packed-FP32 pair
// loop (force_x2.cuh); building with -DNB_PACKED=0 selects the scalar loop of
// force_impl.cuh instead.
#pragma once

#include "force_impl.cuh"
#include "force_slice.cuh"
#include "force_x2.cuh"

namespace nb {

// The packed kernel reads the SoA j-stream when the caller has one (library
// contexts); a float4-only stream (no-alloc callers) goes through the packed
// kernel's transposing variant for the automatic shapes and the scalar kernel
// otherwise.
template <int NT, int IPT>
constexpr bool aos_packed_shape()
{
    return IPT == 1 && (NT == 64 || NT == 256);
}

// The j-subgroup instance (plain and compensated modes, SoA j-stream).
template <int MODE>
cudaError_t launch_force_jsub(const ForceParams &P, const ForceConfig &cfg, cudaStream_t s)
{
    if constexpr (NB_PACKED && (MODE == kModePlain || MODE == kModeComp)) {
        if (P.soa) {
            force_kernel_x2<MODE, kJSubThreads, 1, FoldLen<MODE>::value, true, kJSub>
                <<<dim3(cfg.n_iblk, cfg.split), kJSubThreads, 0, s>>>(P);
            return cudaGetLastError();
        }
    }
    return cudaErrorInvalidConfiguration;
}

template <int MODE>
int occupancy_jsub()
{
    int b = 0;
    if constexpr (NB_PACKED && (MODE == kModePlain || MODE == kModeComp))
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(
            &b, force_kernel_x2<MODE, kJSubThreads, 1, FoldLen<MODE>::value, true, kJSub>, kJSubThreads, 0);
    return b;
}

template <int MODE, int NT, int IPT>
cudaError_t launch_force_instance(const ForceParams &P, const ForceConfig &cfg, cudaStream_t s)
{
    dim3 grid(cfg.n_iblk, cfg.split);
    constexpr int PF = FoldLen<MODE>::value;
    if constexpr (NB_PACKED) {
        if (P.soa) {
            force_kernel_x2<MODE, NT, IPT, PF, true><<<grid, NT, 0, s>>>(P);
            return cudaGetLastError();
        }
        if constexpr (aos_packed_shape<NT, IPT>()) {
            force_kernel_x2<MODE, NT, IPT, PF, false><<<grid, NT, 0, s>>>(P);
            return cudaGetLastError();
        }
    }
    force_kernel<MODE, NT, IPT, PF><<<grid, NT, 0, s>>>(P);
    return cudaGetLastError();
}

template <int MODE, int NT, int IPT>
int occupancy_instance(int *blocks)
{
    if constexpr (NB_PACKED)
        return cudaOccupancyMaxActiveBlocksPerMultiprocessor(
            blocks, force_kernel_x2<MODE, NT, IPT, FoldLen<MODE>::value, true>, NT, 0);
    else
        return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks, force_kernel<MODE, NT, IPT, FoldLen<MODE>::value>,
                                                         NT, 0);
}

// Dispatch over the compiled shapes of one mode.
template <int MODE>
cudaError_t force_dispatch(const ForceParams &P, const ForceConfig &cfg, cudaStream_t s)
{
    if (cfg.slice) return launch_force_slice<MODE>(P, cfg, s);
    if (cfg.jsub > 1) return launch_force_jsub<MODE>(P, cfg, s);
#define NB_CASE(T, I) \
    if (cfg.threads == T && cfg.ipt == I) return launch_force_instance<MODE, T, I>(P, cfg, s);
    NB_CASE(64, 1)
    NB_CASE(64, 2)
    NB_CASE(64, 4)
    NB_CASE(128, 1)
    NB_CASE(128, 2)
    NB_CASE(128, 4)
    NB_CASE(256, 1)
    NB_CASE(256, 2)
    NB_CASE(256, 4)
    NB_CASE(512, 1)
#undef NB_CASE
    return cudaErrorInvalidConfiguration;
}

template <int MODE>
int force_occupancy(int threads, int ipt)
{
    if (ipt < 0) return occupancy_jsub<MODE>();  // ipt < 0 asks for the j-subgroup shape
    int b = 0;
#define NB_CASE(T, I) \
    if (threads == T && ipt == I) { occupancy_instance<MODE, T, I>(&b); return b; }
    NB_CASE(64, 1)
    NB_CASE(64, 2)
    NB_CASE(64, 4)
    NB_CASE(128, 1)
    NB_CASE(128, 2)
    NB_CASE(128, 4)
    NB_CASE(256, 1)
    NB_CASE(256, 2)
    NB_CASE(256, 4)
    NB_CASE(512, 1)
#undef NB_CASE
    return 0;
}

// n_act sizes the launch; with n_act_dev the kernels read the actual (smaller
// or equal) block size on the device.
template <int MODE>
cudaError_t reduce_launch(const float *part, int split, int n_act, double *acc, double *jerk,
                          double *pot, cudaStream_t s, const long long *n_act_dev = nullptr)
{
    const int nt = 256;
    if (split >= 8)
        reduce_partials_2d_kernel<MODE, 8><<<dim3(static_cast<unsigned>((n_act + 7) / 8), 7), nt, 0, s>>>(
            part, split, n_act, acc, jerk, pot, n_act_dev);
    else
        reduce_partials_kernel<MODE><<<static_cast<unsigned>((7LL * n_act + nt - 1) / nt), nt, 0, s>>>(
            part, split, n_act, acc, jerk, pot, n_act_dev);
    return cudaGetLastError();
}

}  // namespace nb
