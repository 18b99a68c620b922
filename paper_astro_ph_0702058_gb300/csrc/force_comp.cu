// Instantiates the force kernels of the comp mode (see force_impl.cuh).
#include "force_dispatch.cuh"

namespace nb {

cudaError_t force_dispatch_comp(const ForceParams &P, const ForceConfig &cfg, cudaStream_t s)
{
    return force_dispatch<kModeComp>(P, cfg, s);
}

int force_occupancy_comp(int threads, int ipt) { return force_occupancy<kModeComp>(threads, ipt); }

cudaError_t reduce_comp(const float *part, int split, int n_act, double *acc, double *jerk, double *pot,
                         cudaStream_t s, const long long *n_act_dev)
{
    return reduce_launch<kModeComp>(part, split, n_act, acc, jerk, pot, s, n_act_dev);
}

}  // namespace nb
