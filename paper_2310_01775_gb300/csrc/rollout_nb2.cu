// Rollout kernels for scenes of 2 block(s): one instantiation per supported lane count.
#include "rollout.cuh"

namespace stamp {

cudaError_t launch_rollout_nb2(const SimConst& sc, const RolloutArgs& a, int lanes, bool adjoint,
                                 cudaStream_t st) {
    switch (lanes) {
        case 2: return rollout::launch<2, 2>(sc, a, adjoint, st);
        case 4: return rollout::launch<2, 4>(sc, a, adjoint, st);
        case 8: return rollout::launch<2, 8>(sc, a, adjoint, st);
        case 16: return rollout::launch<2, 16>(sc, a, adjoint, st);
    }
    return cudaErrorInvalidValue;
}

cudaError_t launch_rollout_batch_nb2(const SimConst& sc, const BatchArgs& b, int lanes, int cta,
                                        bool adjoint, cudaStream_t st) {
    switch (lanes) {
        case 2: return rollout::launch_batch<2, 2>(sc, b, cta, adjoint, st);
        case 4: return rollout::launch_batch<2, 4>(sc, b, cta, adjoint, st);
        case 8: return rollout::launch_batch<2, 8>(sc, b, cta, adjoint, st);
        case 16: return rollout::launch_batch<2, 16>(sc, b, cta, adjoint, st);
    }
    return cudaErrorInvalidValue;
}

cudaError_t launch_replay_nb2(const SimConst& sc, const RolloutArgs& a, int lanes, float* full,
                                cudaStream_t st) {
    switch (lanes) {
        case 2: return rollout::launch_replay<2, 2>(sc, a, full, st);
        case 4: return rollout::launch_replay<2, 4>(sc, a, full, st);
        case 8: return rollout::launch_replay<2, 8>(sc, a, full, st);
        case 16: return rollout::launch_replay<2, 16>(sc, a, full, st);
    }
    return cudaErrorInvalidValue;
}

}  // namespace stamp
