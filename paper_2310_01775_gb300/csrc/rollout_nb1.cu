// Rollout kernels for scenes of 1 block(s): one instantiation per supported lane count.
#include "rollout.cuh"

namespace stamp {

cudaError_t launch_rollout_nb1(const SimConst& sc, const RolloutArgs& a, int lanes, bool adjoint,
                                 cudaStream_t st) {
    switch (lanes) {
        case 1: return rollout::launch<1, 1>(sc, a, adjoint, st);
        case 2: return rollout::launch<1, 2>(sc, a, adjoint, st);
        case 4: return rollout::launch<1, 4>(sc, a, adjoint, st);
    }
    return cudaErrorInvalidValue;
}

cudaError_t launch_rollout_batch_nb1(const SimConst& sc, const BatchArgs& b, int lanes, int cta,
                                        bool adjoint, cudaStream_t st) {
    switch (lanes) {
        case 1: return rollout::launch_batch<1, 1>(sc, b, cta, adjoint, st);
        case 2: return rollout::launch_batch<1, 2>(sc, b, cta, adjoint, st);
        case 4: return rollout::launch_batch<1, 4>(sc, b, cta, adjoint, st);
    }
    return cudaErrorInvalidValue;
}

cudaError_t launch_replay_nb1(const SimConst& sc, const RolloutArgs& a, int lanes, float* full,
                                cudaStream_t st) {
    switch (lanes) {
        case 1: return rollout::launch_replay<1, 1>(sc, a, full, st);
        case 2: return rollout::launch_replay<1, 2>(sc, a, full, st);
        case 4: return rollout::launch_replay<1, 4>(sc, a, full, st);
    }
    return cudaErrorInvalidValue;
}

}  // namespace stamp
