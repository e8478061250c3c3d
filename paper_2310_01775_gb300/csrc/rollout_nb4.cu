// Rollout kernels for scenes of 4 block(s): one instantiation per supported lane count.
#include "rollout.cuh"

namespace stamp {

cudaError_t launch_rollout_nb4(const SimConst& sc, const RolloutArgs& a, int lanes, bool adjoint,
                                 cudaStream_t st) {
    switch (lanes) {
        case 8: return rollout::launch<4, 8>(sc, a, adjoint, st);
        case 16: return rollout::launch<4, 16>(sc, a, adjoint, st);
        case 32: return rollout::launch<4, 32>(sc, a, adjoint, st);
    }
    return cudaErrorInvalidValue;
}

cudaError_t launch_rollout_batch_nb4(const SimConst& sc, const BatchArgs& b, int lanes, int cta,
                                        bool adjoint, cudaStream_t st) {
    switch (lanes) {
        case 8: return rollout::launch_batch<4, 8>(sc, b, cta, adjoint, st);
        case 16: return rollout::launch_batch<4, 16>(sc, b, cta, adjoint, st);
        case 32: return rollout::launch_batch<4, 32>(sc, b, cta, adjoint, st);
    }
    return cudaErrorInvalidValue;
}

cudaError_t launch_replay_nb4(const SimConst& sc, const RolloutArgs& a, int lanes, float* full,
                                cudaStream_t st) {
    switch (lanes) {
        case 4: return rollout::launch_replay<4, 4>(sc, a, full, st);
        case 8: return rollout::launch_replay<4, 8>(sc, a, full, st);
        case 16: return rollout::launch_replay<4, 16>(sc, a, full, st);
        case 32: return rollout::launch_replay<4, 32>(sc, a, full, st);
    }
    return cudaErrorInvalidValue;
}

}  // namespace stamp
