// Rollout kernels for scenes of 3 block(s): one instantiation per supported lane count.
#include "rollout.cuh"

namespace stamp {

cudaError_t launch_rollout_nb3(const SimConst& sc, const RolloutArgs& a, int lanes, bool adjoint,
                                 cudaStream_t st) {
    switch (lanes) {
        case 8: return rollout::launch<3, 8>(sc, a, adjoint, st);
        case 16: return rollout::launch<3, 16>(sc, a, adjoint, st);
        case 32: return rollout::launch<3, 32>(sc, a, adjoint, st);
    }
    return cudaErrorInvalidValue;
}

cudaError_t launch_rollout_batch_nb3(const SimConst& sc, const BatchArgs& b, int lanes, int cta,
                                        bool adjoint, cudaStream_t st) {
    switch (lanes) {
        case 8: return rollout::launch_batch<3, 8>(sc, b, cta, adjoint, st);
        case 16: return rollout::launch_batch<3, 16>(sc, b, cta, adjoint, st);
        case 32: return rollout::launch_batch<3, 32>(sc, b, cta, adjoint, st);
    }
    return cudaErrorInvalidValue;
}

cudaError_t launch_replay_nb3(const SimConst& sc, const RolloutArgs& a, int lanes, float* full,
                                cudaStream_t st) {
    switch (lanes) {
        case 2: return rollout::launch_replay<3, 2>(sc, a, full, st);
        case 4: return rollout::launch_replay<3, 4>(sc, a, full, st);
        case 8: return rollout::launch_replay<3, 8>(sc, a, full, st);
        case 16: return rollout::launch_replay<3, 16>(sc, a, full, st);
        case 32: return rollout::launch_replay<3, 32>(sc, a, full, st);
    }
    return cudaErrorInvalidValue;
}

}  // namespace stamp
