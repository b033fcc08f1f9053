// k_score_32_24.cu - score kernel instantiated for 32-thread CTAs, registers capped for
// 24 CTAs per SM.
#include "k_score.cuh"

namespace b3d {
template int launch_score_nt<PoseList, 32, 24>(const SceneView &, const Lik &, PoseList, int64_t, float *, int,
                                                  cudaStream_t);
template int launch_score_nt<PoseGrid, 32, 24>(const SceneView &, const Lik &, PoseGrid, int64_t, float *, int,
                                                  cudaStream_t);
template int launch_score_multi_nt<32, 24>(const BatchItem *, int, const int64_t *, int64_t, int,
                                             unsigned long long *, int, int, int, cudaStream_t);
}  // namespace b3d
