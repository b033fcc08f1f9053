// k_score_128_8.cu - score kernel instantiated for 128-thread CTAs, registers capped for
// 8 CTAs per SM.
#include "k_score.cuh"

namespace b3d {
template int launch_score_nt<PoseList, 128, 8>(const SceneView &, const Lik &, PoseList, int64_t, float *, int,
                                                  cudaStream_t);
template int launch_score_nt<PoseGrid, 128, 8>(const SceneView &, const Lik &, PoseGrid, int64_t, float *, int,
                                                  cudaStream_t);
template int launch_score_multi_nt<128, 8>(const BatchItem *, int, const int64_t *, int64_t, int,
                                             unsigned long long *, int, int, int, cudaStream_t);
}  // namespace b3d
