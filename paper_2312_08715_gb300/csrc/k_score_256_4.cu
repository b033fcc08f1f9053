// k_score_256_4.cu - score kernel instantiated for 256-thread CTAs, registers capped for
// 4 CTAs per SM.
// The 256-thread shapes serve the larger images (320x240 and up), whose rectangles span
// several pixels in x: candidate blocks of 4 pixels share each owner lookup and record
// load among more pixel tests (320x240 tabletop parse: 7.65 -> 7.40 ms per launch, the
// same scores bit for bit). The 128-thread shapes, picked for 160x120, keep pixel pairs:
// there 4-pixel blocks cost 5%, since most rectangles are one or two pixels wide.
#define B3D_CAND_X 4
#include "k_score.cuh"

namespace b3d {
template int launch_score_nt<PoseList, 256, 4>(const SceneView &, const Lik &, PoseList, int64_t, float *, int,
                                                  cudaStream_t);
template int launch_score_nt<PoseGrid, 256, 4>(const SceneView &, const Lik &, PoseGrid, int64_t, float *, int,
                                                  cudaStream_t);
template int launch_score_multi_nt<256, 4>(const BatchItem *, int, const int64_t *, int64_t, int,
                                             unsigned long long *, int, int, int, cudaStream_t);
}  // namespace b3d
