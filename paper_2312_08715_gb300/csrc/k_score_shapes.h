// k_score_shapes.h - launch shapes of the score kernel, each instantiated in its own
// translation unit (k_score_<threads>_<ctas>.cu) so the library compiles in parallel.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "b3d_internal.h"

namespace b3d {

template <class PS, int NT, int MINB>
int launch_score_nt(const SceneView &sv, const Lik &L, PS P, int64_t n, float *ll, int grid, cudaStream_t s);
template <int NT, int MINB>
int launch_score_multi_nt(const BatchItem *items, int n_items, const int64_t *item_begin, int64_t total, int chunk,
                          unsigned long long *counter, int w, int max_lat, int grid, cudaStream_t s);

#define B3D_SCORE_SHAPE(NT, MINB)                                                                           \
    extern template int launch_score_nt<PoseList, NT, MINB>(const SceneView &, const Lik &, PoseList, int64_t, \
                                                            float *, int, cudaStream_t);                     \
    extern template int launch_score_nt<PoseGrid, NT, MINB>(const SceneView &, const Lik &, PoseGrid, int64_t, \
                                                            float *, int, cudaStream_t);                     \
    extern template int launch_score_multi_nt<NT, MINB>(const BatchItem *, int, const int64_t *, int64_t, int,    \
                                                        unsigned long long *, int, int, int, cudaStream_t);
B3D_SCORE_SHAPE(256, 3)
B3D_SCORE_SHAPE(128, 6)
B3D_SCORE_SHAPE(64, 10)
B3D_SCORE_SHAPE(32, 16)
B3D_SCORE_SHAPE(256, 4)
B3D_SCORE_SHAPE(128, 8)
B3D_SCORE_SHAPE(64, 14)
B3D_SCORE_SHAPE(32, 24)
#undef B3D_SCORE_SHAPE

}  // namespace b3d
