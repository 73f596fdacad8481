// The two loop skeletons of Sec. 2 over vector chunks, shared by the vector
// kernels (k_vec.cu, k_vec_ext.cu).
#pragma once

#include "lak_internal.cuh"

namespace lak {

// Chunk range of this thread under the two skeletons.
struct Range {
    int64_t begin, end, stride;
};

__device__ __forceinline__ Range chunk_range(int64_t nchunks, int inc) {
    Range r;
    if (inc == LAK_INC_GLOBAL) {
        r.begin = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
        r.end = nchunks;
        r.stride = (int64_t)gridDim.x * blockDim.x;
    } else {
        // block b owns chunks [b*per, (b+1)*per); per is a multiple of the block
        // size so that every block starts on a whole-block boundary
        int64_t per = (nchunks + gridDim.x - 1) / gridDim.x;
        per = (per + blockDim.x - 1) / blockDim.x * blockDim.x;
        int64_t b0 = (int64_t)blockIdx.x * per;
        r.begin = b0 + threadIdx.x;
        r.end = b0 + per < nchunks ? b0 + per : nchunks;
        r.stride = blockDim.x;
    }
    return r;
}

// Index of the t-th element outside the vectorised body (prologue, then tail).
__device__ __forceinline__ int64_t extra_index(int64_t t, int64_t head, int64_t body_end) {
    return t < head ? t : body_end + (t - head);
}

}  // namespace lak
