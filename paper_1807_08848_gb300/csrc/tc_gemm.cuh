// Tensor-core GEMM of the serving map (see tc_gemm.cu): operands pre-tiled and
// split into TF32 high and FP32 low parts.
#pragma once

#include <cuda_runtime.h>

#include "../../include/msp.h"

namespace msp {

struct TcMapArgs {
    const float* a_hi;   // G tiled: [row tile][slab] blocks of 128 x 32
    const float* a_lo;
    const float* b_hi;   // phi tiled: [data-set tile][slab] blocks of 32 x 32
    const float* b_lo;
    int M;               // rows of G (unknowns)
    int B;               // data sets
    int n_slabs;         // K slabs of 32
    float* c;            // c[j][b], element-major
    int* err;            // set on a timed-out wait
};

int tc_slabs(int K);
int tc_row_tiles(int M);
int tc_n_tiles(int B);
long long tc_a_floats(int M, int K);
long long tc_b_floats(int B, int K);
// X element (r, k) at X[r * ld_r + k * ld_k]; a_operand: 128-row tiles, else 32-row tiles
void tc_tile_split(const float* X, long long ld_r, long long ld_k, int rows, int K, bool a_operand, float* hi,
                   float* lo, cudaStream_t s);
msp_status tc_map_gemm(const TcMapArgs& args, cudaStream_t s);

}  // namespace msp
