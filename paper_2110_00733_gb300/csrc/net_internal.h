// net_internal.h -- kernel arguments and launchers of the warm-start network.
#pragma once
#include <cuda_bf16.h>
#include <cuda_runtime.h>

namespace hnet {

// One periodic 3x3x3 convolution.  Input channels are the concatenation
// [src0 (c0s channels, full resolution), src1 (c1s channels, half
// resolution, upsampled by nearest neighbour)]; c0s, c1s multiples of 16,
// c1s = 0 for a single source.  W: [27][cout][c0s + c1s] BF16.  Output
// [voxels][cout], BF16 (out_bf16) or FP32 (out_f32), cout a multiple of 16.
struct ConvArgs {
    int B, n1, n2, n3;
    const __nv_bfloat16 *src0;
    int c0s;
    const __nv_bfloat16 *src1;
    int c1s;
    const __nv_bfloat16 *W;
    const float *bias;      // [cout] or null
    int cout;
    int relu;
    __nv_bfloat16 *out_bf16;
    float *out_f32;
};

// Weight gradient of a convolution whose input is described by `in` (sources
// and grid only) and whose output gradient is G [voxels][cout] BF16:
// partial[s][t][cout][c0s + c1s] FP32 over S voxel splits.
struct WgradArgs {
    ConvArgs in;
    const __nv_bfloat16 *G;
    int cout;
    float *partial;
    int S;
};

int conv3_forward_tc(const ConvArgs &a, cudaStream_t st);   // tcgen05, cout <= 256
// nonzero if a tcgen05 convolution gave up a bounded wait (clears it if asked)
int conv3_tc_error(int clear);
int conv3_wgrad(const WgradArgs &a, cudaStream_t st);      // tcgen05 where bricks tile the grid, else mma.sync
int conv3_wgrad_tc(const WgradArgs &a, cudaStream_t st);   // -1 if the shape does not suit it

}  // namespace hnet
