// mlmc_reduce.cuh -- the warp stage of the fixed-order block reductions.
//
// Twelve FP64 sums over the 32 lanes of a warp, each by the binary tree that
// v[lane] += v[lane + h] for h = 16, 8, 4, 2, 1 leaves in lane 0.  A shuffle
// form of that tree issues 12 FP64 additions per level whatever the number
// of lanes that need one; FP64 instructions are slow to issue on this GPU,
// so here each level's additions are spread over the lanes: the first level
// from registers (lanes 0..15 form sums 0..5, lanes 16..31 sums 6..11, one
// exchange with the partner lane 16 away per sum), the others through shared
// memory -- 6 + 3 + 2 + 1 + 1 additions per lane at most.  Every addition has
// the tree's operands, so the sums are bit for bit those of the shuffle form.
#pragma once

namespace mlmc {

// buf: this warp's [12][16] doubles of shared memory.  The sums end in
// buf[k][0]; the warp is synchronised on return.
__device__ __forceinline__ void warp_tree12(const double v[12], double (*buf)[16], int lane) {
  const bool lo = lane < 16;
  const int i0 = lane & 15;
#pragma unroll
  for (int m = 0; m < 6; ++m) {
    // lane i0 < 16 forms sum m, lane i0 + 16 sum 6 + m, both v_i0 + v_(i0+16)
    const double got = __shfl_xor_sync(0xFFFFFFFFu, lo ? v[6 + m] : v[m], 16);
    if (lo) buf[m][i0] = v[m] + got;
    else buf[6 + m][i0] = got + v[6 + m];
  }
  __syncwarp();
#pragma unroll
  for (int h = 8; h >= 1; h >>= 1) {
#pragma unroll
    for (int j0 = 0; j0 < 12 * h; j0 += 32) {
      const int j = j0 + lane;
      if (j < 12 * h) {
        const int k = j / h, i = j - k * h;
        buf[k][i] = buf[k][i] + buf[k][i + h];
      }
    }
    __syncwarp();
  }
}

}  // namespace mlmc
