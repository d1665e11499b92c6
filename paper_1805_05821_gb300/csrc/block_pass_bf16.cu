// Block passes over V with BF16 storage (the kernel template is block_pass.cuh).
#include "block_pass.cuh"

namespace foa {
namespace blk {

cudaError_t launch_block_pass_bf16(int mode, int T, int fc, int P, const BlockArgs &a, int grid, cudaStream_t s) {
  return launch_block_pass<__nv_bfloat16>(mode, T, fc, P, a, grid, s);
}

}  // namespace blk
}  // namespace foa
