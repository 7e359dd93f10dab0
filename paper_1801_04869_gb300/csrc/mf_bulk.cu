// Bulk (3D) kernel: placeholder until the 3D passes land.
#include "mf_common.cuh"
namespace mf {
int bulk_max_blocks(int, size_t) { return 0; }
cudaError_t bulk_launch(int, const Desc&, const KernelArgs&, cudaStream_t) { return cudaErrorNotSupported; }
}  // namespace mf
