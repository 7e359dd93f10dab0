// Thin-film (2D) persistent kernel for one film on the whole grid, and its launch helpers.
// The method and the device code it runs are in mf_film.cuh.
#include "mf_film.cuh"

namespace mf {

// one film on the whole grid
template <typename T>
__global__ void __launch_bounds__(NT, 2) film_kernel(const Desc* __restrict__ dg, KernelArgs a) {
  film_main<T>(*dg, a, (int)blockIdx.x, gridDim.x);
}

// film passes: two FFT buffers; bulk passes: a third one for the next item's gather
size_t kernel_smem_bytes(const Desc& d) {
  return film_smem_bytes(d.precision) / 2 * (d.dim == 3 ? 3 : 2);
}

int film_max_blocks(int precision, size_t smem) {
  int nb = 0;
  if (precision) {
    cudaFuncSetAttribute(film_kernel<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, film_kernel<float>, NT, smem);
  } else {
    cudaFuncSetAttribute(film_kernel<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, film_kernel<double>, NT, smem);
  }
  return nb;
}

cudaError_t film_launch(int precision, const Desc& d, const KernelArgs& a, cudaStream_t s) {
  const Desc* dg = d.dev;
  KernelArgs aa = a;
  void* args[] = {&dg, &aa};
  const size_t smem = kernel_smem_bytes(d);
  const void* fn = precision ? (const void*)film_kernel<float> : (const void*)film_kernel<double>;
  return cudaLaunchCooperativeKernel(fn, dim3(d.grid), dim3(NT), args, smem, s);
}

}  // namespace mf
