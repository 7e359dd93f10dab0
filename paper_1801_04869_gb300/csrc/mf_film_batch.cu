// Several thin films advanced in one persistent cooperative launch: the grid is cut into
// consecutive CTA ranges, one per film, and each range runs the same device code as a
// one-film launch (mf_film.cuh) with the film's own descriptor, grid barrier, items and
// partial sums.  Films never wait on each other.
#include "mf_film.cuh"

namespace mf {

// several films in one launch, each advanced (MODE_ADVANCE) by its own range of CTAs
template <typename T>
__global__ void __launch_bounds__(NT, 2) film_batch_kernel(const __grid_constant__ BatchTable tab) {
  __shared__ int s_job;
  if (threadIdx.x == 0) {
    // the job whose range [b0, b0 + nb) holds this CTA (ranges ascend and tile the grid)
    int lo = 0, hi = tab.n - 1;
    const int b = (int)blockIdx.x;
    while (lo < hi) {
      const int mid = (lo + hi + 1) >> 1;
      if (tab.job[mid].b0 <= b) lo = mid;
      else hi = mid - 1;
    }
    s_job = lo;
  }
  __syncthreads();
  const BatchJob& j = tab.job[s_job];
  KernelArgs a{};
  a.mode = MODE_ADVANCE;
  a.t_target = j.t_target;
  a.max_attempts = j.max_attempts;
  film_main<T>(*j.desc, a, (int)blockIdx.x - j.b0, (unsigned)j.nb);
}

int film_batch_max_blocks(int precision, size_t smem) {
  int nb = 0;
  if (precision) {
    cudaFuncSetAttribute(film_batch_kernel<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, film_batch_kernel<float>, NT, smem);
  } else {
    cudaFuncSetAttribute(film_batch_kernel<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, film_batch_kernel<double>, NT, smem);
  }
  return nb;
}

cudaError_t film_batch_launch(int precision, const BatchTable& tab, int grid, cudaStream_t s) {
  BatchTable t = tab;
  void* args[] = {&t};
  const size_t smem = film_smem_bytes(precision);
  const void* fn = precision ? (const void*)film_batch_kernel<float> : (const void*)film_batch_kernel<double>;
  return cudaLaunchCooperativeKernel(fn, dim3(grid), dim3(NT), args, smem, s);
}

}  // namespace mf
