// FP32 row / entropy-epilogue kernels for the transform sizes 96, 192, 384, 768 (3 * 2^k).
#include "pipeline_impl.cuh"
namespace cmif {
template cudaError_t Sized<float, 96>::pair_rows(const Geom&, const PipeArgs<float>&, cudaStream_t);
template size_t Sized<float, 96>::rows_smem(int, bool);
template int Sized<float, 96>::rows_threads();
template cudaError_t Sized<float, 96>::rows_max_blocks(int, bool, int*);
template cudaError_t Sized<float, 192>::pair_rows(const Geom&, const PipeArgs<float>&, cudaStream_t);
template size_t Sized<float, 192>::rows_smem(int, bool);
template int Sized<float, 192>::rows_threads();
template cudaError_t Sized<float, 192>::rows_max_blocks(int, bool, int*);
template cudaError_t Sized<float, 384>::pair_rows(const Geom&, const PipeArgs<float>&, cudaStream_t);
template size_t Sized<float, 384>::rows_smem(int, bool);
template int Sized<float, 384>::rows_threads();
template cudaError_t Sized<float, 384>::rows_max_blocks(int, bool, int*);
template cudaError_t Sized<float, 768>::pair_rows(const Geom&, const PipeArgs<float>&, cudaStream_t);
template size_t Sized<float, 768>::rows_smem(int, bool);
template int Sized<float, 768>::rows_threads();
template cudaError_t Sized<float, 768>::rows_max_blocks(int, bool, int*);
}
