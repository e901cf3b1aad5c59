// FP32 row / entropy-epilogue kernels for the transform sizes 1536, 3072 (3 * 2^k).
#include "pipeline_impl.cuh"
namespace cmif {
template cudaError_t Sized<float, 1536>::pair_rows(const Geom&, const PipeArgs<float>&, cudaStream_t);
template size_t Sized<float, 1536>::rows_smem(int, bool);
template int Sized<float, 1536>::rows_threads();
template cudaError_t Sized<float, 1536>::rows_max_blocks(int, bool, int*);
template cudaError_t Sized<float, 3072>::pair_rows(const Geom&, const PipeArgs<float>&, cudaStream_t);
template size_t Sized<float, 3072>::rows_smem(int, bool);
template int Sized<float, 3072>::rows_threads();
template cudaError_t Sized<float, 3072>::rows_max_blocks(int, bool, int*);
}
