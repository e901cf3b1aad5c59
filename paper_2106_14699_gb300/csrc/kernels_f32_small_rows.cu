// FP32 row / entropy-epilogue kernels for transform sizes 16, 32, 64, 128, 256.
#include "pipeline_impl.cuh"
namespace cmif {
template cudaError_t Sized<float, 16>::pair_rows(const Geom&, const PipeArgs<float>&, cudaStream_t);
template size_t Sized<float, 16>::rows_smem(int, bool);
template int Sized<float, 16>::rows_threads();
template cudaError_t Sized<float, 16>::rows_max_blocks(int, bool, int*);
template cudaError_t Sized<float, 32>::pair_rows(const Geom&, const PipeArgs<float>&, cudaStream_t);
template size_t Sized<float, 32>::rows_smem(int, bool);
template int Sized<float, 32>::rows_threads();
template cudaError_t Sized<float, 32>::rows_max_blocks(int, bool, int*);
template cudaError_t Sized<float, 64>::pair_rows(const Geom&, const PipeArgs<float>&, cudaStream_t);
template size_t Sized<float, 64>::rows_smem(int, bool);
template int Sized<float, 64>::rows_threads();
template cudaError_t Sized<float, 64>::rows_max_blocks(int, bool, int*);
template cudaError_t Sized<float, 128>::pair_rows(const Geom&, const PipeArgs<float>&, cudaStream_t);
template size_t Sized<float, 128>::rows_smem(int, bool);
template int Sized<float, 128>::rows_threads();
template cudaError_t Sized<float, 128>::rows_max_blocks(int, bool, int*);
template cudaError_t Sized<float, 256>::pair_rows(const Geom&, const PipeArgs<float>&, cudaStream_t);
template size_t Sized<float, 256>::rows_smem(int, bool);
template int Sized<float, 256>::rows_threads();
template cudaError_t Sized<float, 256>::rows_max_blocks(int, bool, int*);
}
