// FP64 row / entropy-epilogue kernels for transform sizes 16, 32, 64, 128, 256.
#include "pipeline_impl.cuh"
namespace cmif {
template cudaError_t Sized<double, 16>::pair_rows(const Geom&, const PipeArgs<double>&, cudaStream_t);
template cudaError_t Sized<double, 16>::pair_rows_counts(const Geom&, const PipeArgs<double>&, cudaStream_t);
template size_t Sized<double, 16>::rows_smem(int, bool);
template int Sized<double, 16>::rows_threads();
template cudaError_t Sized<double, 16>::rows_max_blocks(int, bool, int*);
template cudaError_t Sized<double, 32>::pair_rows(const Geom&, const PipeArgs<double>&, cudaStream_t);
template cudaError_t Sized<double, 32>::pair_rows_counts(const Geom&, const PipeArgs<double>&, cudaStream_t);
template size_t Sized<double, 32>::rows_smem(int, bool);
template int Sized<double, 32>::rows_threads();
template cudaError_t Sized<double, 32>::rows_max_blocks(int, bool, int*);
template cudaError_t Sized<double, 64>::pair_rows(const Geom&, const PipeArgs<double>&, cudaStream_t);
template cudaError_t Sized<double, 64>::pair_rows_counts(const Geom&, const PipeArgs<double>&, cudaStream_t);
template size_t Sized<double, 64>::rows_smem(int, bool);
template int Sized<double, 64>::rows_threads();
template cudaError_t Sized<double, 64>::rows_max_blocks(int, bool, int*);
template cudaError_t Sized<double, 128>::pair_rows(const Geom&, const PipeArgs<double>&, cudaStream_t);
template cudaError_t Sized<double, 128>::pair_rows_counts(const Geom&, const PipeArgs<double>&, cudaStream_t);
template size_t Sized<double, 128>::rows_smem(int, bool);
template int Sized<double, 128>::rows_threads();
template cudaError_t Sized<double, 128>::rows_max_blocks(int, bool, int*);
template cudaError_t Sized<double, 256>::pair_rows(const Geom&, const PipeArgs<double>&, cudaStream_t);
template cudaError_t Sized<double, 256>::pair_rows_counts(const Geom&, const PipeArgs<double>&, cudaStream_t);
template size_t Sized<double, 256>::rows_smem(int, bool);
template int Sized<double, 256>::rows_threads();
template cudaError_t Sized<double, 256>::rows_max_blocks(int, bool, int*);
}
