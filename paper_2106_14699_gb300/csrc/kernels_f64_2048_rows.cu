// FP64 row / entropy-epilogue kernels for transform size 2048.
#include "pipeline_impl.cuh"
namespace cmif {
template cudaError_t Sized<double, 2048>::pair_rows(const Geom&, const PipeArgs<double>&, cudaStream_t);
template cudaError_t Sized<double, 2048>::pair_rows_counts(const Geom&, const PipeArgs<double>&, cudaStream_t);
template size_t Sized<double, 2048>::rows_smem(int, bool);
template int Sized<double, 2048>::rows_threads();
template cudaError_t Sized<double, 2048>::rows_max_blocks(int, bool, int*);
}
