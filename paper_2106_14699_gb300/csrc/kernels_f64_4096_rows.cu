// FP64 row / entropy-epilogue kernels for transform size 4096.
#include "pipeline_impl.cuh"
namespace cmif {
template cudaError_t Sized<double, 4096>::pair_rows(const Geom&, const PipeArgs<double>&, cudaStream_t);
template cudaError_t Sized<double, 4096>::pair_rows_counts(const Geom&, const PipeArgs<double>&, cudaStream_t);
template size_t Sized<double, 4096>::rows_smem(int, bool);
template int Sized<double, 4096>::rows_threads();
template cudaError_t Sized<double, 4096>::rows_max_blocks(int, bool, int*);
}
