// FP64 row / entropy-epilogue kernels for transform size 1024.
#include "pipeline_impl.cuh"
namespace cmif {
template cudaError_t Sized<double, 1024>::pair_rows(const Geom&, const PipeArgs<double>&, cudaStream_t);
template cudaError_t Sized<double, 1024>::pair_rows_counts(const Geom&, const PipeArgs<double>&, cudaStream_t);
template size_t Sized<double, 1024>::rows_smem(int, bool);
template int Sized<double, 1024>::rows_threads();
template cudaError_t Sized<double, 1024>::rows_max_blocks(int, bool, int*);
}
