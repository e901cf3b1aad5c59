// two-term FP32 row / entropy-epilogue kernels for transform size 512.
#include "pipeline_impl.cuh"
namespace cmif {
template cudaError_t Sized<df32, 512>::pair_rows(const Geom&, const PipeArgs<df32>&, cudaStream_t);
template cudaError_t Sized<df32, 512>::pair_rows_counts(const Geom&, const PipeArgs<df32>&, cudaStream_t);
template size_t Sized<df32, 512>::rows_smem(int, bool);
template int Sized<df32, 512>::rows_threads();
template cudaError_t Sized<df32, 512>::rows_max_blocks(int, bool, int*);
}
